"""The multi-GPU path is replicas: each rank renders its own frames; only the timing is reduced.

Runs the bench's host-side replica logic on two gloo ranks on the CPU.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    frames = bench.replica_frames(rank, world, 12)
    slowest = bench.max_over_ranks(10.0 + rank, world)
    dist.destroy_process_group()
    q.put((rank, frames, slowest))


def test_two_replicas_on_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict((r, (f, m)) for r, f, m in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank renders a full set of its own frames, in range, and the ranks' sets differ
    assert all(len(out[r][0]) == 12 and all(0 <= f < 300 for f in out[r][0]) for r in (0, 1))
    assert out[0][0] != out[1][0]
    # the job's time is the slowest rank's
    assert out[0][1] == out[1][1] == 11.0


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.replica_frames(0, 1, 3) == [0, 7, 14]
