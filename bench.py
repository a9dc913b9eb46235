"""Benchmark of the per-frame path on the crowd composition (select + project + sort + blend).

Workload: 10 synthetic assets of 1M leaf Gaussians (4-ary hierarchies, FP32 attributes, SH degree
3), 1000 instances on a 200 x 200 ground, 1920x1080, horizontal fov 45 deg, tau = 1 px, camera
walking a 300-frame circle.  One step = one frame (v3dg_select + v3dg_render) at the next walk
frame.  Multi-GPU: replicas (each rank renders its own walk frames; no collective on the path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_ASSETS = 10
N_LEAVES = 1_000_000
N_INST = 1000
WIDTH, HEIGHT = 1920, 1080
TAU_PX = 1.0
STAGES = ["select", "project", "depth_sort", "bin", "tile_sort", "ranges", "blend"]
METRIC = "crowd 1080p frames/s & p99 latency, served vs plain, PSNR>=50dB vs FP64 oracle"
WORKLOAD = "crowd: 10 assets x 1M leaves (FP32, SH3), 1000 instances, 1920x1080, fov 45, tau 1 px, 300-frame walk"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tau", type=float, default=TAU_PX)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--assets", type=int, default=N_ASSETS, help="fewer assets: a smaller case for profiling")
    ap.add_argument("--instances", type=int, default=N_INST, help="fewer instances: a smaller case for profiling")
    ap.add_argument("--slots", type=int, default=4, help="server slots of the served leg (0: no served leg)")
    ap.add_argument("--serve-requests", type=int, default=150)
    ap.add_argument("--views", type=int, default=8, help="views per launch of the batched leg (0: none)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_frames(rank: int, world: int, count: int, frames: int = 300) -> list[int]:
    """Walk frames rendered by one replica: each rank starts at its own offset (no collective)."""
    return [(rank * 37 + 7 * s) % frames for s in range(count)]


def max_over_ranks(value: float, world: int) -> float:
    """Largest value over all ranks (the slowest replica sets the time); identity for one rank."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def load_scene(n_assets=N_ASSETS, n_inst=N_INST):
    from synth import scenes
    from synth.assets import cached_assets
    assets = cached_assets(list(range(n_assets)), N_LEAVES)
    inst = scenes.crowd_instances(n_inst, n_assets=n_assets)
    return assets, inst


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 7:
                continue
            try:
                sm.append(float(p[0]))
                mx = float(p[1])
            except ValueError:
                continue
            for n, v in zip(names, p[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def cpu_baseline(assets, inst, tau, frame_t=0, inst_frac=0.1, n_pix=16, seed=0):
    """The FP64 oracle on a bounded sample of one crowd frame, extrapolated to a whole frame.

    Sample: for a random fraction of the instances, selection, projection of their cut and the
    per-pixel blend of a few random pixels over those Gaussians; selection and projection scale
    with 1 / fraction, the blend with the pixel count and 1 / fraction.  Returns frames/s, seconds
    spent, description.
    """
    import oracle
    from synth import scenes
    cam = scenes.crowd_camera(frame_t)
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(inst.n, size=max(1, int(round(inst.n * inst_frac))), replace=False))
    sub_inst = scenes.subset(inst, pick)
    t0 = time.perf_counter()
    cut = oracle.select(assets, sub_inst, cam, tau)
    t_sel = time.perf_counter() - t0
    t1 = time.perf_counter()
    proj = oracle.project(assets, sub_inst, cam, cut)
    t_proj = time.perf_counter() - t1
    pix = [(int(rng.integers(0, WIDTH)), int(rng.integers(0, HEIGHT))) for _ in range(n_pix)]
    t2 = time.perf_counter()
    oracle.render_pixels(proj, pix)
    t_pix = time.perf_counter() - t2
    scale = inst.n / len(pick)
    frame_s = (t_sel + t_proj) * scale + t_pix * scale * (WIDTH * HEIGHT / n_pix)
    desc = (f"walk frame {frame_t}, {len(pick)} random instances of {inst.n}: select ({t_sel:.2f} s) and project "
            f"their cut ({t_proj:.2f} s), both x{scale:.0f}; blend {n_pix} random pixels ({t_pix:.2f} s, "
            f"x{WIDTH * HEIGHT / n_pix * scale:.3g}); whole frame extrapolated to {frame_s:.0f} s")
    return 1.0 / frame_s, t_sel + t_proj + t_pix, desc


REF_RUN_S = 180.0   # oracle work of the whole reference run (warm-up and timed steps), seconds


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return
    assets, inst = load_scene()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    # each step samples enough instances for about REF_RUN_S / (warmup + steps) seconds of oracle
    # work (2% of the instances take about 17 s), so the whole run ends within a few minutes
    per_step_s = max(1.0, REF_RUN_S / max(1, args.warmup + args.steps))
    frac = min(0.02, max(1.0 / inst.n, 0.02 * per_step_s / 17.0))
    vals, spent, desc = [], 0.0, ""
    for s in range(args.warmup + args.steps):
        v, sec, desc = cpu_baseline(assets, inst, args.tau, frame_t=(7 * s) % 300, seed=s, inst_frac=frac, n_pix=4)
        if s >= args.warmup:
            vals.append(v)
            spent += sec
    fps = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / fps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "tau_px": args.tau},
            "cpu_baseline": {"kind": "oracle", "value": fps, "unit": "frames/s", "cores": 1,
                             "sample": "per step: " + desc + f"; host has {cores} cores, numpy runs on 1"},
            "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo", rank=rank, world_size=world)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2505_06523_gb300 import Context
    from paper_2505_06523_gb300 import _native as N
    from synth import scenes

    assets, inst = load_scene(args.assets, args.instances)
    ctx = Context(local)
    for a in assets:
        ctx.load_hierarchy(a)
    inst16 = None
    if args.slots > 0:   # the served path's copies of the assets: opacity and SH stored as FP16
        ctx.set_option(N.V3DG_OPT_ATTR_FP16, 1)
        for a in assets:
            ctx.load_hierarchy(a)
        ctx.set_option(N.V3DG_OPT_ATTR_FP16, 0)
        inst16 = scenes.subset(inst, np.arange(inst.n))
        inst16.asset = inst16.asset + np.uint32(len(assets))
    ctx.set_instances(inst)
    cams = [scenes.crowd_camera(t) for t in range(300)]
    frame_ids = replica_frames(rank, world, args.warmup + args.steps)
    rgb = torch.empty((HEIGHT, WIDTH, 3), dtype=torch.float32, device=f"cuda:{local}")
    stream = ctx.stream

    # warm-up with checked frames, then one untimed checked pass over the frames the timed region
    # will render, so that every buffer has grown to its size; then run fully asynchronously
    for s in range(args.warmup):
        ctx.select(cams[frame_ids[s]], args.tau)
        ctx.render(rgb)
    for fid in sorted(set(frame_ids[args.warmup:])):
        ctx.select(cams[fid], args.tau)
        ctx.render(rgb)
    ctx.set_option(N.V3DG_OPT_SYNC_CHECK, 0)

    # timed region: K frames, CUDA events on the library's stream
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    n0 = ctx.launches()
    with ClockSampler(local) as clk:
        ev[0].record(stream)
        for s in range(args.steps):
            ctx.select(cams[frame_ids[args.warmup + s]], args.tau)
            ctx.render(rgb)
            ev[s + 1].record(stream)
        torch.cuda.synchronize()
    launches = ctx.launches() - n0
    per = [ev[s].elapsed_time(ev[s + 1]) for s in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    stats = ctx.frame_stats()   # overflow / timeout flags are sticky over every timed frame
    if stats["overflow"] or stats["timeout"]:
        raise RuntimeError(f"a frame of the timed region was invalid: {stats}")
    total_ms = max_over_ranks(total_ms, world)
    value = world * args.steps / (total_ms / 1000.0)

    # per-stage device times over the same frames: replay them with stage events (synchronous, so
    # the sum of the stages excludes the launch gaps that the asynchronous timed loop hides)
    timed_ids = frame_ids[args.warmup:]
    ctx.set_option(N.V3DG_OPT_SYNC_CHECK, 1)
    ctx.set_option(N.V3DG_OPT_STAGE_TIMING, 1)
    stage_runs = []
    for fid in timed_ids:
        ctx.select(cams[fid], args.tau)
        ctx.render(rgb)
        ms, _ = ctx.stage_times(len(STAGES))
        stage_runs.append(ms)
    # the same frames with the flat selection (the default walks large scenes top-down; same cut
    # and image, only the select stage differs)
    ctx.set_option(N.V3DG_OPT_SELECT_TOPDOWN, 0)
    flat_select = []
    for fid in timed_ids:
        ctx.select(cams[fid], args.tau)
        ctx.render(rgb)
        flat_select.append(ctx.stage_times(len(STAGES))[0][0])
    ctx.set_option(N.V3DG_OPT_SELECT_TOPDOWN, 2)
    ctx.set_option(N.V3DG_OPT_STAGE_TIMING, 0)
    stage_ms = {k: float(np.mean([r[i] for r in stage_runs])) for i, k in enumerate(STAGES)}
    # the blend's algorithmic work on the same frames (a separate, counting replay)
    ctx.set_option(N.V3DG_OPT_COUNT_WORK, 1)
    frame_tot = {k: 0 for k in ("cut_nodes", "cut_gaussians", "render_nodes", "visible", "pairs", "blend_evals",
                                "blend_contribs")}
    for fid in timed_ids:
        ctx.select(cams[fid], args.tau)
        ctx.render(rgb)
        st = ctx.frame_stats()
        for k in frame_tot:
            frame_tot[k] += st[k]
    ctx.set_option(N.V3DG_OPT_COUNT_WORK, 0)
    fs = {k: v / len(timed_ids) for k, v in frame_tot.items()}

    # e2e through the public API with host buffers: per step, the instance table (host FP64) goes
    # in, the camera is set, and the RGB image comes back into pinned host memory
    host_rgb = torch.empty((HEIGHT, WIDTH, 3), dtype=torch.float32, pin_memory=True).numpy()
    e2e_steps = max(3, args.e2e_steps)
    for s in range(3):
        ctx.set_instances(inst)
        ctx.select(cams[frame_ids[s % len(frame_ids)]], args.tau)
        ctx.render_host(host_rgb)
    t0 = time.perf_counter()
    for s in range(e2e_steps):
        ctx.set_instances(inst)
        ctx.select(cams[timed_ids[s % len(timed_ids)]], args.tau)
        ctx.render_host(host_rgb)
    e2e_s = time.perf_counter() - t0
    e2e_val = world * e2e_steps / max_over_ranks(e2e_s, world)
    h2d = inst.n * 256
    d2h = WIDTH * HEIGHT * 3 * 4

    served = None
    if args.slots > 0:
        # the autotuner times the blend of one FP16 walk frame with every batch size and split
        ctx.set_instances(inst16)
        ctx.select(cams[timed_ids[0]], args.tau)
        ctx.render(rgb)
        tuned = ctx.autotune_blend()
        ctx.set_instances(inst)
        served = serve_leg(ctx, inst, inst16, cams, timed_ids, args.tau, args.slots, args.serve_requests,
                           {"batch": tuned["batch"], "split_pairs": tuned["split_pairs"]})
        served["autotune"] = tuned
        served["psnr_fp16_vs_fp32_db"] = fp16_psnr(ctx, inst, inst16, cams, timed_ids, args.tau)
        if args.views > 0:
            served["batched"] = batched_leg(ctx, inst, inst16, cams, timed_ids, args.tau, args.views, tuned)

    peaks, peak_kind = measured_peaks()
    dom = max(stage_ms, key=stage_ms.get)
    roofline = roofline_for(dom, stage_ms, fs, peaks, peak_kind)

    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            v, spent, desc = cpu_baseline(assets, inst, args.tau, inst_frac=0.02, n_pix=16)
            cpu = {"value": v, "unit": "frames/s", "cores": 1, "kind": "oracle",
                   "sample": desc + f" ({spent:.0f} s of CPU work, single-threaded numpy)"}
        line = {
            "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if (args.assets, args.instances) == (N_ASSETS, N_INST) else
                       f"profiling case: {args.assets} assets, {args.instances} instances", "tau_px": args.tau,
                       "path": "plain FP32, one frame at a time",
                       "parallelism": f"replicas x{world}", "l2": "inputs larger than L2 (3.1 GB of attributes; "
                       "per-frame gathers of the selected Gaussians exceed the 129 MB L2)"},
            "p50_ms": float(np.percentile(per, 50)), "p99_ms": float(np.percentile(per, 99)),
            "e2e": {"value": e2e_val, "unit": "frames/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "served": served,
            "gpu_launches": int(launches),
            "stages_ms": stage_ms,
            "select_flat_ms": float(np.mean(flat_select)),
            "frame_mean": {k: int(round(v)) for k, v in fs.items()},
            "stages_sum_ms": float(sum(stage_ms.values())),
            "roofline": roofline,
            "cpu_baseline": cpu,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def _wait(ctx, ticket):
    r = None
    while r is None:
        r = ctx.poll(ticket, 100_000)
    return r[0]


def _closed_loop(ctx, inst, cam_of, tau, inflight_n, n_req):
    """`inflight_n` requests always in flight: frames/s over the run, per-request latencies."""
    lat, t0 = [], time.perf_counter()
    inflight = [ctx.submit(inst, cam_of(k), tau) for k in range(min(inflight_n, n_req))]
    nxt = len(inflight)
    while inflight:
        rec = _wait(ctx, inflight.pop(0))
        lat.append(rec["done_ms"] - rec["submit_ms"])
        if nxt < n_req:
            inflight.append(ctx.submit(inst, cam_of(nxt), tau))
            nxt += 1
    return n_req / (time.perf_counter() - t0), lat


def _open_loop(ctx, inst, cam_of, tau, arrivals):
    """Requests submitted at the given arrival times (s): latencies (submit -> done) and the rate
    achieved over the run."""
    pending, lat = [], []
    t0 = time.perf_counter()
    k, n_req = 0, len(arrivals)
    while k < n_req or pending:
        now = time.perf_counter() - t0
        while k < n_req and arrivals[k] <= now:
            pending.append(ctx.submit(inst, cam_of(k), tau))
            k += 1
        still = []
        for t in pending:
            r = ctx.poll(t, 0)
            if r is None:
                still.append(t)
            else:
                lat.append(r[0]["done_ms"] - r[0]["submit_ms"])
        pending = still
        if pending or k < n_req:
            time.sleep(0.0005)
    return n_req / (time.perf_counter() - t0), lat


def _pcts(lat):
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))}


DEFAULT_BLEND = {"batch": 512, "split_pairs": 0xFFFFFFFF}


def _blend_options(ctx, opts):
    from paper_2505_06523_gb300 import _native as N
    ctx.set_option(N.V3DG_OPT_BLEND_BATCH, opts["batch"])
    ctx.set_option(N.V3DG_OPT_SPLIT_PAIRS, opts["split_pairs"])


def serve_leg(ctx, inst, inst16, cams, frame_ids, tau, slots, n_req, tuned):
    """Served vs plain on the same request streams, through the library's server (v3dg_submit /
    v3dg_poll) with host buffers (instances in, image back into pinned host memory).

    plain:  one slot, FP32 attributes, default blend options -- serial one-request-at-a-time
            rendering;
    served: `slots` slots whose frames overlap on the GPU, opacity and SH stored as FP16, blend
            batch and split threshold from the autotuner (`tuned`).
    closed: as many requests in flight as slots (frames/s = capacity); poisson: open-loop Poisson
    arrivals at 50% and 90% of the plain capacity, the same arrival times and frames for both."""
    cam_of = lambda k: cams[frame_ids[k % len(frame_ids)]]
    arms = {"plain": (1, inst, "FP32 attributes, 1 slot", DEFAULT_BLEND),
            "served": (slots, inst16, f"FP16 colour, {slots} slots, autotuned blend", tuned)}
    out = {"requests": n_req, "frames": "the timed walk frames, 1000 instances, 1080p, host buffers"}
    cap = {}
    for name, (k, ins, desc, bopts) in arms.items():
        _blend_options(ctx, bopts)
        ctx.server_start(k)
        for t in [ctx.submit(ins, cam_of(j), tau) for j in range(2 * k)]:   # slots grow their buffers
            _wait(ctx, t)
        fps, lat = _closed_loop(ctx, ins, cam_of, tau, k, n_req)
        ctx.server_stop()
        cap[name] = fps
        out[name] = {"path": desc, "closed": {"value": fps, "unit": "frames/s", **_pcts(lat)}, "poisson": []}
    rng = np.random.default_rng(7)
    for load in (0.5, 0.9):
        rate = load * cap["plain"]
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
        for name, (k, ins, _, bopts) in arms.items():
            _blend_options(ctx, bopts)
            ctx.server_start(k)
            for t in [ctx.submit(ins, cam_of(j), tau) for j in range(k)]:
                _wait(ctx, t)
            achieved, lat = _open_loop(ctx, ins, cam_of, tau, arrivals)
            ctx.server_stop()
            out[name]["poisson"].append({"rate": rate, "achieved": achieved, **_pcts(lat)})
    _blend_options(ctx, DEFAULT_BLEND)
    out["served_vs_plain"] = {
        "frames_per_s": cap["served"] / cap["plain"],
        "p99_at_90pct_load": out["served"]["poisson"][1]["p99_ms"] / out["plain"]["poisson"][1]["p99_ms"]}
    return out


def batched_leg(ctx, inst, inst16, cams, frame_ids, tau, views, tuned):
    """Frames in batches: `views` consecutive walk frames per v3dg_select_views + v3dg_render
    (every stage one launch for all of them), replayed as a CUDA graph, FP16 colour, autotuned
    blend; device images.  frames/s = views x batches / time (CUDA events), beside the same frames
    one at a time with the same options."""
    import torch
    from paper_2505_06523_gb300 import _native as N
    _blend_options(ctx, tuned)
    ctx.set_instances(inst16)
    ctx.set_option(N.V3DG_OPT_GRAPHS, 1)
    groups = [[cams[(f + v) % len(cams)] for v in range(views)] for f in frame_ids[:6]]
    out = torch.empty((views, HEIGHT, WIDTH, 3), dtype=torch.float32, device="cuda")
    for g in groups[:2]:   # buffers grow, the graph is captured
        ctx.select_views(g, tau)
        ctx.render(out)
    ctx.set_option(N.V3DG_OPT_SYNC_CHECK, 0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(ctx.stream)
    for g in groups:
        ctx.select_views(g, tau)
        ctx.render(out)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    batched_ms = e0.elapsed_time(e1)
    st = ctx.frame_stats()
    one = torch.empty((HEIGHT, WIDTH, 3), dtype=torch.float32, device="cuda")
    for g in groups[:1]:
        for cam in g:
            ctx.select(cam, tau)
            ctx.render(one)
    torch.cuda.synchronize()
    e0.record(ctx.stream)
    for g in groups:
        for cam in g:
            ctx.select(cam, tau)
            ctx.render(one)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    single_ms = e0.elapsed_time(e1)
    ctx.set_option(N.V3DG_OPT_SYNC_CHECK, 1)
    ctx.set_option(N.V3DG_OPT_GRAPHS, 0)
    ctx.set_instances(inst)
    _blend_options(ctx, DEFAULT_BLEND)
    if st["overflow"] or st["timeout"]:
        raise RuntimeError(f"a batched frame was invalid: {st}")
    n = views * len(groups)
    return {"views_per_launch": views, "frames": n, "path": "FP16 colour, autotuned blend, CUDA graph",
            "value": n / (batched_ms / 1000.0), "unit": "frames/s",
            "same_frames_one_at_a_time": n / (single_ms / 1000.0)}


def fp16_psnr(ctx, inst, inst16, cams, frame_ids, tau):
    """PSNR (peak 1) of the FP16-colour image against the FP32 one, per walk frame (device images;
    the FP32 path itself is within 1e-4 of the FP64 oracle in the tests)."""
    import torch
    vals = []
    for f in sorted(set(frame_ids))[:4]:
        img = []
        for ins in (inst, inst16):
            ctx.set_instances(ins)
            ctx.select(cams[f], tau)
            img.append(ctx.render()[0].double())
        mse = float(((img[0] - img[1]) ** 2).mean())
        vals.append(float("inf") if mse == 0 else 10.0 * np.log10(1.0 / mse))
        del img
    ctx.set_instances(inst)
    torch.cuda.synchronize()
    return vals


# FP32 lanes of the GB300 (152 SMs x 128) at the maximum SM clock: the issue peak of the blend
FP32_LANES = 152 * 128
# algorithmic FP32 operations of the blend: per (pixel, Gaussian) evaluated inside the Gaussian's
# pixel box (dx, dy, the quadratic form, the skip test) and per contribution (exp2, clamp, skip
# test, 1 - alpha, T update, stop test, weight, three colour FMAs)
BLEND_OPS_EVAL, BLEND_OPS_CONTRIB = 8, 10


# DRAM bytes per unit from one ncu capture of the same kernel on the crowd's profiling case (2
# assets, 300 instances): dram__bytes_read.sum + dram__bytes_write.sum of one launch / the units
# of its frame.  Scaled to a full launch by the units processed (traffic grows with them).
NCU_DRAM_PER_UNIT = {
    "blend": (7.21, "pair", "profiles/k_blend_crowd_small.md"),      # (250.3 + 6.2) MB / 35.6M pairs
    "project": (220.0, "slot", "profiles/k_project_crowd_small.md"),  # (2,999.5 + 854.7) MB / 17.5M slots
    "bin": (11.84, "pair", "profiles/k_expand_crowd_small.md"),       # (175.4 + 245.8) MB / 35.6M pairs
}


def roofline_for(stage, stage_ms, fs, peaks, peak_kind):
    """Algorithmic work per launch of every stage (means over the timed frames) over its mean
    measured duration; the top-level fields are those of the dominant stage."""
    vis, pairs, nodes = fs["visible"], fs["pairs"], fs["render_nodes"]
    slots = nodes * 64
    units = {"pair": pairs, "slot": slots}
    bytes_per = {
        # selection: the node tables are L2-resident; HBM traffic is the render list write
        "select": 8 * nodes,
        # projection: 236 B of attributes per slot read, 48 B record + 8 B rect + 4 B key written
        "project": 236 * slots + (48 + 8 + 4) * vis + 4 * (slots - vis),
        # depth sort: 4 passes of (key, value) read + write, plus the histogram read
        "depth_sort": slots * (4 * 16 + 4),
        # binning: sorted slots + pixel boxes read, pairs written
        "bin": vis * (4 + 8) + pairs * 8,
        # tile sort: 2 passes of (key, value) read + write, plus the histogram read
        "tile_sort": pairs * (2 * 16 + 4),
        "ranges": pairs * 4 + 8 * 8160,
    }
    hbm_peak = float(peaks["hbm_gbs"])
    per_stage = {k: {"bound": "hbm", "gbs": v / (stage_ms[k] / 1000.0) / 1e9, "frac": v / (stage_ms[k] / 1000.0) / 1e9 / hbm_peak,
                     "ms": stage_ms[k]} for k, v in bytes_per.items() if stage_ms.get(k)}
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = FP32_LANES * mhz * 1e6 / 1e12
    if fs.get("blend_evals") and stage_ms.get("blend"):
        ops = BLEND_OPS_EVAL * fs["blend_evals"] + BLEND_OPS_CONTRIB * fs["blend_contribs"]
        tf = ops / (stage_ms["blend"] / 1000.0) / 1e12
        per_stage["blend"] = {"bound": "alu", "tflops": tf, "frac": tf / alu_peak, "ms": stage_ms["blend"]}

    def traffic(st):   # DRAM bytes per launch, from the ncu capture scaled by the units processed
        if st not in NCU_DRAM_PER_UNIT:
            return None
        per, unit, _ = NCU_DRAM_PER_UNIT[st]
        return per * units[unit]

    def traffic_source(st):
        if st not in NCU_DRAM_PER_UNIT:
            return None
        per, unit, src = NCU_DRAM_PER_UNIT[st]
        return {"bytes_per_unit": per, "unit": unit, "from": src}

    # the frame's roofline: each stage at its own bound (HBM bytes at the copy bandwidth, the blend's
    # FP32 operations at the issue peak), summed, against the measured stage times
    ideal_ms = sum(v / (hbm_peak * 1e9) * 1e3 for k, v in bytes_per.items() if k in per_stage)
    if "blend" in per_stage:
        ideal_ms += per_stage["blend"]["tflops"] * per_stage["blend"]["ms"] / alu_peak
    frame = {"ideal_ms": ideal_ms, "measured_ms": sum(v["ms"] for v in per_stage.values()),
             "frac": ideal_ms / max(sum(v["ms"] for v in per_stage.values()), 1e-9)}
    ms = stage_ms[stage]
    if stage == "blend" and "blend" in per_stage:
        return {"stage": "blend", "kernel": "k_blend", "bound": "alu", "achieved": per_stage["blend"]["tflops"],
                "peak": alu_peak, "unit": "TFLOP/s", "frac": per_stage["blend"]["frac"], "traffic": traffic("blend"),
                "traffic_source": traffic_source("blend"),
                "peak_source": f"derived: {FP32_LANES} FP32 lanes x {mhz:.0f} MHz (MEASURED_PEAKS sm_max_mhz)",
                "work": {"evals": fs["blend_evals"], "contribs": fs["blend_contribs"],
                         "ops_per_eval": BLEND_OPS_EVAL, "ops_per_contrib": BLEND_OPS_CONTRIB, "ms": ms},
                "per_stage": per_stage, "frame": frame}
    kernel = {"select": "k_select", "project": "k_project", "depth_sort": "k_onesweep", "bin": "k_expand",
              "tile_sort": "k_onesweep", "ranges": "k_ranges"}[stage]
    return {"stage": stage, "kernel": kernel, "bound": "hbm", "achieved": per_stage[stage]["gbs"], "peak": hbm_peak,
            "unit": "GB/s", "frac": per_stage[stage]["frac"], "traffic": traffic(stage),
            "traffic_source": traffic_source(stage), "peak_source": peak_kind,
            "per_stage": per_stage, "frame": frame}


if __name__ == "__main__":
    main()
