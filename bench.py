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
    ap.add_argument("--serve-requests", type=int, default=600)
    ap.add_argument("--views", type=int, default=16, help="views per launch of the batched leg (0: none)")
    ap.add_argument("--no-extra-legs", action="store_true", help="skip the orbit table and the no-LOD comparison")
    ap.add_argument("--mix-seconds", type=float, default=2.5,
                    help="seconds of Poisson arrivals per rate of the serving mix (config 5; 0: no mix leg)")
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


# ---------------------------------------------------------------- the oracle on the host cores
# The FP64 oracle (oracle/) timed on all host cores: a pool of spawned worker processes (no CUDA in
# them) renders bands of rows of a frame and selects and projects instances in parallel.


def host_cores() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def oracle_pool(cores: int):
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(cores)


_ASSET = {}


def _asset(seed: int, n_leaves: int):
    """The worker's assets, at most three at a time (each is ~0.5 GB in host memory)."""
    if (seed, n_leaves) not in _ASSET:
        from synth.assets import cached_asset
        while len(_ASSET) >= 3:
            _ASSET.pop(next(iter(_ASSET)))
        _ASSET[(seed, n_leaves)] = cached_asset(seed, n_leaves)
    return _ASSET[(seed, n_leaves)]


def _w_band(args):
    """Worker: a region of a frame by the per-pixel definition."""
    import oracle
    p_sub, width, height, region = args
    return region, oracle.render_image(p_sub, width, height, region=region)


def _near_windows(p, windows):
    """Gaussians whose widened pixel box (the oracle's +-2 px) overlaps one of the windows."""
    hit = np.zeros(len(p.inst), bool)
    for x0, y0, x1, y1 in windows:
        hit |= (p.pix[:, 0] - 2 <= x1) & (p.pix[:, 1] + 2 >= x0) & (p.pix[:, 2] - 2 <= y1) & (p.pix[:, 3] + 2 >= y0)
    return np.nonzero(hit & p.visible)[0]


def _w_instances(args):
    """Worker: selection and projection of some instances of one asset, each timed on its own
    (asset loading excluded); returns the times, the visible counts and a random sample of at most
    `keep` visible Gaussians per instance."""
    import oracle
    from synth import scenes
    seed, n_leaves, ids, inst, cam, tau, keep = args
    asset = _asset(seed, n_leaves)
    times, n_vis, parts = [], [], []
    for k, i in enumerate(ids):
        one = scenes.subset(inst, [k])
        one.asset[:] = 0
        t0 = time.perf_counter()
        cut = oracle.select([asset], one, cam, tau)
        p = oracle.project([asset], one, cam, cut)
        times.append(time.perf_counter() - t0)
        vis = np.nonzero(p.visible)[0]
        n_vis.append(len(vis))
        pick = np.random.default_rng(i).choice(vis, size=min(keep, len(vis)), replace=False) if len(vis) else vis
        sub = oracle.subset_projected(p, np.sort(pick))
        sub.inst[:] = i
        parts.append(sub)
    return times, n_vis, parts


def _render_frame_parallel(pool, p, width, height, band=16):
    import oracle
    tasks = []
    for y0 in range(0, height, band):
        y1 = min(y0 + band - 1, height - 1)
        idx = _near_windows(p, [(0, y0, width - 1, y1)])
        tasks.append((oracle.subset_projected(p, idx), width, height, (0, y0, width - 1, y1)))
    C = np.zeros((height, width, 3))
    for (x0, y0, x1, y1), (c, _, _) in pool.imap_unordered(_w_band, tasks):
        C[y0:y1 + 1] = c
    return C


def oracle_config1(pool, frames: int = 2):
    """Config 1 (100k leaves, 256x256, fov 60, distance 3, tau 1 px), whole frames measured end
    to end: selection and projection, then the image in bands of 16 rows over the pool."""
    import oracle
    from synth import scenes
    from synth.assets import cached_asset
    asset = cached_asset(0, 100_000)
    inst = scenes.single_instance()
    cam = scenes.tiny_camera()
    t0 = time.perf_counter()
    for _ in range(frames):
        cut = oracle.select([asset], inst, cam, 1.0)
        p = oracle.project([asset], inst, cam, cut)
        _render_frame_parallel(pool, p, cam.width, cam.height)
    dt = time.perf_counter() - t0
    return frames / dt, dt


def oracle_crowd_sample(pool, cores, assets_n, inst, tau, frame_t, n_sample, seed, n_leaves=N_LEAVES, keep=2000):
    """One crowd frame estimated from a sample.  n_sample random instances are selected and
    projected on the pool (each timed by its worker); then a random sample of their visible
    Gaussians is rendered over the whole frame by the per-pixel definition (Gaussian by Gaussian,
    whose cost grows with the number of Gaussians).  Selection and projection scale with the
    instances, the image with the visible Gaussians, and both divide over the cores: an
    extrapolation.  Returns (frames/s, wall s, description)."""
    import oracle
    from synth import scenes
    cam = scenes.crowd_camera(frame_t)
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(inst.n, size=min(n_sample, inst.n), replace=False))
    tasks = []
    for a in range(assets_n):
        ids = pick[inst.asset[pick] == a]
        for chunk in np.array_split(ids, max(1, min(len(ids), 2))):
            if len(chunk):
                tasks.append((a, n_leaves, chunk.tolist(), scenes.subset(inst, chunk), cam, tau, keep))
    t0 = time.perf_counter()
    times, n_vis, parts = [], [], []
    for tt, nv, pp in pool.imap_unordered(_w_instances, tasks):
        times += tt
        n_vis += nv
        parts += pp
    t_par = time.perf_counter() - t0
    fields = oracle.Projected.__dataclass_fields__
    p = oracle.Projected(**{k: np.concatenate([getattr(q, k) for q in parts]) for k in fields})
    t1 = time.perf_counter()
    oracle.render_image(p, WIDTH, HEIGHT)
    t_img = time.perf_counter() - t1
    scale = inst.n / len(pick)
    per_g = t_img / max(1, len(p.inst))
    frame_s = (sum(times) * scale + per_g * sum(n_vis) * scale) / cores
    desc = (f"walk frame {frame_t}: {len(pick)} random instances of {inst.n} selected and projected on the pool "
            f"({sum(times):.1f} CPU-s, x{scale:.0f}); {len(p.inst)} of their {sum(n_vis)} visible Gaussians "
            f"rendered over the whole frame ({t_img:.2f} s, {per_g * 1e6:.0f} us per Gaussian, x{sum(n_vis) * scale:.3g} "
            f"Gaussians); extrapolated to {frame_s:.0f} s per frame on {cores} cores")
    return 1.0 / frame_s, t_par + t_img, desc


def cpu_baseline_leg(assets_n, inst, tau):
    """The oracle on all host cores: config 1 whole frames (measured) and the crowd walk frames
    0, 150, 299 (extrapolated from samples)."""
    cores = host_cores()
    with oracle_pool(cores) as pool:
        c1_fps, c1_s = oracle_config1(pool)
        vals, spent, descs = [], 0.0, []
        for t in (0, 150, 299):
            v, sec, d = oracle_crowd_sample(pool, cores, assets_n, inst, tau, t, n_sample=cores, seed=t)
            vals.append(v)
            spent += sec
            descs.append(d)
    return {"value": float(np.mean(vals)), "unit": "frames/s", "cores": cores, "kind": "oracle",
            "extrapolated": True,
            "sample": "; ".join(descs) + f" ({spent:.0f} s wall)",
            "config1_measured": {"value": c1_fps, "unit": "frames/s", "frames": 2, "seconds": c1_s,
                                 "workload": "config 1: 100k leaves, 256x256, fov 60, distance 3, tau 1 px, "
                                             "whole frames (selection, projection, image in 16-row bands on the pool)"}}


REF_RUN_S = 150.0   # wall time of the whole reference run (warm-up and timed steps), seconds


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle on all host cores (rank 0 only), one crowd walk frame
    per step, each extrapolated from a sample of instances and pixels sized from the step count."""
    if rank != 0:
        return
    assets, inst = load_scene()
    cores = host_cores()
    steps = max(1, args.warmup + args.steps)
    # about 1 s of wall time per sampled instance per core (selection and projection on the Grace
    # host), so the whole run stays near REF_RUN_S
    n_sample = int(min(4 * cores, max(cores // 2, REF_RUN_S / steps * cores / 2)))
    vals, spent, desc = [], 0.0, ""
    with oracle_pool(cores) as pool:
        for s in range(steps):
            v, sec, desc = oracle_crowd_sample(pool, cores, len(assets), inst, args.tau, (7 * s) % 300, n_sample, s)
            if s >= args.warmup:
                vals.append(v)
                spent += sec
    fps = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / fps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "tau_px": args.tau},
            "cpu_baseline": {"kind": "oracle", "value": fps, "unit": "frames/s", "cores": cores, "extrapolated": True,
                             "sample": "per step: " + desc},
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
    # the same frames with the flat selection and the projection in list order (the defaults walk
    # large scenes top-down and project the render list grouped by cluster; same cut, records and
    # image, only the select and project stages differ)
    ctx.set_option(N.V3DG_OPT_SELECT_TOPDOWN, 0)
    ctx.set_option(N.V3DG_OPT_PROJECT_ORDER, 0)
    flat_select, list_project = [], []
    for fid in timed_ids:
        ctx.select(cams[fid], args.tau)
        ctx.render(rgb)
        ms, _ = ctx.stage_times(len(STAGES))
        flat_select.append(ms[0])
        list_project.append(ms[1])
    ctx.set_option(N.V3DG_OPT_SELECT_TOPDOWN, 2)
    ctx.set_option(N.V3DG_OPT_PROJECT_ORDER, 2)
    ctx.set_option(N.V3DG_OPT_STAGE_TIMING, 0)
    stage_ms = {k: float(np.mean([r[i] for r in stage_runs])) for i, k in enumerate(STAGES)}
    # the blend's algorithmic work on the same frames (a separate, counting replay)
    ctx.set_option(N.V3DG_OPT_COUNT_WORK, 1)
    frame_tot = {k: 0 for k in ("cut_nodes", "cut_gaussians", "render_nodes", "render_clusters", "visible", "pairs",
                                "blend_evals", "blend_contribs")}
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

    served, view_samples = None, []
    if args.slots > 0:
        # the autotuner times the blend of one FP16 walk frame with every batch size and split
        ctx.set_instances(inst16)
        ctx.select(cams[timed_ids[0]], args.tau)
        ctx.render(rgb)
        tuned = ctx.autotune_blend()
        ctx.set_instances(inst)
        served = serve_leg(ctx, inst, inst16, cams, timed_ids, args.tau, args.slots, args.serve_requests,
                           {"mode": tuned["mode"], "batch": tuned["batch"], "split_pairs": tuned["split_pairs"]})
        served["autotune"] = tuned
        served["psnr_fp16_vs_fp32_db"] = fp16_psnr(ctx, inst, inst16, cams, timed_ids, args.tau)
        if args.mix_seconds > 0:
            sc32 = mix_scenes(inst, len(assets))
            sc16 = {k: scenes.subset(v, np.arange(v.n)) for k, v in sc32.items()}
            for v in sc16.values():
                v.asset = v.asset + np.uint32(len(assets))
            served["mix"] = serve_mix_leg(ctx, sc32, sc16, args.slots,
                                          {"mode": tuned["mode"], "batch": tuned["batch"],
                                           "split_pairs": tuned["split_pairs"]}, args.mix_seconds)
        if args.views > 0:
            served["batched"], view_samples = batched_leg(ctx, inst, inst16, cams, timed_ids, (1.0, 2.0), args.views,
                                                          tuned)
            # the views' buffers (~100 GB at 16 crowd views) go back to the device before the next legs
            ctx.release_buffers()
            torch.cuda.empty_cache()

    extra = {}
    if not args.no_extra_legs:
        extra["vanilla"] = vanilla_leg(ctx, inst, cams, timed_ids, args.tau)
        extra["orbit"] = orbit_leg(ctx, 0)
        ctx.set_instances(inst)

    peaks, peak_kind = measured_peaks()
    dom = max(stage_ms, key=stage_ms.get)
    roofline = roofline_for(dom, stage_ms, fs, peaks, peak_kind)

    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            cpu = cpu_baseline_leg(len(assets), inst, args.tau)
            if view_samples:
                served["batched"]["per_view_vs_oracle"] = oracle_view_parity(view_samples, assets, inst)
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
            "v3dg_vs_vanilla": extra.get("vanilla"),
            "orbit": extra.get("orbit"),
            "gpu_launches": int(launches),
            "stages_ms": stage_ms,
            "select_flat_ms": float(np.mean(flat_select)),
            "project_list_order_ms": float(np.mean(list_project)),
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


DEFAULT_BLEND = {"mode": 0, "batch": 512, "split_pairs": 0xFFFFFFFF}


def _blend_options(ctx, opts):
    from paper_2505_06523_gb300 import _native as N
    ctx.set_option(N.V3DG_OPT_BLEND_MODE, opts["mode"])
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


MIX_RES = [(1280, 720), (1920, 1080), (3840, 2160)]
MIX_TAUS = [0.5, 1.0, 2.0, 4.0]
MIX_RATES = [30.0, 100.0, 250.0, 500.0]


def mix_scenes(inst1000, n_assets):
    """Config 5's scenes: 100 instances (the first of the crowd layout), the 1000-instance crowd,
    and 5000 (the crowd extended by 4000 more instances from the same generator, seed 1001)."""
    from synth import scenes
    ext = scenes.crowd_instances(4000, n_assets=n_assets, seed=1001)
    five = scenes.Instances(np.concatenate([inst1000.asset, ext.asset]), np.concatenate([inst1000.rot, ext.rot]),
                            np.concatenate([inst1000.trans, ext.trans]), np.concatenate([inst1000.scale, ext.scale]))
    return {100: scenes.subset(inst1000, np.arange(100)), 1000: inst1000, 5000: five}


def mix_requests(n, seed):
    """n requests drawn from config 5's mix: scene size, resolution, tau and walk frame."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        out.append((int(rng.choice([100, 1000, 5000])), MIX_RES[int(rng.integers(0, 3))],
                    float(MIX_TAUS[int(rng.integers(0, 4))]), int(rng.integers(0, 300))))
    return out


def serve_mix_leg(ctx, scenes_fp32, scenes_fp16, slots, tuned, seconds, max_outstanding=64, rates=MIX_RATES,
                  min_requests=500):
    """Config 5: Poisson arrivals at each rate for `seconds` (and at least `min_requests` arrivals),
    each request drawn from the mix
    (100 / 1000 / 5000 instances, 720p / 1080p / 4K, tau 0.5-4 px, a walk frame), images back into
    pinned host memory.  served: `slots` slots, FP16 colour, autotuned blend; served_merged: the
    same, and up to 8 waiting requests of one image size rendered as one frame while requests pile
    up; served_one_slot: FP16 colour and the autotuned blend on one slot (no frames side by side);
    plain: one slot, FP32 attributes, one request per frame, default blend (serial plain
    rendering of the same stream).  A client keeps at most
    max_outstanding requests in flight (host output buffers) and drops arrivals beyond that
    (counted).  Latency = submit -> done on the server's clock."""
    from paper_2505_06523_gb300 import _native as N
    from synth import scenes
    cams = {}

    def cam_of(res, f):
        if (res, f) not in cams:
            cams[(res, f)] = scenes.crowd_camera(f, res[0], res[1])
        return cams[(res, f)]

    out = {"seconds_per_rate": seconds, "max_outstanding": max_outstanding, "slots": slots, "rates": []}
    arms = {"plain": (1, 1, scenes_fp32, DEFAULT_BLEND), "served": (slots, 1, scenes_fp16, tuned),
            "served_merged": (slots, 8, scenes_fp16, tuned), "served_one_slot": (1, 1, scenes_fp16, tuned)}
    rng = np.random.default_rng(3000)
    for rate in rates:
        n = max(min_requests, int(round(rate * seconds)))   # arrivals at this rate (at least min_requests)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
        reqs = mix_requests(n, seed=int(rate))
        row = {"rate": rate, "requests": n}
        for name, (k, merge, sc, bopts) in arms.items():
            _blend_options(ctx, bopts)
            ctx.set_option(N.V3DG_OPT_SERVE_MERGE, merge)
            ctx.server_start(k)
            for (ni, res, tau, f) in reqs[:2 * k]:   # slots grow their buffers
                _wait(ctx, ctx.submit(sc[ni], cam_of(res, f), tau))
            pending, lat, dropped, failed, views = [], [], 0, {}, []
            cls_of, by_cls = {}, {}
            t0 = time.perf_counter()
            i = 0
            while i < n or pending:
                now = time.perf_counter() - t0
                while i < n and arrivals[i] <= now:
                    if len(pending) < max_outstanding:
                        ni, res, tau, f = reqs[i]
                        t = ctx.submit(sc[ni], cam_of(res, f), tau)
                        pending.append(t)
                        cls_of[t] = f"{ni}@{res[1]}p"
                    else:
                        dropped += 1
                    i += 1
                still = []
                for t in pending:
                    try:
                        r = ctx.poll(t, 0)
                    except N.V3dgError as e:   # a failed request: counted by its status, not timed
                        key = N.STATUS_NAMES[e.status] if 0 <= e.status < len(N.STATUS_NAMES) else str(e.status)
                        failed[key] = failed.get(key, 0) + 1
                        continue
                    if r is None:
                        still.append(t)
                    else:
                        lat.append(r[0]["done_ms"] - r[0]["submit_ms"])
                        views.append(r[0]["batch_views"])
                        by_cls.setdefault(cls_of.pop(t, "?"), []).append(r[0]["done_ms"] - r[0]["start_ms"])
                pending = still
                if pending or i < n:
                    time.sleep(0.0005)
            wall = time.perf_counter() - t0
            ctx.server_stop()
            row[name] = {"completed": len(lat), "dropped": dropped, "failed": failed, "achieved": len(lat) / wall,
                         "mean_views_per_frame": float(np.mean(views)) if views else 0.0, **_pcts(lat),
                         "service_ms_by_class": {k: round(float(np.mean(v)), 1) for k, v in sorted(by_cls.items())}}
        out["rates"].append(row)
    ctx.set_option(N.V3DG_OPT_SERVE_MERGE, 1)
    _blend_options(ctx, DEFAULT_BLEND)
    return out


def batched_leg(ctx, inst, inst16, cams, frame_ids, taus, views, tuned, n_groups=3):
    """Config 4: `views` consecutive walk frames per v3dg_select_views + v3dg_render (every stage one
    launch for all of them), replayed as a CUDA graph, FP16 colour, autotuned blend, device images,
    for each tau.  frames/s = views x batches / time (CUDA events), beside the same frames one at a
    time with the same options.  Per view: PSNR of the FP16 image against the FP32 one (device), and
    pixel samples of both (two 8x8 windows) that the oracle leg compares with the FP64 oracle."""
    import torch
    from paper_2505_06523_gb300 import _native as N
    out = {"views_per_launch": views, "path": "FP16 colour, autotuned blend, CUDA graph", "taus": {}}
    samples = []
    for tau in taus:
        _blend_options(ctx, tuned)
        ctx.set_instances(inst16)
        ctx.set_option(N.V3DG_OPT_GRAPHS, 1)
        groups = [[(f + v) % len(cams) for v in range(views)] for f in frame_ids[:n_groups]]
        img = torch.empty((views, HEIGHT, WIDTH, 3), dtype=torch.float32, device="cuda")
        for g in groups[:2]:   # buffers grow, the graph is captured
            ctx.select_views([cams[f] for f in g], tau)
            ctx.render(img)
        ctx.set_option(N.V3DG_OPT_SYNC_CHECK, 0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(ctx.stream)
        for g in groups:
            ctx.select_views([cams[f] for f in g], tau)
            ctx.render(img)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        batched_ms = e0.elapsed_time(e1)
        st = ctx.frame_stats()
        one = torch.empty((HEIGHT, WIDTH, 3), dtype=torch.float32, device="cuda")
        for f in groups[0]:
            ctx.select(cams[f], tau)
            ctx.render(one)
        torch.cuda.synchronize()
        e0.record(ctx.stream)
        for g in groups:
            for f in g:
                ctx.select(cams[f], tau)
                ctx.render(one)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        single_ms = e0.elapsed_time(e1)
        ctx.set_option(N.V3DG_OPT_SYNC_CHECK, 1)
        ctx.set_option(N.V3DG_OPT_GRAPHS, 0)
        if st["overflow"] or st["timeout"]:
            raise RuntimeError(f"a batched frame was invalid: {st}")
        # per view of the last batch: FP16 (the batched image) against FP32 (plain, one at a time)
        g = groups[-1]
        ctx.set_instances(inst)
        _blend_options(ctx, DEFAULT_BLEND)
        psnr, maxabs = [], []
        rng = np.random.default_rng(int(tau * 100))
        for v, f in enumerate(g):
            ctx.select(cams[f], tau)
            ref = ctx.render(one)[0]
            d = (img[v].double() - ref.double())
            mse = float((d ** 2).mean())
            psnr.append(float("inf") if mse == 0 else 10.0 * np.log10(1.0 / mse))
            maxabs.append(float(d.abs().max()))
            if v in (0, views - 1):
                drawn = torch.nonzero(ref.amax(dim=-1) > 0.05).cpu().numpy()
                wins = []
                for y, x in drawn[rng.choice(len(drawn), size=2, replace=False)]:
                    x0, y0 = int(min(max(x - 4, 0), WIDTH - 8)), int(min(max(y - 4, 0), HEIGHT - 8))
                    wins.append((x0, y0, x0 + 7, y0 + 7))
                pix = [(x, y) for x0, y0, x1, y1 in wins for y in range(y0, y1 + 1) for x in range(x0, x1 + 1)]
                i16, i32 = img[v].cpu().numpy(), ref.cpu().numpy()
                samples.append({"tau": tau, "view": v, "frame": f, "windows": wins, "pixels": pix,
                                "fp16": np.array([i16[y, x] for x, y in pix]),
                                "fp32": np.array([i32[y, x] for x, y in pix])})
        n = views * len(groups)
        out["taus"][f"{tau:g}"] = {"frames": n, "value": n / (batched_ms / 1000.0), "unit": "frames/s",
                                   "same_frames_one_at_a_time": n / (single_ms / 1000.0),
                                   "pairs_last_batch": st["pairs"], "visible_last_batch": st["visible"],
                                   "psnr_fp16_vs_fp32_db": psnr, "maxabs_fp16_vs_fp32": maxabs}
        del img
        torch.cuda.synchronize()
    ctx.set_instances(inst)
    _blend_options(ctx, DEFAULT_BLEND)
    return out, samples


def oracle_view_parity(samples, assets, inst):
    """Part of the oracle leg: the sampled pixels of the batched views against the FP64 oracle,
    on the FP32 attributes and on the FP16-rounded ones (what the FP16 path stores).  Per sample:
    PSNR and max abs error over the pixels outside the decision bands, for the FP16 image and for
    the plain FP32 image of the same frame."""
    import copy
    import oracle
    from synth import scenes

    def rounded(a):
        b = copy.copy(a)
        b.sh = a.sh.astype(np.float16).astype(np.float32)
        b.opacity = a.opacity.astype(np.float16).astype(np.float32)
        return b

    a16 = [rounded(a) for a in assets]
    rows = []
    for smp in samples:
        cam = scenes.crowd_camera(smp["frame"])
        row = {"tau": smp["tau"], "view": smp["view"], "frame": smp["frame"], "pixels": len(smp["pixels"])}
        for attrs, name in ((assets, "oracle_fp32_attrs"), (a16, "oracle_fp16_attrs")):
            cut = oracle.select(attrs, inst, cam, smp["tau"])
            sub, only = oracle.gaussians_reaching_pixels(attrs, inst, cam, cut, smp["pixels"], windows=smp["windows"])
            p = oracle.project(attrs, inst, cam, sub, only=only)
            c, _, b = oracle.render_pixels(p, smp["pixels"])
            for img in ("fp16", "fp32"):
                g = smp[img].astype(np.float64)
                mse = float(np.mean((g - c) ** 2))
                row[f"{img}_image_vs_{name}"] = {
                    "psnr_db": float("inf") if mse == 0 else 10.0 * np.log10(1.0 / mse),
                    "maxabs_outside_bands": float(np.abs(g - c).max(axis=1)[~b].max()) if (~b).any() else 0.0,
                    "band_pixels": int(b.sum())}
        rows.append(row)
    return rows


def _frame_ms(ctx, cams, tau, rgb, reps=1):
    """Mean device time (CUDA events on the library's stream) of select + render over the cameras,
    after one checked warm-up pass over them (buffers grown); also the last frame's counters."""
    import torch
    for cam in cams:
        ctx.select(cam, tau)
        ctx.render(rgb)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(ctx.stream)
    for _ in range(reps):
        for cam in cams:
            ctx.select(cam, tau)
            ctx.render(rgb)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / (reps * len(cams)), ctx.frame_stats()


def orbit_leg(ctx, asset_id):
    """Config 2: one 1M-leaf asset at 1920x1080, fov 45, elevation 30, eight orbit distances
    1.5 (50 / 1.5)^(k / 7), tau in {0.5, 1, 2, 4} px and tau = 0 (every leaf: the scene without
    LOD).  Per (distance, tau): cut clusters, selected and rendered (visible) Gaussians, pairs and
    the frame's device time."""
    import torch
    from synth import scenes
    one = scenes.single_instance()
    one.asset[:] = asset_id
    ctx.set_instances(one)
    rgb = torch.empty((HEIGHT, WIDTH, 3), dtype=torch.float32, device="cuda")
    rows = []
    for k, d in enumerate(scenes.orbit_distances()):
        cam = scenes.orbit_camera(d)
        row = {"k": k, "distance": d}
        for tau in (0.0, 0.5, 1.0, 2.0, 4.0):
            ms, st = _frame_ms(ctx, [cam], tau, rgb, reps=5)
            row[f"tau{tau:g}"] = {"ms": ms, "cut_nodes": st["cut_nodes"], "selected": st["cut_gaussians"],
                                  "rendered": st["visible"], "pairs": st["pairs"]}
        row["speedup_tau1_vs_tau0"] = row["tau0"]["ms"] / row["tau1"]["ms"]
        rows.append(row)
    return {"workload": "asset 0 (1M leaves), 1920x1080, fov 45, elevation 30, 8 distances, tau 0 (no LOD) and "
                        "0.5-4 px; ms = device time of select + render, mean of 5 frames", "rows": rows}


def vanilla_leg(ctx, inst, cams, frame_ids, tau):
    """The crowd with V3DG's cut against the same scene without LOD (tau = 0: every leaf cluster is
    selected), on the same walk frames: the paper's speed-up comparison (Sec. 5.3)."""
    import torch
    rgb = torch.empty((HEIGHT, WIDTH, 3), dtype=torch.float32, device="cuda")
    ctx.set_instances(inst)
    sel = [cams[f] for f in frame_ids[:8]]
    out = {}
    for name, t in (("v3dg", tau), ("vanilla", 0.0)):
        ms, st = _frame_ms(ctx, sel, t, rgb)
        out[name] = {"tau_px": t, "ms": ms, "frames_per_s": 1000.0 / ms, "selected_last": st["cut_gaussians"],
                     "rendered_last": st["visible"], "pairs_last": st["pairs"]}
    out["speedup"] = out["vanilla"]["ms"] / out["v3dg"]["ms"]
    out["frames"] = len(sel)
    return out


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
    "project": (98.9, "slot", "profiles/k_project_crowd_small.md"),   # (897.0 + 838.8) MB / 17.56M slots
    "bin": (11.84, "pair", "profiles/k_expand_crowd_small.md"),       # (175.4 + 245.8) MB / 35.6M pairs
}


def roofline_for(stage, stage_ms, fs, peaks, peak_kind):
    """Algorithmic work per launch of every stage (means over the timed frames) over its mean
    measured duration; the top-level fields are those of the dominant stage."""
    vis, pairs, nodes = fs["visible"], fs["pairs"], fs["render_nodes"]
    slots = nodes * 64
    clusters = fs.get("render_clusters", 0)
    units = {"pair": pairs, "slot": slots}
    bytes_per = {
        # selection: the node tables are L2-resident; HBM traffic is the render list write
        "select": 8 * nodes,
        # projection: 236 B of attributes per slot read -- once per distinct cluster (64 slots) when
        # the render list is projected grouped by cluster, the instances after the first reading
        # them from L2, plus the entry, its FP64 reference and its order (8 + 32 + 4 B per node) --
        # and a 48 B record + 8 B rect + 4 B key written per visible Gaussian
        "project": ((236 * 64 * clusters + 44 * nodes) if clusters else 236 * slots)
                   + (48 + 8 + 4) * vis + 4 * (slots - vis),
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
    if "select" in per_stage:   # its node tables stay in L2 / L1: the HBM figures are its writes only
        per_stage["select"]["bound"] = "latency"
        per_stage["select"]["note"] = ("node tables L2/L1-resident; HBM bytes are the render list written; "
                                       "issue and L2 figures in profiles/k_select_crowd_small.md")
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
