"""GPU splatting (projection, binning + sort, blend) against the FP64 oracle."""
import math

import numpy as np
import pytest

import oracle
from synth import scenes
from v3dg_cases import (IMG_ABS, PSNR_MIN, assert_cut_parity, assert_image_matches_oracle, assert_pairs_parity,
                        assert_projection_parity, image_errors)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Context():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2505_06523_gb300 import Context
    return Context


def _frame(Context, assets, inst, cam, tau, opts=None):
    with Context(0) as ctx:
        for k, v in (opts or {}).items():
            ctx.set_option(k, v)
        for a in assets:
            ctx.load_hierarchy(a)
        ctx.set_instances(inst)
        ctx.select(cam, tau)
        rgb, T = ctx.render(want_T=True)
        out = {"rgb": rgb.cpu().numpy(), "T": T.cpu().numpy(), "cut": ctx.get_cut(), "proj": ctx.get_projected(),
               "pairs": ctx.get_pairs(), "ranges": ctx.tile_ranges(), "stats": ctx.frame_stats()}
    return out


def _check_ranges(out, cam):
    pr, rg = out["pairs"], out["ranges"]
    n_tiles = ((cam.width + 15) // 16) * ((cam.height + 15) // 16)
    assert rg.shape == (n_tiles, 2)
    for t in np.unique(pr["tile"]):
        s, e = rg[t]
        assert (pr["tile"][s:e] == t).all() and (s == 0 or pr["tile"][s - 1] != t) and (e == len(pr["tile"]) or pr["tile"][e] != t)
    empty = np.setdiff1d(np.arange(n_tiles), np.unique(pr["tile"]))
    assert (rg[empty, 0] == rg[empty, 1]).all()


def test_tiny_full_parity(Context, tiny_asset):
    """100k-leaf asset, 256x256, tau = 1 px: cut, records, pairs, ranges and the whole image."""
    cam = scenes.tiny_camera()
    inst = scenes.single_instance()
    out = _frame(Context, [tiny_asset], inst, cam, 1.0)
    cut = oracle.select([tiny_asset], inst, cam, 1.0)
    assert_cut_parity(out["cut"], cut)
    p = oracle.project([tiny_asset], inst, cam, cut)
    assert_projection_parity(out["proj"], p)
    assert_pairs_parity(out["pairs"], p, cam)
    _check_ranges(out, cam)
    C, T, B = oracle.render_image(p, cam.width, cam.height)
    err, ps, nb = image_errors(out["rgb"], C, B)
    assert err <= IMG_ABS, f"max |err| {err} over {cam.width * cam.height - nb} pixels"
    assert ps >= PSNR_MIN
    assert np.abs(out["T"].astype(np.float64) - T)[~B].max() <= IMG_ABS


def test_tiny_other_views(Context, tiny_asset):
    inst = scenes.single_instance()
    for cam, tau in [(scenes.look_at((1.2, -1.6, 0.9), (0, 0, 0), 200, 136, 70.0), 0.5),
                     (scenes.look_at((0.3, 0.2, 2.2), (0, 0, 0), 97, 75, 50.0), 2.0),
                     (scenes.look_at((0.0, -1.15, 0.0), (0, 1, 0.2), 160, 120, 90.0), 1.0)]:
        out = _frame(Context, [tiny_asset], inst, cam, tau)
        cut = oracle.select([tiny_asset], inst, cam, tau)
        assert_cut_parity(out["cut"], cut)
        p = oracle.project([tiny_asset], inst, cam, cut)
        assert_projection_parity(out["proj"], p)
        assert_pairs_parity(out["pairs"], p, cam)
        C, T, B = oracle.render_image(p, cam.width, cam.height)
        err, ps, _ = image_errors(out["rgb"], C, B)
        assert err <= IMG_ABS and ps >= PSNR_MIN, (err, ps)


def test_single_gaussian_closed_form(Context):
    """One isotropic Gaussian on the optical axis renders c * min(0.999, o exp(-r^2 / (2 s^2)))."""
    from test_oracle_splat import cam_identity, one_node_asset
    sigma, z, f, o = 0.04, 3.0, 50.0, 0.7
    sh = np.zeros((1, 16, 3))
    sh[0, 0] = [0.4, -0.2, 0.1]
    a = one_node_asset([[0, 0, z]], [[math.log(sigma)] * 3], opacity=[o], sh=sh)
    cam = cam_identity(w=40, h=36, f=f)
    out = _frame(Context, [a], scenes.single_instance(), cam, 1.0)
    s = f * math.exp(float(np.float32(math.log(sigma)))) / z
    ys, xs = np.mgrid[0:36, 0:40]
    r2 = (xs + 0.5 - 20.0) ** 2 + (ys + 0.5 - 18.0) ** 2
    al = np.minimum(0.999, float(np.float32(o)) * np.exp(-r2 / (2 * s * s)))
    near = np.abs(al - 1 / 255) <= 1e-3 / 255
    al = np.where(al >= 1 / 255, al, 0.0)
    col = 0.5 + sh[0, 0].astype(np.float32).astype(np.float64) * 0.5 / math.sqrt(math.pi)
    err = np.abs(out["rgb"] - al[..., None] * col).max(axis=-1)
    assert err[~near].max() <= IMG_ABS
    assert np.abs(out["T"] - (1 - al))[~near].max() <= IMG_ABS


def test_crowd_decimated_pixels(Context, tiny_asset, small_asset):
    """A 200-instance composition at 640x360: full-image parity."""
    inst = scenes.crowd_instances(200, n_assets=2, half_extent=70.0)
    assets = [tiny_asset, small_asset]
    cam = scenes.crowd_camera(40, 640, 360)
    out = _frame(Context, assets, inst, cam, 1.0)
    cut = oracle.select(assets, inst, cam, 1.0)
    assert_cut_parity(out["cut"], cut)
    p = oracle.project(assets, inst, cam, cut)
    assert_projection_parity(out["proj"], p)
    assert_pairs_parity(out["pairs"], p, cam)
    C, T, B = oracle.render_image(p, cam.width, cam.height)
    err, ps, nb = image_errors(out["rgb"], C, B)
    assert err <= IMG_ABS and ps >= PSNR_MIN, (err, ps, nb)


def test_orbit_sampled_pixels(Context):
    """1M-leaf asset at 1920x1080, near / mid / far: sampled pixels against the per-pixel oracle."""
    from synth.assets import cached_asset
    asset = cached_asset(1, 1_000_000)
    inst = scenes.single_instance()
    rng = np.random.default_rng(0)
    for k in (0, 3, 7):
        cam = scenes.orbit_camera(scenes.orbit_distances()[k])
        out = _frame(Context, [asset], inst, cam, 1.0)
        cut = oracle.select([asset], inst, cam, 1.0)
        assert_cut_parity(out["cut"], cut)
        p = oracle.project([asset], inst, cam, cut)
        assert_projection_parity(out["proj"], p)
        # pixels where something is drawn, plus a few random ones
        drawn = np.argwhere(out["T"] < 0.999)
        pick = drawn[rng.choice(len(drawn), size=min(48, len(drawn)), replace=False)] if len(drawn) else np.zeros((0, 2), int)
        pix = [(int(x), int(y)) for y, x in pick] + [(int(rng.integers(0, 1920)), int(rng.integers(0, 1080))) for _ in range(8)]
        c, t, b = oracle.render_pixels(p, pix)
        g = np.array([out["rgb"][y, x] for x, y in pix], np.float64)
        e = np.abs(g - c).max(axis=1)
        assert e[~b].max() <= IMG_ABS, (k, e.max())


def test_growth_from_tiny_capacities(Context, tiny_asset):
    """Start with 64-node / 4096-pair buffers: the frame overflows, grows and matches."""
    from paper_2505_06523_gb300._native import V3DG_OPT_CAP_NODES, V3DG_OPT_CAP_PAIRS
    cam = scenes.tiny_camera()
    inst = scenes.single_instance()
    small = _frame(Context, [tiny_asset], inst, cam, 1.0, {V3DG_OPT_CAP_NODES: 64, V3DG_OPT_CAP_PAIRS: 4096})
    big = _frame(Context, [tiny_asset], inst, cam, 1.0)
    assert (small["rgb"] == big["rgb"]).all()
    assert small["stats"]["overflow"] == 0


def test_render_host_matches_device(Context, tiny_asset):
    cam = scenes.tiny_camera()
    with Context(0) as ctx:
        ctx.load_hierarchy(tiny_asset)
        ctx.set_instances(scenes.single_instance())
        ctx.select(cam, 1.0)
        rgb_d, t_d = ctx.render(want_T=True)
        rgb_h, t_h = ctx.render_host(want_T=True)
    assert (rgb_d.cpu().numpy() == rgb_h).all() and (t_d.cpu().numpy() == t_h).all()


def test_deterministic_repeat(Context, tiny_asset, small_asset):
    inst = scenes.crowd_instances(200, n_assets=2, half_extent=70.0)
    cam = scenes.crowd_camera(150, 480, 270)
    a = _frame(Context, [tiny_asset, small_asset], inst, cam, 1.0)
    b = _frame(Context, [tiny_asset, small_asset], inst, cam, 1.0)
    assert (a["rgb"] == b["rgb"]).all()
    assert all((a["pairs"][k] == b["pairs"][k]).all() for k in a["pairs"])


def test_render_twice_after_one_select(Context, small_asset):
    """Every render recomputes the frame: a second render after one select gives the same image."""
    cam = scenes.look_at((0.3, -2.4, 0.5), (0.0, 0.0, 0.0), 128, 96, 60.0)
    with Context(0) as ctx:
        ctx.load_hierarchy(small_asset)
        ctx.set_instances(scenes.single_instance())
        ctx.select(cam, 1.0)
        a, _ = ctx.render()
        a = a.clone()
        b = ctx.render()[0]
        c = ctx.render()[0]
    assert float(a.abs().sum()) > 0
    assert (a == b).all() and (a == c).all()


def test_quadrant_split_is_bit_identical(Context, tiny_asset, small_asset):
    """Blending long tiles as four quadrants (here: every tile) changes no pixel."""
    from paper_2505_06523_gb300._native import V3DG_OPT_SPLIT_PAIRS
    inst = scenes.crowd_instances(200, n_assets=2, half_extent=70.0)
    cam = scenes.crowd_camera(40, 640, 360)
    whole = _frame(Context, [tiny_asset, small_asset], inst, cam, 1.0, {V3DG_OPT_SPLIT_PAIRS: 1 << 30})
    split = _frame(Context, [tiny_asset, small_asset], inst, cam, 1.0, {V3DG_OPT_SPLIT_PAIRS: 1})
    assert float(np.abs(whole["rgb"]).sum()) > 0
    assert (whole["rgb"] == split["rgb"]).all() and (whole["T"] == split["T"]).all()


@pytest.mark.parametrize("scene", ["crowd", "single"])
def test_projection_order_changes_nothing(Context, tiny_asset, small_asset, scene):
    """Projecting the render list grouped by cluster (V3DG_OPT_PROJECT_ORDER 1) or in list order (0)
    gives the same records, pairs, counters and image, bit for bit; the default (2) picks the
    grouping for the crowd (200 instances of 2 assets) and list order for one instance."""
    from paper_2505_06523_gb300._native import V3DG_OPT_PROJECT_ORDER
    if scene == "crowd":
        inst = scenes.crowd_instances(200, n_assets=2, half_extent=70.0)
        cam = scenes.crowd_camera(40, 640, 360)
    else:
        inst = scenes.single_instance()
        cam = scenes.tiny_camera()
    outs = [_frame(Context, [tiny_asset, small_asset], inst, cam, 1.0, {V3DG_OPT_PROJECT_ORDER: o}) for o in (0, 1, 2)]
    ref = outs[0]
    assert float(np.abs(ref["rgb"]).sum()) > 0
    for o in outs[1:]:
        assert (o["rgb"] == ref["rgb"]).all() and (o["T"] == ref["T"]).all()
        for k in ref["proj"]:
            assert np.array_equal(o["proj"][k], ref["proj"][k], equal_nan=True), k
        for k in ref["pairs"]:
            assert np.array_equal(o["pairs"][k], ref["pairs"][k]), k
        assert {k: v for k, v in o["stats"].items() if k != "render_clusters"} == \
            {k: v for k, v in ref["stats"].items() if k != "render_clusters"}
    # the distinct clusters of the render list, counted only by the grouped projection
    cut = outs[0]["cut"]
    cut_clusters = np.unique(inst.asset[cut[:, 0]].astype(np.uint64) << np.uint64(32) | cut[:, 1].astype(np.uint64))
    assert ref["stats"]["render_clusters"] == 0
    assert 0 < outs[1]["stats"]["render_clusters"] <= min(ref["stats"]["render_nodes"], len(cut_clusters))
    assert outs[2]["stats"]["render_clusters"] == (outs[1]["stats"]["render_clusters"] if scene == "crowd" else 0)


def test_projection_order_mixed_formats(Context, tiny_asset, small_asset):
    """Grouped projection over assets of both colour formats (one float32, one float16): the
    mixed-format kernel gives the same image in both orders, and it matches the oracle on the
    float16-rounded attributes."""
    from paper_2505_06523_gb300._native import V3DG_OPT_ATTR_FP16, V3DG_OPT_PROJECT_ORDER
    inst = scenes.crowd_instances(200, n_assets=2, half_extent=70.0)
    cam = scenes.crowd_camera(40, 640, 360)
    outs = []
    for o in (0, 1):
        with Context(0) as ctx:
            ctx.set_option(V3DG_OPT_PROJECT_ORDER, o)
            ctx.load_hierarchy(tiny_asset)
            ctx.set_option(V3DG_OPT_ATTR_FP16, 1)
            ctx.load_hierarchy(small_asset)
            ctx.set_instances(inst)
            ctx.select(cam, 1.0)
            rgb, T = ctx.render(want_T=True)
            outs.append((rgb.cpu().numpy(), T.cpu().numpy(), ctx.get_projected(), ctx.frame_stats()))
    (rgb0, T0, p0, st0), (rgb1, T1, p1, st1) = outs
    assert float(np.abs(rgb0).sum()) > 0
    assert (rgb0 == rgb1).all() and (T0 == T1).all()
    for k in p0:
        assert np.array_equal(p0[k], p1[k], equal_nan=True), k
    assert st0["render_clusters"] == 0 and st1["render_clusters"] > 0
    assets = [tiny_asset, _fp16_rounded(small_asset)]
    assert_image_matches_oracle(rgb1, T1, assets, inst, cam, 1.0)


def test_projection_order_option_range(Context):
    from paper_2505_06523_gb300._native import V3DG_OPT_PROJECT_ORDER
    with Context(0) as ctx:
        for v in (0, 1, 2):
            ctx.set_option(V3DG_OPT_PROJECT_ORDER, v)
        for v in (-1, 3):
            with pytest.raises(Exception):
                ctx.set_option(V3DG_OPT_PROJECT_ORDER, v)


def _fp16_rounded(asset):
    import copy
    a = copy.copy(asset)
    a.sh = asset.sh.astype(np.float16).astype(np.float32)
    a.opacity = asset.opacity.astype(np.float16).astype(np.float32)
    return a


@pytest.mark.parametrize("view", [0, 1])
def test_fp16_attributes_parity(Context, tiny_asset, view):
    """Opacity and SH stored as float16: parity with the oracle on the rounded attributes, and
    PSNR >= 50 dB against the oracle on the float32 attributes."""
    from paper_2505_06523_gb300._native import V3DG_OPT_ATTR_FP16
    cam = [scenes.tiny_camera(), scenes.look_at((1.2, -1.6, 0.9), (0, 0, 0), 200, 136, 70.0)][view]
    inst = scenes.single_instance()
    out = _frame(Context, [tiny_asset], inst, cam, 1.0, {V3DG_OPT_ATTR_FP16: 1})
    a16 = _fp16_rounded(tiny_asset)
    cut = oracle.select([a16], inst, cam, 1.0)
    assert_cut_parity(out["cut"], cut)
    p16 = oracle.project([a16], inst, cam, cut)
    assert_projection_parity(out["proj"], p16)
    assert_pairs_parity(out["pairs"], p16, cam)
    C16, T16, B16 = oracle.render_image(p16, cam.width, cam.height)
    err, ps, _ = image_errors(out["rgb"], C16, B16)
    assert err <= IMG_ABS and ps >= PSNR_MIN, (err, ps)
    p32 = oracle.project([tiny_asset], inst, cam, cut)
    C32, _, _ = oracle.render_image(p32, cam.width, cam.height)
    assert oracle.psnr(out["rgb"], C32) >= PSNR_MIN


@pytest.mark.parametrize("view,tau", [(0, 0.5), (1, 0.5), (1, 1.0), (2, 2.0)])
def test_paper_shaped_bundle(Context, view, tau):
    """The paper's bundle shape (4096-Gaussian clusters, binary tree, halving simplification,
    tau in the paper's units: tau_px = 0.5 is tau_F = 2048 px^2): cut, records, pairs and image."""
    from synth.paper_tree import make_asset_paper
    asset = make_asset_paper(0, 100_000)
    cam = [scenes.tiny_camera(), scenes.orbit_camera(4.0, 320, 180), scenes.orbit_camera(12.0, 320, 180)][view]
    inst = scenes.single_instance()
    out = _frame(Context, [asset], inst, cam, tau)
    cut = oracle.select([asset], inst, cam, tau)
    assert_cut_parity(out["cut"], cut)
    p = oracle.project([asset], inst, cam, cut)
    assert_projection_parity(out["proj"], p)
    assert_pairs_parity(out["pairs"], p, cam)
    C, T, B = oracle.render_image(p, cam.width, cam.height)
    err, ps, nb = image_errors(out["rgb"], C, B)
    assert err <= IMG_ABS and ps >= PSNR_MIN, (err, ps)


def test_blend_batch_sizes_and_autotuner(Context, tiny_asset, small_asset):
    """Every blend variant and batch size gives the same image bit for bit; the autotuner needs a
    rendered frame, picks one of its candidates, keeps it, and the frames after it are unchanged."""
    from paper_2505_06523_gb300._native import V3DG_OPT_BLEND_BATCH, V3DG_OPT_BLEND_MODE, V3dgError
    inst = scenes.crowd_instances(200, n_assets=2, half_extent=70.0)
    cam = scenes.crowd_camera(40, 640, 360)
    outs = [_frame(Context, [tiny_asset, small_asset], inst, cam, 1.0, {V3DG_OPT_BLEND_BATCH: b, V3DG_OPT_BLEND_MODE: m})
            for m in (0, 1) for b in (128, 256, 512)]
    assert float(np.abs(outs[0]["rgb"]).sum()) > 0
    for o in outs[1:]:
        assert (o["rgb"] == outs[0]["rgb"]).all() and (o["T"] == outs[0]["T"]).all()
    with Context(0) as ctx:
        for a in (tiny_asset, small_asset):
            ctx.load_hierarchy(a)
        ctx.set_instances(inst)
        with pytest.raises(V3dgError):
            ctx.autotune_blend()
        ctx.select(cam, 1.0)
        ctx.render()
        r = ctx.autotune_blend()
        assert r["batch"] in (128, 256, 512) and r["split_pairs"] in (4096, 16384, 65536, 0xFFFFFFFF) and r["ms"] > 0
        assert r["mode"] in (0, 1)
        ctx.select(cam, 1.0)
        rgb, T = ctx.render(want_T=True)
        assert (rgb.cpu().numpy() == outs[0]["rgb"]).all() and (T.cpu().numpy() == outs[0]["T"]).all()
    # the frame rendered with the tuned settings, against the oracle itself
    assert_image_matches_oracle(rgb.cpu().numpy(), T.cpu().numpy(), [tiny_asset, small_asset], inst, cam, 1.0)


def test_views_batch_equals_single_views(Context, tiny_asset, small_asset):
    """Several cameras in one batch: every stage runs once for all views, and each view's image,
    cut and counters are those of the view rendered alone, bit for bit."""
    inst = scenes.crowd_instances(200, n_assets=2, half_extent=70.0)
    assets = [tiny_asset, small_asset]
    cams = [scenes.crowd_camera(t, 480, 270) for t in (0, 40, 150, 151)]
    singles = [_frame(Context, assets, inst, cam, 1.0) for cam in cams]
    with Context(0) as ctx:
        for a in assets:
            ctx.load_hierarchy(a)
        ctx.set_instances(inst)
        ctx.select_views(cams, 1.0)
        rgb, T = ctx.render(want_T=True)
        cut = ctx.get_cut()
        ranges = ctx.tile_ranges()
        host_rgb, host_T = ctx.render_host(want_T=True)
    rgb, T = rgb.cpu().numpy(), T.cpu().numpy()
    assert rgb.shape == (4, 270, 480, 3) and ranges.shape[0] == 4 * 30 * 17
    n = inst.n
    for v, one in enumerate(singles):
        assert (rgb[v] == one["rgb"]).all() and (T[v] == one["T"]).all(), v
        assert (host_rgb[v] == one["rgb"]).all() and (host_T[v] == one["T"]).all(), v
        mine = cut[(cut[:, 0] >= v * n) & (cut[:, 0] < (v + 1) * n)].copy()
        mine[:, 0] -= v * n
        assert np.array_equal(mine, one["cut"])
        rv = ranges[v * 510:(v + 1) * 510].astype(np.int64)
        assert ((rv[:, 1] - rv[:, 0]) == (one["ranges"][:, 1].astype(np.int64) - one["ranges"][:, 0])).all()
    for v in (0, 2):   # views of the batch against the oracle itself
        assert_image_matches_oracle(rgb[v], T[v], assets, inst, cams[v], 1.0)
    with pytest.raises(Exception):
        with Context(0) as ctx:
            ctx.load_hierarchy(tiny_asset)
            ctx.set_instances(inst)
            ctx.select_views([cams[0], scenes.crowd_camera(3, 320, 180)], 1.0)


def test_graph_frames_match_launch_by_launch(Context, tiny_asset, small_asset):
    """CUDA-graph frames: the same images as launching stage by stage, through a buffer overflow
    (the frame is re-run and grows), a camera walk that reuses the captured graph, and an image
    size change that captures a new one."""
    from paper_2505_06523_gb300._native import V3DG_OPT_CAP_NODES, V3DG_OPT_CAP_PAIRS, V3DG_OPT_GRAPHS
    inst = scenes.crowd_instances(200, n_assets=2, half_extent=70.0)
    cams = [scenes.crowd_camera(t, 320, 180) for t in (0, 13, 26, 39)] + [scenes.crowd_camera(50, 480, 270)]
    out = {}
    for graphs in (0, 1):
        imgs = []
        with Context(0) as ctx:
            ctx.set_option(V3DG_OPT_GRAPHS, graphs)
            ctx.set_option(V3DG_OPT_CAP_NODES, 64)
            ctx.set_option(V3DG_OPT_CAP_PAIRS, 4096)
            for a in (tiny_asset, small_asset):
                ctx.load_hierarchy(a)
            ctx.set_instances(inst)
            for cam in cams + cams[:2]:
                ctx.select(cam, 1.0)
                rgb, T = ctx.render(want_T=True)
                st = ctx.frame_stats()
                imgs.append((rgb.cpu().numpy(), T.cpu().numpy(), st["pairs"], st["render_nodes"]))
        out[graphs] = imgs
    assert float(np.abs(out[0][0][0]).sum()) > 0
    for (r0, t0, p0, n0), (r1, t1, p1, n1) in zip(out[0], out[1]):
        assert (r0 == r1).all() and (t0 == t1).all() and p0 == p1 and n0 == n1
    for k in (1, 4, 6):   # graph replays (one after a size change) against the oracle itself
        cam = (cams + cams[:2])[k]
        assert_image_matches_oracle(out[1][k][0], out[1][k][1], [tiny_asset, small_asset], inst, cam, 1.0)


def test_views_topdown_graph_batch512_together(Context, tiny_asset, small_asset):
    """Batched views, top-down selection, CUDA-graph frames and 512-record blend batches at once:
    every view's image is that of the view rendered alone with the plain settings, bit for bit."""
    from paper_2505_06523_gb300._native import V3DG_OPT_BLEND_BATCH, V3DG_OPT_GRAPHS, V3DG_OPT_SELECT_TOPDOWN
    inst = scenes.crowd_instances(200, n_assets=2, half_extent=70.0)
    assets = [tiny_asset, small_asset]
    cams = [scenes.crowd_camera(t, 320, 180) for t in (5, 60, 200)]
    singles = [_frame(Context, assets, inst, cam, 1.0, {V3DG_OPT_SELECT_TOPDOWN: 0, V3DG_OPT_BLEND_BATCH: 256})
               for cam in cams]
    with Context(0) as ctx:
        for k, v in ((V3DG_OPT_SELECT_TOPDOWN, 1), (V3DG_OPT_GRAPHS, 1), (V3DG_OPT_BLEND_BATCH, 512)):
            ctx.set_option(k, v)
        for a in assets:
            ctx.load_hierarchy(a)
        ctx.set_instances(inst)
        for _ in range(2):   # the second round replays the captured graph
            ctx.select_views(cams, 1.0)
            rgb, T = ctx.render(want_T=True)
            rgb, T = rgb.cpu().numpy(), T.cpu().numpy()
            for v, one in enumerate(singles):
                assert (rgb[v] == one["rgb"]).all() and (T[v] == one["T"]).all(), v
    for v, cam in enumerate(cams):   # and each view against the oracle itself
        assert_image_matches_oracle(rgb[v], T[v], assets, inst, cam, 1.0)
