"""The crowd composition at full size, as bench.py renders it: 10 assets of 1M leaves, 1000
instances, 1920x1080, fov 45, tau = 1 px, default options.

Per walk frame: the whole cut bit-exact against the oracle (11M clusters), the tile ranges
against properties that hold at any size, and 512 sampled pixels (eight 8x8 windows, one in the
tile with the longest list) against the per-pixel oracle, which projects only the Gaussians that
can reach them (oracle.gaussians_reaching_pixels).  At most 5% of them may lie within a decision
band; the others are within the image tolerance, and the PSNR over all of them is >= 50 dB.  The float16
colour storage gets the same sampled check against the oracle on the rounded attributes, and its
error against the float32 attributes is reported beside it.
"""
import copy

import numpy as np
import pytest

import oracle
from synth import scenes
from v3dg_cases import IMG_ABS, PSNR_MIN

pytestmark = pytest.mark.gpu

WIDTH, HEIGHT, TAU = 1920, 1080, 1.0


@pytest.fixture(scope="module")
def crowd():
    from synth.assets import cached_assets
    assets = cached_assets(list(range(10)), 1_000_000)
    inst = scenes.crowd_instances(1000, n_assets=10)
    return assets, inst


@pytest.fixture(scope="module")
def Context():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2505_06523_gb300 import Context
    return Context


def _keys(a, b):
    return (np.asarray(a, np.int64) << 32) | np.asarray(b, np.int64)


def _render(Context, assets, inst, cams, opts=None):
    out = []
    with Context(0) as ctx:
        for k, v in (opts or {}).items():
            ctx.set_option(k, v)
        for a in assets:
            ctx.load_hierarchy(a)
        ctx.set_instances(inst)
        for cam in cams:
            ctx.select(cam, TAU)
            rgb, T = ctx.render(want_T=True)
            out.append({"rgb": rgb.cpu().numpy(), "T": T.cpu().numpy(), "cut": ctx.get_cut(),
                        "ranges": ctx.tile_ranges(), "stats": ctx.frame_stats()})
    return out


def _sample_windows(frame, rng, n_windows=8, size=8):
    """Eight 8x8 windows (512 pixels): one in the tile with the longest list, the others around
    drawn pixels.  The oracle projects only the Gaussians that can reach them
    (oracle.gaussians_reaching_pixels, windows tested as wholes)."""
    tiles_x = (WIDTH + 15) // 16
    rg = frame["ranges"].astype(np.int64)
    t = int(np.argmax(rg[:, 1] - rg[:, 0]))
    drawn = np.argwhere(frame["T"] < 0.999)
    corners = [(16 * (t % tiles_x) + 4, 16 * (t // tiles_x) + 4)]
    for y, x in drawn[rng.choice(len(drawn), size=n_windows - 1, replace=False)]:
        corners.append((int(x), int(y)))
    wins = []
    for cx, cy in corners:
        x0 = min(max(cx - size // 2, 0), WIDTH - size)
        y0 = min(max(cy - size // 2, 0), HEIGHT - size)
        wins.append((x0, y0, x0 + size - 1, y0 + size - 1))
    pix = sorted({(x, y) for x0, y0, x1, y1 in wins for y in range(y0, y1 + 1) for x in range(x0, x1 + 1)})
    return wins, pix


def _check_cut(gpu_cut, cut):
    """Bit-exact cut at full size (near ties excluded), in (instance, node) order."""
    got = _keys(gpu_cut[:, 0], gpu_cut[:, 1])
    want = np.sort(_keys(cut.inst, cut.node))
    assert (np.diff(got) > 0).all(), "cut not in (instance, node) order"
    ties = _keys(cut.ties[:, 0], cut.ties[:, 1]) if len(cut.ties) else np.zeros(0, np.int64)
    g, w = got[~np.isin(got, ties)], want[~np.isin(want, ties)]
    assert g.shape == w.shape and (g == w).all(), f"cut differs: {len(np.setdiff1d(g, w))} extra, " \
                                                 f"{len(np.setdiff1d(w, g))} missing"
    return len(ties)


def _check_ranges(rg, pairs):
    """Tile ranges: empty or ascending, disjoint and covering [0, pairs) in tile order."""
    rg = rg.astype(np.int64)
    assert (rg[:, 0] <= rg[:, 1]).all()
    ne = rg[rg[:, 1] > rg[:, 0]]
    assert ne[0, 0] == 0 and ne[-1, 1] == pairs and (ne[1:, 0] == ne[:-1, 1]).all()


def _sampled_errors(assets_oracle, inst, cam, cut, frame, wins, pix):
    sub, only = oracle.gaussians_reaching_pixels(assets_oracle, inst, cam, cut, pix, windows=wins)
    p = oracle.project(assets_oracle, inst, cam, sub, only=only)
    c, t, b = oracle.render_pixels(p, pix)
    g = np.array([frame["rgb"][y, x] for x, y in pix], np.float64)
    gt = np.array([frame["T"][y, x] for x, y in pix], np.float64)
    return np.abs(g - c).max(axis=1), np.abs(gt - t), b, c, g


def _psnr(a, b):
    mse = float(np.mean((a - b) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(1.0 / mse)


@pytest.mark.parametrize("t", [0, 150, 299])
def test_crowd_full_size_fp32(Context, crowd, t):
    assets, inst = crowd
    cam = scenes.crowd_camera(t, WIDTH, HEIGHT)
    (frame,) = _render(Context, assets, inst, [cam])
    st = frame["stats"]
    assert not st["overflow"] and not st["timeout"]
    cut = oracle.select(assets, inst, cam, TAU)
    _check_cut(frame["cut"], cut)
    assert st["cut_nodes"] == len(frame["cut"]) and st["render_nodes"] > 0
    _check_ranges(frame["ranges"], st["pairs"])
    wins, pix = _sample_windows(frame, np.random.default_rng(t))
    e, et, b, c, g = _sampled_errors(assets, inst, cam, cut, frame, wins, pix)
    drawn = int((np.array([frame["T"][y, x] for x, y in pix]) < 0.999).sum())
    print(f"frame {t}: {len(pix)} pixels ({drawn} drawn), {int(b.sum())} within a decision band, "
          f"max |err| {e[~b].max():.2e}, PSNR {_psnr(g, c):.1f} dB")
    assert len(pix) >= 500 and drawn >= 250
    assert b.sum() <= 0.05 * len(pix)   # pixels with a decision within rounding of its threshold
    assert e[~b].max() <= IMG_ABS, (e.max(), pix[int(np.argmax(e))])
    assert et[~b].max() <= IMG_ABS
    assert _psnr(g, c) >= PSNR_MIN


def _fp16_rounded(asset):
    a = copy.copy(asset)
    a.sh = asset.sh.astype(np.float16).astype(np.float32)
    a.opacity = asset.opacity.astype(np.float16).astype(np.float32)
    return a


def test_crowd_full_size_fp16(Context, crowd):
    """Opacity and SH stored as float16: sampled pixels within the image tolerance of the oracle
    on the rounded attributes, and within PSNR 50 dB of the oracle on the float32 attributes."""
    from paper_2505_06523_gb300._native import V3DG_OPT_ATTR_FP16
    assets, inst = crowd
    cam = scenes.crowd_camera(75, WIDTH, HEIGHT)
    (frame,) = _render(Context, assets, inst, [cam], {V3DG_OPT_ATTR_FP16: 1})
    a16 = [_fp16_rounded(a) for a in assets]
    cut = oracle.select(a16, inst, cam, TAU)
    _check_cut(frame["cut"], cut)
    wins, pix = _sample_windows(frame, np.random.default_rng(75))
    e, et, b, _, g = _sampled_errors(a16, inst, cam, cut, frame, wins, pix)
    assert b.sum() <= 0.05 * len(pix)
    assert e[~b].max() <= IMG_ABS and et[~b].max() <= IMG_ABS
    _, _, _, c32, _ = _sampled_errors(assets, inst, cam, cut, frame, wins, pix)
    assert _psnr(g, c32) >= PSNR_MIN
