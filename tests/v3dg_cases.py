"""Shared cases and comparisons for the GPU parity tests (the oracle side is oracle/)."""
from __future__ import annotations

import numpy as np

import oracle

# Tolerances of the per-Gaussian records, about four times the largest errors measured against
# the FP64 oracle on a GB300 (tiny asset from three cameras, 200-instance crowd at 640x360: screen
# mean 7.6e-5 px, conic 2.0e-6 relative, colour 5.1e-7, opacity 2.1e-7).  The image bar is a max
# abs error of 1e-4 per channel outside the decision bands (measured 3e-6) and PSNR >= 50 dB.
U_ABS_PX = 3e-4          # screen mean, px
CONIC_REL = 1e-5         # relative to the largest conic entry
RGB_ABS = 2e-6
OPACITY_REL = 1e-6
IMG_ABS = 1e-4
PSNR_MIN = 50.0


def cut_tuples(inst, node):
    return {(int(i), int(n)) for i, n in zip(inst, node)}


def assert_cut_parity(gpu_cut: np.ndarray, cut: oracle.Cut) -> int:
    """Bit-exact cut (near ties excluded) and ascending (instance, node) order."""
    ties = {tuple(int(v) for v in t) for t in cut.ties}
    got = {tuple(int(v) for v in r) for r in gpu_cut}
    want = cut_tuples(cut.inst, cut.node)
    assert len(got) == len(gpu_cut), "duplicate cut entries"
    extra, missing = (got - want) - ties, (want - got) - ties
    assert not extra and not missing, f"cut differs: {len(extra)} extra {sorted(extra)[:5]}, {len(missing)} missing {sorted(missing)[:5]}"
    if len(gpu_cut) > 1:
        key = gpu_cut[:, 0].astype(np.int64) << 32 | gpu_cut[:, 1].astype(np.int64)
        assert (np.diff(key) > 0).all(), "cut not in (instance, node) order"
    return len(ties)


def gid(inst, local):
    return inst.astype(np.int64) << 32 | local.astype(np.int64)


def assert_projection_parity(g: dict, p: oracle.Projected):
    """Visible sets equal (boundary Gaussians excepted); records within the stated tolerances."""
    vis = p.visible & ~p.boundary
    og = gid(p.inst, p.local)
    gg = gid(g["inst"], g["local"])
    assert (np.diff(gg) > 0).all(), "projected Gaussians not in global-id order"
    bnd = set(og[p.boundary].tolist())
    gs, os_ = set(gg.tolist()) - bnd, set(og[vis].tolist())
    assert gs == os_, f"visible sets differ: {len(gs - os_)} extra, {len(os_ - gs)} missing"
    idx_o = {v: i for i, v in enumerate(og.tolist())}
    sel = np.array([i for i, v in enumerate(gg.tolist()) if v not in bnd], dtype=np.int64)
    oi = np.array([idx_o[v] for v in gg[sel].tolist()], dtype=np.int64)
    if len(sel) == 0:
        return 0
    assert (g["depth_key"][sel] == p.depth_key[oi]).all(), "depth keys differ"
    assert (g["rect"][sel] == p.rect[oi][:, [0, 1, 2, 3]]).all(), "tile rectangles differ"
    du = np.abs(g["u"][sel].astype(np.float64) - p.u[oi]).max()
    assert du <= U_ABS_PX, f"screen mean off by {du} px"
    cs = np.abs(p.conic[oi]).max(axis=1, keepdims=True)
    dc = (np.abs(g["conic"][sel].astype(np.float64) - p.conic[oi]) / cs).max()
    assert dc <= CONIC_REL, f"conic off by {dc} (relative)"
    drgb = np.abs(g["rgb"][sel].astype(np.float64) - p.rgb[oi]).max()
    assert drgb <= RGB_ABS, f"colour off by {drgb}"
    do = (np.abs(g["opacity"][sel].astype(np.float64) - p.opacity[oi]) / p.opacity[oi]).max()
    assert do <= OPACITY_REL, f"opacity off by {do}"
    return len(sel)


def assert_pairs_parity(g: dict, p: oracle.Projected, cam):
    """Sorted (tile, depth, id) pairs equal the oracle's, pairs of boundary Gaussians excepted."""
    tiles, keys, gi, bflag = oracle.sorted_pairs(p, cam)
    bnd = set(gid(p.inst, p.local)[p.boundary].tolist())
    gg = gid(g["inst"], g["local"])
    keep_g = np.array([v not in bnd for v in gg.tolist()], bool) if len(gg) else np.zeros(0, bool)
    want = np.stack([tiles[~bflag], keys[~bflag].astype(np.int64), gid(p.inst[gi[~bflag]], p.local[gi[~bflag]])], axis=1)
    got = np.stack([g["tile"][keep_g].astype(np.int64), g["depth_key"][keep_g].astype(np.int64), gg[keep_g]], axis=1)
    assert got.shape == want.shape, f"pair counts differ: {got.shape[0]} vs {want.shape[0]}"
    assert (got == want).all(), "sorted pairs differ"
    # the full GPU list is sorted by (tile, depth key, id)
    full = np.stack([g["tile"].astype(np.int64), g["depth_key"].astype(np.int64), gg], axis=1)
    o = np.lexsort((full[:, 2], full[:, 1], full[:, 0]))
    assert (o == np.arange(len(o))).all(), "GPU pairs not sorted by (tile, depth, id)"
    return got.shape[0]


def image_errors(img: np.ndarray, C: np.ndarray, B: np.ndarray):
    e = np.abs(img.astype(np.float64) - C).max(axis=-1)
    return float(e[~B].max()) if (~B).any() else 0.0, float(oracle.psnr(img, C)), int(B.sum())


def assert_image_matches_oracle(rgb, T, assets, inst, cam, tau, cut=None):
    """A rendered image (and its final transmittance) against the per-pixel definition, outside
    the decision bands; PSNR over every pixel.  Returns (max abs error, PSNR, band pixels)."""
    if cut is None:
        cut = oracle.select(assets, inst, cam, tau)
    p = oracle.project(assets, inst, cam, cut)
    C, To, B = oracle.render_image(p, cam.width, cam.height)
    err, ps, nb = image_errors(rgb, C, B)
    assert err <= IMG_ABS and ps >= PSNR_MIN, (err, ps, nb)
    if T is not None:
        assert np.abs(np.asarray(T, np.float64) - To)[~B].max() <= IMG_ABS
    return err, ps, nb
