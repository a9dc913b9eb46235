"""Plain FP64 CPU oracle of V3DG's online per-frame path (numpy).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this module.  The product path (the CUDA library and its Python
binding) never calls it, and it shares no code, constants or helpers with that path.

What it computes, in the paper's order:

1. per-(camera, instance) transform M = W [s R | t] in FP64 (the per-frame instances of
   App. B.3 under the camera view V of Sec. 3.4);
2. the footprint of a bounding sphere, F = pi r^2 f_x f_y / z_v^2 (Sec. 3.3, Fig. 4), with the
   sphere in view space under instance scale s (r' = s r);
3. the cut: clusters with F_c <= tau < F_p (Sec. 3.4), leaf F_c := 0 and root F_p := +inf;
4. splatting of the cut's Gaussians (Sec. 2.1, Sec. 5.1): EWA projection without 2D dilation
   (eps2d = 0), degree-3 SH colour, then per pixel front-to-back alpha blending
   C = sum_i c_i alpha_i prod_{j<i} (1 - alpha_j).

Readings where the paper is silent (each is one constant or switch):

* tau is given in pixels; the area tolerance is tau_F = float32(n_nom * tau_px^2) with
  n_nom = Gaussians per cluster group (256 for 64-Gaussian clusters in groups of 4).
* |z| <= r' (sphere straddles the camera plane) gives F = +inf; z enters squared.
* Near plane 0.01; cull z < near, opacity < 1/255, det(Sigma_2D) <= 0, or a pixel rectangle
  with no pixel centre inside the image.
* alpha = min(0.999, o exp(-q/2)); skip alpha < 1/255; stop before T (1 - alpha) < 1e-4.
* Pixel (px, py) samples at (px + 0.5, py + 0.5); 16x16 tiles, tile id = ty * tiles_x + tx.
* The depth sort key is an integer and is defined in the kernel's precision: the bits of the
  float32 value ((M20 x + M21 y) + M22 z) + M23, each operation rounded to float32 (no fused
  multiply-add), with M rounded from the FP64 M.  The near-plane cull compares that same value.
* Ties in depth are broken by global Gaussian id (instance, asset-local index).
* SH: real orthonormal basis, l <= 3, in the asset frame; colour = max(0, sum + 0.5).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

TILE = 16
NEAR_DEFAULT = 0.01
ALPHA_MAX = 0.999
ALPHA_MIN = 1.0 / 255.0
T_STOP = 1e-4
CLAMP_FOV = 1.3          # EWA Jacobian evaluated at the mean clamped to 1.3x the half-fov

# Decision bands that separate rounding noise from real disagreements.  A float32 evaluation can
# take the other side of a threshold only when the exact value lies within its rounding error of
# it: the skip (alpha >= 1/255) and stop (T (1 - alpha) >= 1e-4) rules of the blend, the footprint
# test of the cut, and the pixel-centre test of a Gaussian's tile rectangle.
TIE_REL = 1e-6           # footprint within this relative distance of tau_F: near tie
ALPHA_BAND = 1e-5        # alpha within this relative distance of 1/255: boundary pixel
T_BAND = 1e-5            # T (1 - alpha) within this relative distance of 1e-4: boundary pixel
EDGE_BAND_PX = 5e-4      # pixel-rectangle edge this close to a tile-changing edge: boundary


# ----------------------------------------------------------------------------- transforms


def compose(world_to_cam: np.ndarray, rot: np.ndarray, trans: np.ndarray, scale: np.ndarray) -> np.ndarray:
    """M = W [s R | t] for every instance, FP64, in a fixed operation order.

    M[r][c] = ((W[r][0] A[0][c] + W[r][1] A[1][c]) + W[r][2] A[2][c]) with A = s R, and
    M[r][3] = (((W[r][0] t0 + W[r][1] t1) + W[r][2] t2) + W[r][3]).  Element-wise numpy
    operations round each product and sum separately, so the result is reproducible.
    """
    w = np.asarray(world_to_cam, np.float64)
    n = rot.shape[0]
    a = scale[:, None, None] * rot                       # (n, 3, 3)
    m = np.empty((n, 3, 4))
    for r in range(3):
        for c in range(3):
            m[:, r, c] = (w[r, 0] * a[:, 0, c] + w[r, 1] * a[:, 1, c]) + w[r, 2] * a[:, 2, c]
        m[:, r, 3] = ((w[r, 0] * trans[:, 0] + w[r, 1] * trans[:, 1]) + w[r, 2] * trans[:, 2]) + w[r, 3]
    return m


def tau_area(tau_px: float, gaussians_per_group: int) -> float:
    """Area tolerance tau_F in px^2 (float32 value) for a per-Gaussian tolerance in px."""
    return float(np.float32(float(gaussians_per_group) * float(tau_px) * float(tau_px)))


# ----------------------------------------------------------------------------- footprint


def footprint(center: np.ndarray, radius: np.ndarray, m: np.ndarray, s: float, fx: float, fy: float) -> np.ndarray:
    """F = pi r'^2 fx fy / z^2 of asset-space spheres under one instance transform (Sec. 3.3).

    ``center`` (k, 3) and ``radius`` (k,) are in asset space, ``m`` the (3, 4) transform of
    the instance and ``s`` its uniform scale.  A sphere that reaches the camera plane
    (|z| <= r') has an unbounded footprint and gets +inf.
    """
    c = center.astype(np.float64)
    z = ((m[2, 0] * c[:, 0] + m[2, 1] * c[:, 1]) + m[2, 2] * c[:, 2]) + m[2, 3]
    r = s * radius.astype(np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        f = math.pi * float(fx) * float(fy) * r * r / (z * z)
    return np.where(np.abs(z) > r, f, np.inf)


@dataclasses.dataclass
class Cut:
    inst: np.ndarray        # (k,) uint32, sorted with node
    node: np.ndarray        # (k,) uint32
    ties: np.ndarray        # (t, 2) uint32 (instance, node) within TIE_REL of tau_F


def node_flags(asset):
    is_leaf = asset.node_level == 0
    is_root = asset.node_parent < 0
    par = np.where(is_root, 0, asset.node_parent)
    return is_leaf, is_root, par


def select(assets, inst, cam, tau_px: float) -> Cut:
    """The cut {(i, n) : F_c(i, n) <= tau_F < F_p(i, n)} over all instances (Sec. 3.4).

    F_c uses the node's own sphere (its cluster group) and F_p its parent's own sphere; a leaf
    has F_c = 0 and the root F_p = +inf.  Near ties (|F - tau_F| <= 1e-6 tau_F) are listed.
    """
    m_all = compose(cam.world_to_cam, inst.rot, inst.trans, inst.scale)
    out_i, out_n, ties = [], [], []
    for i in range(inst.n):
        a = assets[int(inst.asset[i])]
        tau = tau_area(tau_px, a.gaussians_per_group)
        is_leaf, is_root, par = node_flags(a)
        f = footprint(a.own_sphere[:, :3], a.own_sphere[:, 3], m_all[i], float(inst.scale[i]), cam.fx, cam.fy)
        f_own = np.where(is_leaf, 0.0, f)
        f_par = np.where(is_root, np.inf, f[par])
        sel = (f_own <= tau) & (tau < f_par)
        nodes = np.nonzero(sel)[0]
        out_i.append(np.full(nodes.shape, i, np.uint32))
        out_n.append(nodes.astype(np.uint32))
        near = (~is_leaf & (np.abs(f_own - tau) <= TIE_REL * tau)) | (~is_root & (np.abs(f_par - tau) <= TIE_REL * tau))
        t = np.nonzero(near)[0]
        ties.append(np.stack([np.full(t.shape, i, np.uint32), t.astype(np.uint32)], axis=1))
    return Cut(np.concatenate(out_i) if out_i else np.zeros(0, np.uint32),
               np.concatenate(out_n) if out_n else np.zeros(0, np.uint32),
               np.concatenate(ties) if ties else np.zeros((0, 2), np.uint32))


def cover_counts(asset, selected_mask: np.ndarray) -> np.ndarray:
    """For every leaf, how many nodes on its leaf-to-root path are selected."""
    cnt = selected_mask.astype(np.int64).copy()
    levels = asset.node_level
    for lvl in range(int(levels.max()) - 1, -1, -1):
        idx = np.nonzero(levels == lvl)[0]
        cnt[idx] += cnt[asset.node_parent[idx]]
    return cnt[levels == 0]


# ----------------------------------------------------------------------------- SH


def sh_basis(d: np.ndarray) -> np.ndarray:
    """Real orthonormal spherical harmonics Y_lm, l <= 3, m = -l..l, at unit directions d.

    Constants are written from their closed forms; signs follow the Condon-Shortley phase as in
    the usual 3DGS colour model.  Returns (k, 16).
    """
    x, y, z = d[:, 0], d[:, 1], d[:, 2]
    pi = math.pi
    k0 = 0.5 / math.sqrt(pi)
    k1 = math.sqrt(3.0 / (4.0 * pi))
    k2a = 0.5 * math.sqrt(15.0 / pi)
    k2b = 0.25 * math.sqrt(5.0 / pi)
    k2c = 0.25 * math.sqrt(15.0 / pi)
    k3a = 0.25 * math.sqrt(35.0 / (2.0 * pi))
    k3b = 0.5 * math.sqrt(105.0 / pi)
    k3c = 0.25 * math.sqrt(21.0 / (2.0 * pi))
    k3d = 0.25 * math.sqrt(7.0 / pi)
    k3e = 0.25 * math.sqrt(105.0 / pi)
    xx, yy, zz = x * x, y * y, z * z
    return np.stack([
        np.full_like(x, k0),
        -k1 * y, k1 * z, -k1 * x,
        k2a * x * y, -k2a * y * z, k2b * (2 * zz - xx - yy), -k2a * x * z, k2c * (xx - yy),
        -k3a * y * (3 * xx - yy), k3b * x * y * z, -k3c * y * (4 * zz - xx - yy),
        k3d * z * (2 * zz - 3 * xx - 3 * yy), -k3c * x * (4 * zz - xx - yy),
        k3e * z * (xx - yy), -k3a * x * (xx - 3 * yy),
    ], axis=1)


def sh_color(sh: np.ndarray, d: np.ndarray, degree: int = 3) -> np.ndarray:
    """max(0, sum_k Y_k(d) sh[k] + 0.5) per channel; ``sh`` (k, 16, 3), ``d`` (k, 3) unit."""
    nb = (degree + 1) ** 2
    y = sh_basis(d)[:, :nb]
    return np.maximum(np.einsum("kb,kbc->kc", y, sh[:, :nb, :].astype(np.float64)) + 0.5, 0.0)


# ----------------------------------------------------------------------------- projection


def quat_to_rot(q: np.ndarray) -> np.ndarray:
    q = q.astype(np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    r = np.empty((q.shape[0], 3, 3))
    r[:, 0, 0] = 1 - 2 * (y * y + z * z)
    r[:, 0, 1] = 2 * (x * y - w * z)
    r[:, 0, 2] = 2 * (x * z + w * y)
    r[:, 1, 0] = 2 * (x * y + w * z)
    r[:, 1, 1] = 1 - 2 * (x * x + z * z)
    r[:, 1, 2] = 2 * (y * z - w * x)
    r[:, 2, 0] = 2 * (x * z - w * y)
    r[:, 2, 1] = 2 * (y * z + w * x)
    r[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return r


def depth_key_f32(m: np.ndarray, mu: np.ndarray) -> np.ndarray:
    """float32 z = ((M20 x + M21 y) + M22 z) + M23 with every step rounded to float32."""
    f = np.float32
    m32 = m.astype(f)
    x, y, z = mu[:, 0].astype(f), mu[:, 1].astype(f), mu[:, 2].astype(f)
    return ((m32[2, 0] * x + m32[2, 1] * y) + m32[2, 2] * z) + m32[2, 3]


def pixel_rect(u, v, hx, hy, width, height):
    """Inclusive pixel-index range whose centres (p + 0.5) lie in [u - hx, u + hx] x [v - hy, v + hy]."""
    x0 = np.maximum(np.ceil(u - hx - 0.5), 0)
    x1 = np.minimum(np.floor(u + hx - 0.5), width - 1)
    y0 = np.maximum(np.ceil(v - hy - 0.5), 0)
    y1 = np.minimum(np.floor(v + hy - 0.5), height - 1)
    return x0, x1, y0, y1


def tile_rect(u, v, hx, hy, width, height):
    """Tile range [tx0, tx1] x [ty0, ty1] of the pixel rectangle, and whether it is empty."""
    x0, x1, y0, y1 = pixel_rect(u, v, hx, hy, width, height)
    empty = (x0 > x1) | (y0 > y1)
    with np.errstate(invalid="ignore"):
        t = [np.where(empty, 0, np.floor_divide(a, TILE)).astype(np.int64) for a in (x0, x1, y0, y1)]
    return t[0], t[1], t[2], t[3], empty


@dataclasses.dataclass
class Projected:
    """Per-Gaussian results for every Gaussian of the cut, in global-id order."""

    inst: np.ndarray         # (k,) instance
    local: np.ndarray        # (k,) asset-local Gaussian index
    visible: np.ndarray      # (k,) bool
    boundary: np.ndarray     # (k,) bool: a tile edge or cull within rounding of its threshold
    u: np.ndarray            # (k, 2) pixel mean
    cov: np.ndarray          # (k, 3) Sigma_2D (a, b, c)
    conic: np.ndarray        # (k, 3) inverse (A, B, C): q = A dx^2 + 2 B dx dy + C dy^2
    opacity: np.ndarray      # (k,)
    rgb: np.ndarray          # (k, 3)
    depth_key: np.ndarray    # (k,) uint32
    rect: np.ndarray         # (k, 4) int64 tiles (tx0, tx1, ty0, ty1), valid where visible
    pix: np.ndarray          # (k, 4) float64 pixel range (x0, x1, y0, y1)


def project(assets, inst, cam, cut: Cut, only=None) -> Projected:
    """EWA projection of every Gaussian of the cut (Sec. 2.1, eps2d = 0 as Sec. 5.1 sets).

    ``only``: optional {instance: asset-local Gaussian indices}; then only those Gaussians of the
    cut are projected (each exactly as without it).
    """
    m_all = compose(cam.world_to_cam, inst.rot, inst.trans, inst.scale)
    cam_c = cam.center
    fx, fy, cx, cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    w, h = cam.width, cam.height
    limx = CLAMP_FOV * (0.5 * w / fx)
    limy = CLAMP_FOV * (0.5 * h / fy)
    parts = {k: [] for k in Projected.__dataclass_fields__}
    order = np.lexsort((cut.node, cut.inst))
    ci, cn = cut.inst[order], cut.node[order]
    for i in np.unique(ci):
        a = assets[int(inst.asset[i])]
        nodes = cn[ci == i]
        first = a.node_first[nodes].astype(np.int64)
        cnt = a.node_count[nodes].astype(np.int64)
        seg = np.repeat(np.arange(len(nodes)), cnt)
        off = np.concatenate([[0], np.cumsum(cnt)[:-1]])
        local = first[seg] + (np.arange(int(cnt.sum())) - off[seg])
        if only is not None:
            local = local[np.isin(local, only.get(int(i), np.zeros(0, np.int64)))]
        m = m_all[i]
        mu = a.means[local].astype(np.float64)
        view = mu @ m[:, :3].T + m[:, 3]
        z32 = depth_key_f32(m, a.means[local])
        near_ok = z32 >= np.float32(cam.near)
        x, y, z = view[:, 0], view[:, 1], view[:, 2]
        with np.errstate(divide="ignore", invalid="ignore"):
            tx = np.clip(x / z, -limx, limx) * z
            ty = np.clip(y / z, -limy, limy) * z
            jac = np.zeros((len(local), 2, 3))
            jac[:, 0, 0] = fx / z
            jac[:, 0, 2] = -fx * tx / (z * z)
            jac[:, 1, 1] = fy / z
            jac[:, 1, 2] = -fy * ty / (z * z)
            rq = quat_to_rot(a.quats[local])
            sc = np.exp(2.0 * a.log_scales[local].astype(np.float64))
            cov3 = np.einsum("nij,nj,nkj->nik", rq, sc, rq)
            m3 = m[:, :3]
            covv = np.einsum("ij,njk,lk->nil", m3, cov3, m3)
            cov2 = np.einsum("nij,njk,nlk->nil", jac, covv, jac)
            ca, cb, cc = cov2[:, 0, 0], cov2[:, 0, 1], cov2[:, 1, 1]
            det = ca * cc - cb * cb
            conic = np.stack([cc / det, -cb / det, ca / det], axis=1)
            u = fx * x / z + cx
            v = fy * y / z + cy
        o = a.opacity[local].astype(np.float64)
        op_ok = o >= ALPHA_MIN
        with np.errstate(invalid="ignore", divide="ignore"):
            kk = 2.0 * np.log(255.0 * o)
            hx = np.sqrt(kk * ca)
            hy = np.sqrt(kk * cc)
        ok = near_ok & op_ok & (det > 0) & np.isfinite(det)
        u_s, v_s = np.where(ok, u, 0.0), np.where(ok, v, 0.0)
        hx_s, hy_s = np.where(ok, hx, 0.0), np.where(ok, hy, 0.0)
        tx0, tx1, ty0, ty1, empty = tile_rect(u_s, v_s, hx_s, hy_s, w, h)
        vis = ok & ~empty
        # boundary: the tile rectangle (or emptiness) changes within +-EDGE_BAND_PX of an edge
        e = EDGE_BAND_PX
        lo = tile_rect(u_s, v_s, np.maximum(hx_s - e, 0), np.maximum(hy_s - e, 0), w, h)
        hi = tile_rect(u_s, v_s, hx_s + e, hy_s + e, w, h)
        bnd = np.zeros(len(local), bool)
        for dxs in (-e, e):
            for dys in (-e, e):
                sh_ = tile_rect(u_s + dxs, v_s + dys, hx_s, hy_s, w, h)
                bnd |= (sh_[4] != empty) | (~empty & ((sh_[0] != tx0) | (sh_[1] != tx1) | (sh_[2] != ty0) | (sh_[3] != ty1)))
        for alt in (lo, hi):
            bnd |= (alt[4] != empty) | (~empty & ((alt[0] != tx0) | (alt[1] != tx1) | (alt[2] != ty0) | (alt[3] != ty1)))
        bnd &= ok
        # colour from the asset-frame view direction
        s = float(inst.scale[i])
        cam_a = inst.rot[i].T @ (cam_c - inst.trans[i]) / s
        dvec = mu - cam_a
        dvec /= np.linalg.norm(dvec, axis=1, keepdims=True)
        rgb = sh_color(a.sh[local], dvec)
        x0, x1, y0, y1 = pixel_rect(u_s, v_s, hx_s, hy_s, w, h)
        parts["inst"].append(np.full(len(local), i, np.uint32))
        parts["local"].append(local.astype(np.uint32))
        parts["visible"].append(vis)
        parts["boundary"].append(bnd)
        parts["u"].append(np.stack([u, v], axis=1))
        parts["cov"].append(np.stack([ca, cb, cc], axis=1))
        parts["conic"].append(conic)
        parts["opacity"].append(o)
        parts["rgb"].append(rgb)
        parts["depth_key"].append(z32.view(np.uint32))
        parts["rect"].append(np.stack([tx0, tx1, ty0, ty1], axis=1))
        parts["pix"].append(np.stack([x0, x1, y0, y1], axis=1))
    if not parts["inst"]:
        z = np.zeros(0)
        return Projected(z.astype(np.uint32), z.astype(np.uint32), z.astype(bool), z.astype(bool),
                         np.zeros((0, 2)), np.zeros((0, 3)), np.zeros((0, 3)), z, np.zeros((0, 3)),
                         z.astype(np.uint32), np.zeros((0, 4), np.int64), np.zeros((0, 4)))
    return Projected(**{k: np.concatenate(v) for k, v in parts.items()})


# ----------------------------------------------------------------------------- sort


def blend_order(p: Projected) -> np.ndarray:
    """Indices of the visible Gaussians in ascending (depth key, global id)."""
    vis = np.nonzero(p.visible)[0]
    o = np.lexsort((p.local[vis], p.inst[vis], p.depth_key[vis]))
    return vis[o]


def sorted_pairs(p: Projected, cam):
    """All (tile, depth key, Gaussian index) pairs sorted by (tile, depth key, global id).

    Returns (tile, depth_key, index into ``p``, boundary flag) arrays.
    """
    tiles_x = (cam.width + TILE - 1) // TILE
    vis = np.nonzero(p.visible)[0]
    tiles, gidx = [], []
    for g in vis:
        tx0, tx1, ty0, ty1 = p.rect[g]
        tt = (np.arange(ty0, ty1 + 1)[:, None] * tiles_x + np.arange(tx0, tx1 + 1)[None, :]).ravel()
        tiles.append(tt)
        gidx.append(np.full(tt.shape, g))
    if not tiles:
        e = np.zeros(0, np.int64)
        return e, e.astype(np.uint32), e, e.astype(bool)
    t = np.concatenate(tiles)
    gi = np.concatenate(gidx)
    o = np.lexsort((p.local[gi], p.inst[gi], p.depth_key[gi], t))
    return t[o], p.depth_key[gi[o]], gi[o], p.boundary[gi[o]]


# ----------------------------------------------------------------------------- blending


def _blend_one(alpha_seq, rgb_seq):
    """Front-to-back blend of one pixel's ordered (alpha, rgb); returns C, T, boundary."""
    t = 1.0
    c = np.zeros(3)
    bnd = False
    for al, col in zip(alpha_seq, rgb_seq):
        if abs(al - ALPHA_MIN) <= ALPHA_BAND * ALPHA_MIN:
            bnd = True
        if al < ALPHA_MIN:
            continue
        tn = t * (1.0 - al)
        if abs(tn - T_STOP) <= T_BAND * T_STOP:
            bnd = True
        if tn < T_STOP:
            break
        c += al * t * col
        t = tn
    return c, t, bnd


def gaussian_alpha(p: Projected, idx: np.ndarray, px: float, py: float) -> np.ndarray:
    dx = px + 0.5 - p.u[idx, 0]
    dy = py + 0.5 - p.u[idx, 1]
    q = p.conic[idx, 0] * dx * dx + 2.0 * p.conic[idx, 1] * dx * dy + p.conic[idx, 2] * dy * dy
    return np.minimum(ALPHA_MAX, p.opacity[idx] * np.exp(-0.5 * q))


def render_pixels(p: Projected, pixels) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Per-pixel definition at the listed (px, py): every visible Gaussian, in blend order.

    Gaussians whose pixel rectangle, widened by 2 px, misses the pixel are dropped first: there
    alpha < 1/255 holds exactly, so they would be skipped anyway.
    """
    order = blend_order(p)
    out_c, out_t, out_b = [], [], []
    for px, py in pixels:
        r = p.pix[order]
        near = (r[:, 0] - 2 <= px) & (px <= r[:, 1] + 2) & (r[:, 2] - 2 <= py) & (py <= r[:, 3] + 2)
        idx = order[near]
        al = gaussian_alpha(p, idx, px, py)
        c, t, b = _blend_one(al, p.rgb[idx])
        out_c.append(c)
        out_t.append(t)
        out_b.append(b)
    return np.array(out_c).reshape(-1, 3), np.array(out_t), np.array(out_b, bool)


def node_mean_balls(asset):
    """Per node: a ball holding the means of its Gaussians and their largest standard deviation.

    Centre = mean of the node's Gaussian means, radius = the largest distance from it (both
    FP64, asset frame), sigma = max over the node's Gaussians of exp(max log-scale).  Used only
    to bound where a node's Gaussians can land on screen.
    """
    first = asset.node_first.astype(np.int64)
    cnt = asset.node_count.astype(np.int64)
    start = np.cumsum(cnt) - cnt
    idx = np.repeat(first, cnt) + (np.arange(int(cnt.sum())) - np.repeat(start, cnt))
    mu = asset.means[idx].astype(np.float64)
    centre = np.add.reduceat(mu, start, axis=0) / cnt[:, None]
    d = np.sqrt(((mu - np.repeat(centre, cnt, axis=0)) ** 2).sum(axis=1))
    radius = np.maximum.reduceat(d, start)
    sigma = np.exp(np.maximum.reduceat(asset.log_scales[idx].astype(np.float64).max(axis=1), start))
    return centre, radius, sigma


def _near_any(ux, uy, dx, dy, pixels, windows):
    """Whether some listed pixel centre (px + 0.5, py + 0.5) lies within (dx, dy) of (ux, uy), or,
    with ``windows`` ((x0, y0, x1, y1) inclusive pixel rectangles), whether the box around (ux, uy)
    overlaps a window's span of pixel centres (a superset of the per-pixel test)."""
    hit = np.zeros(np.shape(ux), bool)
    if windows is not None:
        for x0, y0, x1, y1 in windows:
            hit |= (ux + dx >= x0 + 0.5) & (ux - dx <= x1 + 0.5) & (uy + dy >= y0 + 0.5) & (uy - dy <= y1 + 0.5)
        return hit
    for qx, qy in np.asarray([(px + 0.5, py + 0.5) for px, py in pixels], np.float64).reshape(-1, 2):
        hit |= (np.abs(qx - ux) <= dx) & (np.abs(qy - uy) <= dy)
    return hit


def nodes_reaching_pixels(assets, inst, cam, cut: Cut, pixels, slack_px: float = 1.0, windows=None) -> Cut:
    """The nodes of the cut whose Gaussians can have alpha >= 1/255 at one of the pixels.

    A conservative screen bound per (instance, node), so that the per-pixel definition at a
    few pixels of a large frame needs only these nodes' Gaussians projected.  With the node's
    means in the view-space ball (c, R) (R = s r) and c_z - R = z_min > near:
      * a mean p of the ball has |p_x / p_z - c_x / c_z| <= R sqrt(c_x^2 + c_z^2) / (c_z z_min)
        (and likewise in y), so its pixel mean is within f_x times that of f_x c_x / c_z + c_x0;
      * the EWA Jacobian at the clamped mean has ||J||_2 <= sqrt(f_x^2 (1 + l_x^2) + f_y^2
        (1 + l_y^2)) / z_min (Frobenius bound, |x'/z| <= l_x, |y'/z| <= l_y), and the view-space
        covariance has largest eigenvalue (s sigma)^2, so the alpha >= 1/255 ellipse
        (q <= 2 ln(255 o) <= 2 ln 255) lies within sqrt(2 ln 255) ||J||_2 s sigma of the mean.
    Nodes with z_min <= near are kept unless the whole ball lies behind the near plane (then the
    projection culls all of their Gaussians).  The bound is widened by 2 px (the margin of
    render_pixels) plus ``slack_px``.  ``windows``: rectangles of pixels tested as wholes (keeps
    a superset of the nodes that the pixels inside them would keep).
    """
    m_all = compose(cam.world_to_cam, inst.rot, inst.trans, inst.scale)
    fx, fy, cx, cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    limx = CLAMP_FOV * (0.5 * cam.width / fx)
    limy = CLAMP_FOV * (0.5 * cam.height / fy)
    jn = math.sqrt(fx * fx * (1.0 + limx * limx) + fy * fy * (1.0 + limy * limy))
    ksig = math.sqrt(2.0 * math.log(255.0))
    balls = {}
    keep = np.zeros(len(cut.inst), bool)
    by_inst = np.argsort(cut.inst, kind="stable")
    inst_sorted = cut.inst[by_inst]
    for i in np.unique(cut.inst):
        lo, hi = np.searchsorted(inst_sorted, [i, i + 1])
        sel = by_inst[lo:hi]
        a_id = int(inst.asset[i])
        if a_id not in balls:
            balls[a_id] = node_mean_balls(assets[a_id])
        centre, radius, sigma = balls[a_id]
        nodes = cut.node[sel].astype(np.int64)
        m = m_all[i]
        s = float(inst.scale[i])
        cv = centre[nodes] @ m[:, :3].T + m[:, 3]
        rv = s * radius[nodes]
        zmin = cv[:, 2] - rv
        front = zmin > float(cam.near)
        with np.errstate(divide="ignore", invalid="ignore"):
            ux = fx * cv[:, 0] / cv[:, 2] + cx
            uy = fy * cv[:, 1] / cv[:, 2] + cy
            spread = ksig * jn * s * sigma[nodes] / zmin + 2.0 + slack_px
            dx = fx * rv * np.sqrt(cv[:, 0] ** 2 + cv[:, 2] ** 2) / (cv[:, 2] * zmin) + spread
            dy = fy * rv * np.sqrt(cv[:, 1] ** 2 + cv[:, 2] ** 2) / (cv[:, 2] * zmin) + spread
        behind = cv[:, 2] + rv < float(cam.near)   # every mean behind the near plane: all culled
        hit = (~front & ~behind) | (front & _near_any(ux, uy, dx, dy, pixels, windows))
        keep[sel] = hit
    return Cut(cut.inst[keep], cut.node[keep], cut.ties)


def gaussians_reaching_pixels(assets, inst, cam, cut: Cut, pixels, slack_px: float = 1.0, windows=None):
    """The Gaussians of the cut that can have alpha >= 1/255 at one of the pixels.

    First the clusters (nodes_reaching_pixels), then each of their Gaussians by its own bound:
    with its mean at view depth z > near and pixel position u, its alpha >= 1/255 ellipse lies
    within sqrt(2 ln 255) ||J||_2 s sigma of u, ||J||_2 <= sqrt(f_x^2 (1 + l_x^2) + f_y^2
    (1 + l_y^2)) / z and sigma = exp(its largest log-scale).  Gaussians with z <= near are kept.
    ``windows`` as in nodes_reaching_pixels.
    Returns (the sub-cut of those clusters, {instance: sorted asset-local indices}) for project.
    """
    sub = nodes_reaching_pixels(assets, inst, cam, cut, pixels, slack_px, windows)
    m_all = compose(cam.world_to_cam, inst.rot, inst.trans, inst.scale)
    fx, fy, cx, cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    limx = CLAMP_FOV * (0.5 * cam.width / fx)
    limy = CLAMP_FOV * (0.5 * cam.height / fy)
    jn = math.sqrt(fx * fx * (1.0 + limx * limx) + fy * fy * (1.0 + limy * limy))
    ksig = math.sqrt(2.0 * math.log(255.0))
    only = {}
    by_inst = np.argsort(sub.inst, kind="stable")
    inst_sorted = sub.inst[by_inst]
    for i in np.unique(sub.inst):
        lo, hi = np.searchsorted(inst_sorted, [i, i + 1])
        nodes = np.sort(sub.node[by_inst[lo:hi]]).astype(np.int64)
        a = assets[int(inst.asset[i])]
        cnt = a.node_count[nodes].astype(np.int64)
        start = np.cumsum(cnt) - cnt
        local = np.repeat(a.node_first[nodes].astype(np.int64), cnt) + (np.arange(int(cnt.sum())) - np.repeat(start, cnt))
        m = m_all[i]
        s = float(inst.scale[i])
        view = a.means[local].astype(np.float64) @ m[:, :3].T + m[:, 3]
        z = view[:, 2]
        front = z > float(cam.near)
        sigma = np.exp(a.log_scales[local].astype(np.float64).max(axis=1))
        with np.errstate(divide="ignore", invalid="ignore"):
            u = fx * view[:, 0] / z + cx
            v = fy * view[:, 1] / z + cy
            spread = ksig * jn * s * sigma / z + 2.0 + slack_px
        hit = ~front | (front & _near_any(u, v, spread, spread, pixels, windows))
        if hit.any():
            only[int(i)] = local[hit]
    return sub, only


def render_image(p: Projected, width: int, height: int, region=None):
    """Whole image by the per-pixel definition, processed Gaussian by Gaussian.

    Pixels are updated in blend order; a pixel stops once its stop rule fires.  Only the
    Gaussian's pixel rectangle (where alpha >= 1/255 can hold) is visited, widened by 2 px so
    that near-threshold pixels are still checked and flagged.  ``region`` (x0, y0, x1, y1),
    inclusive: only those pixels are computed (every pixel depends only on its own Gaussians, so
    regions stitch into the whole image exactly).
    Returns (C (h, w, 3), T (h, w), boundary (h, w)) of the image or of the region.
    """
    rx0, ry0, rx1, ry1 = (0, 0, width - 1, height - 1) if region is None else region
    h, w = ry1 - ry0 + 1, rx1 - rx0 + 1
    C = np.zeros((h, w, 3))
    T = np.ones((h, w))
    done = np.zeros((h, w), bool)
    bnd = np.zeros((h, w), bool)
    for g in blend_order(p):
        x0, x1, y0, y1 = p.pix[g]
        x0 = int(max(x0 - 2, rx0)); x1 = int(min(x1 + 2, rx1))
        y0 = int(max(y0 - 2, ry0)); y1 = int(min(y1 + 2, ry1))
        if x0 > x1 or y0 > y1:
            continue
        ys, xs = np.mgrid[y0:y1 + 1, x0:x1 + 1]
        dx = xs + 0.5 - p.u[g, 0]
        dy = ys + 0.5 - p.u[g, 1]
        A, B, Cc = p.conic[g]
        q = A * dx * dx + 2.0 * B * dx * dy + Cc * dy * dy
        al = np.minimum(ALPHA_MAX, p.opacity[g] * np.exp(-0.5 * q))
        sl = (slice(y0 - ry0, y1 - ry0 + 1), slice(x0 - rx0, x1 - rx0 + 1))
        live = ~done[sl]
        bnd[sl] |= live & (np.abs(al - ALPHA_MIN) <= ALPHA_BAND * ALPHA_MIN)
        use = live & (al >= ALPHA_MIN)
        t = T[sl]
        tn = t * (1.0 - al)
        bnd[sl] |= use & (np.abs(tn - T_STOP) <= T_BAND * T_STOP)
        stop = use & (tn < T_STOP)
        add = use & ~stop
        C[sl] += np.where(add[..., None], (al * t)[..., None] * p.rgb[g], 0.0)
        T[sl] = np.where(add, tn, t)
        done[sl] |= stop
    return C, T, bnd


def subset_projected(p: Projected, idx) -> Projected:
    """The listed Gaussians of ``p`` (blend order among them is unchanged)."""
    return Projected(**{k: getattr(p, k)[idx] for k in Projected.__dataclass_fields__})


def psnr(a: np.ndarray, b: np.ndarray) -> float:
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * math.log10(1.0 / mse)
