"""Seeded synthetic 3DGS assets with a cluster hierarchy (stand-in for the offline build).

The paper builds its hierarchy offline (Sec. 3.1-3.2, Algorithm 1) with a binary median split,
cluster groups of two and local-splatting simplification; that stage is out of scope here. This
module generates inputs of the same shape instead:

* leaf Gaussians: means on the unit sphere plus N(0, 0.01) jitter per axis, log-scales
  N(-4, 0.5), uniform unit quaternions (Shoemake), opacity sigmoid(N(0, 1)), degree-3 SH
  coefficients N(0, 0.3), all stored as float32;
* leaf clusters: 64 consecutive Gaussians in Morton order (the last one may be partial);
* a 4-ary tree: parent j of level k+1 owns children [4j, min(4j+4, n_k)) of level k, and its
  Gaussians are the children's Gaussians merged pairwise, in order, by moment matching while
  more than 64 remain (an odd tail is carried over unchanged);
* one bounding sphere per cluster group, as Sec. 3.3 defines it: centre = mean of the group's
  Gaussian positions, radius = largest distance from that centre.  A node's *own* sphere is the
  sphere of the group it belongs to (its siblings); the root forms a group of its own.  Spheres
  are then enlarged so that every group sphere contains the group spheres one level below it
  (the paper only states that r_p > r_c is ensured, Sec. 3.4), with a relative margin of 2^-16
  and the radius rounded up to float32.

Nothing in here evaluates a footprint, selects, projects or blends: the module only produces
the arrays that the library's ``v3dg_load_hierarchy`` and the oracle both read.
"""
from __future__ import annotations

import dataclasses
import os

import numpy as np

LEAF_SIZE = 64          # Gaussians per cluster
BRANCH = 4              # clusters per cluster group (children per parent)
SH_COEFFS = 16          # (degree 3 + 1)^2
SPHERE_MARGIN = 2.0 ** -16


@dataclasses.dataclass
class Asset:
    """One asset: Gaussians in node order plus the node table (all arrays C-contiguous)."""

    means: np.ndarray        # (n, 3) float32
    log_scales: np.ndarray   # (n, 3) float32
    quats: np.ndarray        # (n, 4) float32, (w, x, y, z), not necessarily unit length
    opacity: np.ndarray      # (n,)   float32, activated, in (0, 1)
    sh: np.ndarray           # (n, 16, 3) float32, coefficient-major, channel-minor
    node_first: np.ndarray   # (m,) uint32: first Gaussian of the node
    node_count: np.ndarray   # (m,) uint32: Gaussians in the node (1..64)
    node_level: np.ndarray   # (m,) uint8: 0 for leaves
    node_parent: np.ndarray  # (m,) int32: -1 for the root
    own_sphere: np.ndarray   # (m, 4) float32: (cx, cy, cz, r) of the node's cluster group
    gaussians_per_group: int = LEAF_SIZE * BRANCH

    @property
    def n_gauss(self) -> int:
        return int(self.means.shape[0])

    @property
    def n_nodes(self) -> int:
        return int(self.node_first.shape[0])

    @property
    def n_levels(self) -> int:
        return int(self.node_level.max()) + 1


# ----------------------------------------------------------------------------- leaves


def _shoemake_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniformly distributed unit quaternions (w, x, y, z) from three uniforms (Shoemake)."""
    u = rng.random((n, 3))
    a = np.sqrt(1.0 - u[:, 0])
    b = np.sqrt(u[:, 0])
    t1 = 2.0 * np.pi * u[:, 1]
    t2 = 2.0 * np.pi * u[:, 2]
    return np.stack([b * np.cos(t2), a * np.sin(t1), a * np.cos(t1), b * np.sin(t2)], axis=1)


def _morton_order(p: np.ndarray) -> np.ndarray:
    """Stable argsort of 3D points by a 63-bit Morton code (21 bits per axis)."""
    lo = p.min(axis=0)
    span = np.maximum(p.max(axis=0) - lo, 1e-30)
    q = np.clip(((p - lo) / span * (2 ** 21 - 1)).astype(np.int64), 0, 2 ** 21 - 1).astype(np.uint64)

    def spread(v: np.ndarray) -> np.ndarray:
        v = v & np.uint64(0x1FFFFF)
        v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
        v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
        v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
        v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
        v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
        return v

    code = spread(q[:, 0]) | (spread(q[:, 1]) << np.uint64(1)) | (spread(q[:, 2]) << np.uint64(2))
    return np.argsort(code, kind="stable")


def leaf_gaussians(seed: int, n_leaves: int):
    """Draw the leaf Gaussians of one asset and return them in Morton order (float32)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = rng.standard_normal((n_leaves, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    means = g + 0.01 * rng.standard_normal((n_leaves, 3))
    log_scales = -4.0 + 0.5 * rng.standard_normal((n_leaves, 3))
    quats = _shoemake_quats(rng, n_leaves)
    opacity = 1.0 / (1.0 + np.exp(-rng.standard_normal(n_leaves)))
    sh = 0.3 * rng.standard_normal((n_leaves, SH_COEFFS, 3))
    order = _morton_order(means)
    f32 = np.float32
    return (means[order].astype(f32), log_scales[order].astype(f32), quats[order].astype(f32),
            opacity[order].astype(f32), sh[order].astype(f32))


# ----------------------------------------------------------------------------- merging


def _quat_to_rot(q: np.ndarray) -> np.ndarray:
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    r = np.empty(q.shape[:-1] + (3, 3))
    r[..., 0, 0] = 1 - 2 * (y * y + z * z)
    r[..., 0, 1] = 2 * (x * y - w * z)
    r[..., 0, 2] = 2 * (x * z + w * y)
    r[..., 1, 0] = 2 * (x * y + w * z)
    r[..., 1, 1] = 1 - 2 * (x * x + z * z)
    r[..., 1, 2] = 2 * (y * z - w * x)
    r[..., 2, 0] = 2 * (x * z - w * y)
    r[..., 2, 1] = 2 * (y * z + w * x)
    r[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return r


def _rot_to_quat(r: np.ndarray) -> np.ndarray:
    """Rotation matrices (det +1) to unit quaternions (w, x, y, z), largest-component branch."""
    m00, m11, m22 = r[:, 0, 0], r[:, 1, 1], r[:, 2, 2]
    tr = m00 + m11 + m22
    q = np.empty((r.shape[0], 4))
    cand = np.stack([tr, m00, m11, m22], axis=1)
    k = np.argmax(cand, axis=1)
    # branch 0: w largest
    s = np.sqrt(np.maximum(1.0 + cand[np.arange(len(k)), k] * 2.0 - tr, 1e-300)) * 2.0
    # For k == 0 the expression above is sqrt(1 + tr) * 2.
    b = k == 0
    q[b, 0] = 0.25 * s[b]
    q[b, 1] = (r[b, 2, 1] - r[b, 1, 2]) / s[b]
    q[b, 2] = (r[b, 0, 2] - r[b, 2, 0]) / s[b]
    q[b, 3] = (r[b, 1, 0] - r[b, 0, 1]) / s[b]
    b = k == 1
    q[b, 0] = (r[b, 2, 1] - r[b, 1, 2]) / s[b]
    q[b, 1] = 0.25 * s[b]
    q[b, 2] = (r[b, 0, 1] + r[b, 1, 0]) / s[b]
    q[b, 3] = (r[b, 0, 2] + r[b, 2, 0]) / s[b]
    b = k == 2
    q[b, 0] = (r[b, 0, 2] - r[b, 2, 0]) / s[b]
    q[b, 1] = (r[b, 0, 1] + r[b, 1, 0]) / s[b]
    q[b, 2] = 0.25 * s[b]
    q[b, 3] = (r[b, 1, 2] + r[b, 2, 1]) / s[b]
    b = k == 3
    q[b, 0] = (r[b, 1, 0] - r[b, 0, 1]) / s[b]
    q[b, 1] = (r[b, 0, 2] + r[b, 2, 0]) / s[b]
    q[b, 2] = (r[b, 1, 2] + r[b, 2, 1]) / s[b]
    q[b, 3] = 0.25 * s[b]
    q *= np.where(q[:, :1] < 0, -1.0, 1.0)
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def merge_pairs(means, log_scales, quats, opacity, sh, ia, ib):
    """Moment-matched merge of Gaussians ia[k] and ib[k] (float64 in, float32 out).

    Weights w = o * s1 * s2 * s3; mean and covariance are the weighted moments of the pair,
    opacity is 1 - (1 - o_a)(1 - o_b) capped at 0.999, SH is the weighted mean.  The merged
    covariance is re-factored into scales and a rotation (eigenvalues in descending order,
    eigenvector frame with determinant +1).
    """
    mu = means.astype(np.float64)
    s = np.exp(log_scales.astype(np.float64))
    o = opacity.astype(np.float64)
    w_all = o * s[:, 0] * s[:, 1] * s[:, 2]
    wa, wb = w_all[ia], w_all[ib]
    wsum = wa + wb
    ta, tb = (wa / wsum)[:, None], (wb / wsum)[:, None]
    m = ta * mu[ia] + tb * mu[ib]
    ra, rb = _quat_to_rot(quats[ia].astype(np.float64)), _quat_to_rot(quats[ib].astype(np.float64))
    ca = np.einsum("nij,nj,nkj->nik", ra, s[ia] ** 2, ra)
    cb = np.einsum("nij,nj,nkj->nik", rb, s[ib] ** 2, rb)
    da, db = mu[ia] - m, mu[ib] - m
    cov = (ta[:, :, None] * (ca + da[:, :, None] * da[:, None, :])
           + tb[:, :, None] * (cb + db[:, :, None] * db[:, None, :]))
    cov = 0.5 * (cov + np.swapaxes(cov, 1, 2))
    lam, vec = np.linalg.eigh(cov)
    lam = lam[:, ::-1]
    vec = vec[:, :, ::-1].copy()
    det = np.linalg.det(vec)
    vec[det < 0, :, 2] *= -1.0
    lam = np.maximum(lam, 1e-30)
    new_ls = 0.5 * np.log(lam)
    new_q = _rot_to_quat(vec)
    new_o = np.minimum(1.0 - (1.0 - o[ia]) * (1.0 - o[ib]), 0.999)
    shd = sh.astype(np.float64)
    new_sh = ta[:, :, None] * shd[ia] + tb[:, :, None] * shd[ib]
    f32 = np.float32
    return m.astype(f32), new_ls.astype(f32), new_q.astype(f32), new_o.astype(f32), new_sh.astype(f32)


def _merge_round(arrs, seg_start, seg_len):
    """One pairwise merge round over the segments longer than LEAF_SIZE."""
    means, log_scales, quats, opacity, sh = arrs
    merge = seg_len > LEAF_SIZE
    new_len = np.where(merge, (seg_len + 1) // 2, seg_len)
    new_start = np.concatenate([[0], np.cumsum(new_len)[:-1]]).astype(np.int64)
    total = int(new_len.sum())
    seg_of = np.repeat(np.arange(len(seg_len)), new_len)
    k = np.arange(total) - new_start[seg_of]        # position within the new segment
    m = merge[seg_of]
    ia = np.where(m, seg_start[seg_of] + 2 * k, seg_start[seg_of] + k)
    ib = np.where(m, seg_start[seg_of] + 2 * k + 1, -1)
    # the odd tail of a merged segment is copied
    ib = np.where(m & (ib >= seg_start[seg_of] + seg_len[seg_of]), -1, ib)
    out = [a[ia].copy() for a in arrs]
    pm = ib >= 0
    if pm.any():
        merged = merge_pairs(means, log_scales, quats, opacity, sh, ia[pm], ib[pm])
        for o_arr, mv in zip(out, merged):
            o_arr[pm] = mv
    return out, new_start, new_len


# ----------------------------------------------------------------------------- spheres


def _round_up_f32(x: np.ndarray) -> np.ndarray:
    r = x.astype(np.float32)
    low = r.astype(np.float64) < x
    r[low] = np.nextafter(r[low], np.float32(np.inf))
    return r


def _group_spheres(means: np.ndarray, seg_start: np.ndarray, seg_len: np.ndarray) -> np.ndarray:
    """(centre, radius) of each contiguous segment of Gaussian positions (Sec. 3.3, Fig. 4)."""
    p = means.astype(np.float64)
    seg_of = np.repeat(np.arange(len(seg_len)), seg_len)
    idx = _ranges(seg_start, seg_len)
    c = np.add.reduceat(p[idx], np.concatenate([[0], np.cumsum(seg_len)[:-1]]), axis=0) / seg_len[:, None]
    c32 = c.astype(np.float32)
    d = np.linalg.norm(p[idx] - c32.astype(np.float64)[seg_of], axis=1)
    r = np.maximum.reduceat(d, np.concatenate([[0], np.cumsum(seg_len)[:-1]]))
    return np.concatenate([c32, _round_up_f32(r)[:, None]], axis=1)


def _ranges(start: np.ndarray, length: np.ndarray) -> np.ndarray:
    seg_of = np.repeat(np.arange(len(length)), length)
    off = np.concatenate([[0], np.cumsum(length)[:-1]])
    return start[seg_of] + (np.arange(int(length.sum())) - off[seg_of])


# ----------------------------------------------------------------------------- assets


def make_asset(seed: int, n_leaves: int) -> Asset:
    """Generate one asset with ``n_leaves`` leaf Gaussians from ``seed`` (deterministic)."""
    level_arrs = [list(leaf_gaussians(seed, n_leaves))]
    n0 = (n_leaves + LEAF_SIZE - 1) // LEAF_SIZE
    counts = [np.minimum(LEAF_SIZE, n_leaves - LEAF_SIZE * np.arange(n0)).astype(np.int64)]
    while len(counts[-1]) > 1:
        ck = counts[-1]
        nk = len(ck)
        npar = (nk + BRANCH - 1) // BRANCH
        first_k = np.concatenate([[0], np.cumsum(ck)[:-1]])
        seg_start = first_k[::BRANCH].astype(np.int64)
        seg_len = np.add.reduceat(ck, np.arange(0, nk, BRANCH)).astype(np.int64)
        arrs = level_arrs[-1]
        while (seg_len > LEAF_SIZE).any():
            arrs, seg_start, seg_len = _merge_round(arrs, seg_start, seg_len)
        assert len(seg_len) == npar
        level_arrs.append(arrs)
        counts.append(seg_len)

    n_levels = len(counts)
    level_node_base = np.concatenate([[0], np.cumsum([len(c) for c in counts])[:-1]])
    level_gauss_base = np.concatenate([[0], np.cumsum([int(c.sum()) for c in counts])[:-1]])
    n_nodes = int(sum(len(c) for c in counts))

    node_first = np.empty(n_nodes, np.uint32)
    node_count = np.empty(n_nodes, np.uint32)
    node_level = np.empty(n_nodes, np.uint8)
    node_parent = np.empty(n_nodes, np.int32)
    own = np.empty((n_nodes, 4), np.float32)

    # group spheres: group_of_parent[k][j] = sphere of the children of node j at level k (k>=1)
    group_sph = [None]
    for k in range(1, n_levels):
        ck = counts[k - 1]
        nk = len(ck)
        first_k = np.concatenate([[0], np.cumsum(ck)[:-1]]).astype(np.int64)
        gstart = first_k[::BRANCH]
        glen = np.add.reduceat(ck, np.arange(0, nk, BRANCH)).astype(np.int64)
        group_sph.append(_group_spheres(level_arrs[k - 1][0], gstart, glen))
    root_sph = _group_spheres(level_arrs[-1][0], np.array([0]), counts[-1].astype(np.int64))[0]

    # containment: the group of node p's level must contain the group below each of its members
    for k in range(2, n_levels):
        g = group_sph[k]                      # groups of level-(k-1) nodes, one per level-k node
        below = group_sph[k - 1]              # groups of level-(k-2) nodes, one per level-(k-1) node
        owner = np.arange(len(below)) // BRANCH   # level-k parent that owns that level-(k-1) node
        d = np.linalg.norm(g[owner, :3].astype(np.float64) - below[:, :3].astype(np.float64), axis=1)
        need = np.zeros(len(g))
        np.maximum.at(need, owner, d + below[:, 3].astype(np.float64))
        r = np.maximum(g[:, 3].astype(np.float64), need * (1.0 + SPHERE_MARGIN))
        g[:, 3] = _round_up_f32(r)
    if n_levels > 1:
        top = group_sph[-1]
        d = np.linalg.norm(root_sph[:3].astype(np.float64) - top[0, :3].astype(np.float64))
        need = (d + float(top[0, 3])) * (1.0 + SPHERE_MARGIN)
        root_sph[3] = _round_up_f32(np.array([max(float(root_sph[3]), need)]))[0]

    for k in range(n_levels):
        nb, gb = level_node_base[k], level_gauss_base[k]
        ck = counts[k]
        nk = len(ck)
        sl = slice(nb, nb + nk)
        node_first[sl] = (gb + np.concatenate([[0], np.cumsum(ck)[:-1]])).astype(np.uint32)
        node_count[sl] = ck.astype(np.uint32)
        node_level[sl] = k
        if k + 1 < n_levels:
            node_parent[sl] = (level_node_base[k + 1] + np.arange(nk) // BRANCH).astype(np.int32)
            own[sl] = group_sph[k + 1][np.arange(nk) // BRANCH]
        else:
            node_parent[sl] = -1
            own[sl] = root_sph

    cat = [np.concatenate([la[i] for la in level_arrs]) for i in range(5)]
    return Asset(means=np.ascontiguousarray(cat[0]), log_scales=np.ascontiguousarray(cat[1]),
                 quats=np.ascontiguousarray(cat[2]), opacity=np.ascontiguousarray(cat[3]),
                 sh=np.ascontiguousarray(cat[4]), node_first=node_first, node_count=node_count,
                 node_level=node_level, node_parent=node_parent, own_sphere=own)


def cached_asset(seed: int, n_leaves: int, cache_dir: str | None = None) -> Asset:
    """``make_asset`` with an on-disk cache (``V3DG_CACHE`` or /tmp/v3dg_cache)."""
    cache_dir = cache_dir or os.environ.get("V3DG_CACHE", "/tmp/v3dg_cache")
    path = os.path.join(cache_dir, f"asset_s{seed}_n{n_leaves}_v1.npz")
    if os.path.exists(path):
        with np.load(path) as z:
            return Asset(**{f.name: z[f.name] for f in dataclasses.fields(Asset)
                            if f.name != "gaussians_per_group"})
    a = make_asset(seed, n_leaves)
    os.makedirs(cache_dir, exist_ok=True)
    tmp = path + f".tmp{os.getpid()}.npz"
    np.savez(tmp, **{f.name: getattr(a, f.name) for f in dataclasses.fields(Asset)
                     if f.name != "gaussians_per_group"})
    os.replace(tmp, path)
    return a


def _cached_asset_job(args):
    seed, n_leaves, cache_dir = args
    cached_asset(seed, n_leaves, cache_dir)
    return seed


def cached_assets(seeds, n_leaves: int, workers: int | None = None, cache_dir: str | None = None) -> list[Asset]:
    """Several cached assets; missing ones are generated in parallel worker processes (spawned)."""
    cache_dir = cache_dir or os.environ.get("V3DG_CACHE", "/tmp/v3dg_cache")
    missing = [s for s in seeds
               if not os.path.exists(os.path.join(cache_dir, f"asset_s{s}_n{n_leaves}_v1.npz"))]
    if len(missing) > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        workers = workers or min(len(missing), os.cpu_count() or 1, 4)   # each worker peaks at a few GB
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            list(ex.map(_cached_asset_job, [(s, n_leaves, cache_dir) for s in missing]))
    return [cached_asset(s, n_leaves, cache_dir) for s in seeds]
