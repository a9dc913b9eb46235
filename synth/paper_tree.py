"""Generator variant with the paper's own bundle shape (Sec. 3.1-3.2), for the online path.

The default generator (synth.assets) groups 64-Gaussian clusters four at a time and merges
Gaussians by moment matching.  This one follows the paper's construction instead:

* leaf clusters of n_{G in C} = 4096 Gaussians by binary median split of the positions
  (Sec. 3.1: split at the median of the longest axis until a part holds at most 4096);
* cluster groups of n_{C in CG} = 2 adjacent clusters (siblings of the split, Sec. 3.2), each
  simplified into one cluster by the "0-iteration" rule: keep the half of the group's Gaussians
  with the larger product of scale and opacity, and multiply their scales by 2^(1/6) (Sec. 3.2;
  the local-splatting optimisation that follows in the paper is training and is not done);
* so tau is in the paper's units: gaussians_per_group = 4096 * 2 = 8192, and tau_px = 0.5 gives
  the paper's default tau_F = 2048 px^2.

Readings (the paper is silent):
* "scale" in the retention rule is the product of the three axis scales (the volume factor; the
  merge weights of the default generator use the same product), ties kept in index order;
* the library stores at most 64 Gaussians per node, so a cluster is stored as consecutive nodes
  of 64 (Morton order within the cluster, the last one partial) that share the cluster's spheres
  and are therefore always selected together; the nodes of a group hang under the nodes of the
  group's simplified cluster in proportion;
* once one cluster is left, it keeps being halved by the same rule (a group of one) until it
  fits one node, so that the bundle has a single root;
* spheres and their containment as in the default generator (Fig. 4 centre and radius, then
  each group sphere enlarged to hold the group spheres below it).
"""
from __future__ import annotations

import numpy as np

from .assets import (LEAF_SIZE, SPHERE_MARGIN, Asset, _group_spheres, _morton_order, _round_up_f32,
                     leaf_gaussians)

PAPER_CLUSTER = 4096
PAPER_GROUP = 2
SCALE_UP_LOG = float(np.log(2.0) / 6.0)   # scales x 2^(1/6)


def median_split(means: np.ndarray, idx: np.ndarray, max_size: int) -> list[np.ndarray]:
    """Binary median split of the points ``means[idx]``: parts of at most ``max_size``, in split
    order (the lower half first), so that consecutive parts are siblings."""
    if len(idx) <= max_size:
        return [idx]
    p = means[idx].astype(np.float64)
    axis = int(np.argmax(p.max(axis=0) - p.min(axis=0)))
    order = np.argsort(p[:, axis], kind="stable")
    half = len(idx) // 2
    return median_split(means, idx[order[:half]], max_size) + median_split(means, idx[order[half:]], max_size)


def simplify(arrs, members: np.ndarray):
    """One group's simplified cluster: the larger half (by s1 s2 s3 * opacity) of its Gaussians,
    scales multiplied by 2^(1/6); returned in index order."""
    means, log_scales, quats, opacity, sh = arrs
    ls = log_scales[members].astype(np.float64)
    score = np.exp(ls.sum(axis=1)) * opacity[members].astype(np.float64)
    keep_n = (len(members) + 1) // 2
    # stable: among equal scores the earlier Gaussian wins
    top = np.sort(np.argsort(-score, kind="stable")[:keep_n])
    kept = members[top]
    out = [a[kept].copy() for a in arrs]
    out[1] = (out[1].astype(np.float64) + SCALE_UP_LOG).astype(np.float32)
    return out


def make_asset_paper(seed: int, n_leaves: int, cluster: int = PAPER_CLUSTER) -> Asset:
    """An asset with the paper's bundle shape (binary tree of 4096-Gaussian clusters)."""
    leaves = leaf_gaussians(seed, n_leaves)
    parts = median_split(leaves[0], np.arange(n_leaves), cluster)
    # levels[k]: list of clusters, each a list of 5 arrays (Morton order within the cluster)
    def morton(arrs):
        o = _morton_order(arrs[0])
        return [a[o] for a in arrs]
    levels = [[morton([a[p] for a in leaves]) for p in parts]]
    groups = []   # groups[k][j]: indices (into levels[k]) of the clusters simplified into levels[k + 1][j]
    while len(levels[-1]) > 1 or levels[-1][0][0].shape[0] > LEAF_SIZE:
        cur = levels[-1]
        if len(cur) > 1:
            g = [list(range(j, min(j + PAPER_GROUP, len(cur)))) for j in range(0, len(cur), PAPER_GROUP)]
        else:
            g = [[0]]
        nxt = []
        for members in g:
            cat = [np.concatenate([cur[m][i] for m in members]) for i in range(5)]
            nxt.append(morton(simplify(cat, np.arange(cat[0].shape[0]))))
        groups.append(g)
        levels.append(nxt)

    # nodes: each cluster as consecutive nodes of <= 64 Gaussians, level by level
    node_cluster, node_level, node_first, node_count = [], [], [], []
    cluster_nodes = []   # [k][c] -> (first node, node count)
    g_off = 0
    for k, lev in enumerate(levels):
        cn = []
        for c, arrs in enumerate(lev):
            n = arrs[0].shape[0]
            m = (n + LEAF_SIZE - 1) // LEAF_SIZE
            cn.append((len(node_count), m))
            for q in range(m):
                node_cluster.append((k, c))
                node_level.append(k)
                node_first.append(g_off + q * LEAF_SIZE)
                node_count.append(min(LEAF_SIZE, n - q * LEAF_SIZE))
            g_off += n
        cluster_nodes.append(cn)
    n_nodes = len(node_count)
    node_parent = np.full(n_nodes, -1, np.int32)
    for k, g in enumerate(groups):
        for j, members in enumerate(g):
            pf, pm = cluster_nodes[k + 1][j]
            child_nodes = [cluster_nodes[k][m][0] + q for m in members for q in range(cluster_nodes[k][m][1])]
            for t, node in enumerate(child_nodes):
                node_parent[node] = pf + (t * pm) // len(child_nodes)

    # spheres of every group (Fig. 4), then containment from the bottom up
    def sphere(arr_list):
        p = np.concatenate(arr_list)
        return _group_spheres(p, np.array([0]), np.array([p.shape[0]], np.int64))[0]
    group_sph = [[sphere([levels[k][m][0] for m in members]) for members in g] for k, g in enumerate(groups)]
    root_sph = sphere([levels[-1][0][0]])
    group_of = [{m: j for j, members in enumerate(g) for m in members} for g in groups]
    for k in range(1, len(groups)):
        for j, members in enumerate(groups[k]):
            s = group_sph[k][j]
            need = float(s[3])
            for m in members:   # cluster m of level k is what group m of level k - 1 became
                below = group_sph[k - 1][m]
                d = float(np.linalg.norm(s[:3].astype(np.float64) - below[:3].astype(np.float64)))
                need = max(need, (d + float(below[3])) * (1.0 + SPHERE_MARGIN))
            s[3] = _round_up_f32(np.array([need]))[0]
    if groups:
        below = group_sph[-1][0]
        d = float(np.linalg.norm(root_sph[:3].astype(np.float64) - below[:3].astype(np.float64)))
        need = max(float(root_sph[3]), (d + float(below[3])) * (1.0 + SPHERE_MARGIN))
        root_sph[3] = _round_up_f32(np.array([need]))[0]
    own = np.empty((n_nodes, 4), np.float32)
    for node, (k, c) in enumerate(node_cluster):
        own[node] = root_sph if k == len(levels) - 1 else group_sph[k][group_of[k][c]]

    cat = [np.concatenate([arrs[i] for lev in levels for arrs in lev]) for i in range(5)]
    return Asset(means=np.ascontiguousarray(cat[0]), log_scales=np.ascontiguousarray(cat[1]),
                 quats=np.ascontiguousarray(cat[2]), opacity=np.ascontiguousarray(cat[3]),
                 sh=np.ascontiguousarray(cat[4]), node_first=np.asarray(node_first, np.uint32),
                 node_count=np.asarray(node_count, np.uint32), node_level=np.asarray(node_level, np.uint8),
                 node_parent=node_parent, own_sphere=own, gaussians_per_group=cluster * PAPER_GROUP)
