"""The generator variant with the paper's bundle shape (Sec. 3.1-3.2): 4096-Gaussian clusters by
binary median split, a binary tree of cluster groups simplified by keeping the half with the
larger scale x opacity product and scaling it by 2^(1/6)."""
import numpy as np
import pytest

import oracle
from synth import scenes
from synth.assets import LEAF_SIZE, leaf_gaussians
from synth.paper_tree import make_asset_paper, median_split, simplify


@pytest.fixture(scope="module")
def tree():
    return make_asset_paper(5, 40_000)


def test_shape(tree):
    a = tree
    lv, par = a.node_level, a.node_parent
    assert (par < 0).sum() == 1 and lv[par < 0][0] == lv.max()
    assert (lv[par[par >= 0]] == lv[par >= 0] + 1).all()
    assert (a.node_count >= 1).all() and (a.node_count <= LEAF_SIZE).all()
    assert a.node_first[0] == 0 and (a.node_first[1:] == a.node_first[:-1] + a.node_count[:-1]).all()
    assert a.gaussians_per_group == 8192
    # Gaussians per level halve (each group keeps the larger half of its members)
    per = np.array([a.node_count[lv == k].sum() for k in range(lv.max() + 1)])
    assert per[0] == 40_000
    assert ((per[:-1] + 1) // 2 <= per[1:]).all() and (per[1:] <= per[:-1] // 2 + 8).all()
    assert per[-1] <= LEAF_SIZE


def test_median_split_parts():
    means = leaf_gaussians(2, 20_000)[0]
    parts = median_split(means, np.arange(20_000), 4096)
    assert sorted(np.concatenate(parts).tolist()) == list(range(20_000))
    assert max(len(p) for p in parts) <= 4096 and len(parts) == 8
    # siblings: the first split separates parts 0-3 from 4-7 along the widest axis at the median
    ax = int(np.argmax(means.max(axis=0) - means.min(axis=0)))
    lo = np.concatenate(parts[:4])
    hi = np.concatenate(parts[4:])
    assert len(lo) == len(hi) == 10_000 and means[lo, ax].max() <= means[hi, ax].min()


def test_simplify_keeps_larger_half_and_scales_up():
    rng = np.random.default_rng(0)
    n = 9
    arrs = [rng.normal(size=(n, 3)).astype(np.float32), rng.normal(-3, 0.5, size=(n, 3)).astype(np.float32),
            rng.normal(size=(n, 4)).astype(np.float32), rng.uniform(0.05, 0.95, n).astype(np.float32),
            rng.normal(size=(n, 16, 3)).astype(np.float32)]
    out = simplify(arrs, np.arange(n))
    score = np.exp(arrs[1].astype(np.float64).sum(axis=1)) * arrs[3]
    want = np.sort(np.argsort(-score)[:5])          # ceil(9 / 2) of them, in index order
    assert np.array_equal(out[0], arrs[0][want]) and np.array_equal(out[3], arrs[3][want])
    np.testing.assert_allclose(np.exp(out[1].astype(np.float64)), np.exp(arrs[1][want].astype(np.float64)) * 2 ** (1 / 6),
                               rtol=1e-6)


def test_group_spheres_and_containment(tree):
    a = tree
    # every node's own sphere contains its Gaussians and its children's own spheres
    for n in range(a.n_nodes):
        c, r = a.own_sphere[n, :3].astype(np.float64), float(a.own_sphere[n, 3])
        mu = a.means[a.node_first[n]:a.node_first[n] + a.node_count[n]].astype(np.float64)
        assert (np.linalg.norm(mu - c, axis=1) <= r).all()
    ch = np.nonzero(a.node_parent >= 0)[0]
    p = a.node_parent[ch]
    d = np.linalg.norm(a.own_sphere[p, :3].astype(np.float64) - a.own_sphere[ch, :3].astype(np.float64), axis=1)
    assert (d + a.own_sphere[ch, 3] <= a.own_sphere[p, 3]).all()


def test_exact_cover_and_paper_tau(tree):
    """Every leaf has exactly one selected ancestor; all nodes of a cluster are selected together;
    tau_px = 0.5 is the paper's default tau_F = 2048 px^2 for 4096-Gaussian clusters in pairs."""
    a = tree
    assert oracle.tau_area(0.5, a.gaussians_per_group) == 2048.0
    inst = scenes.single_instance()
    for dist in (2.0, 6.0, 20.0):
        cam = scenes.orbit_camera(dist, 640, 360)
        for tau in (0.25, 0.5, 1.0, 2.0):
            cut = oracle.select([a], inst, cam, tau)
            sel = np.zeros(a.n_nodes, bool)
            sel[cut.node] = True
            assert (oracle.cover_counts(a, sel) == 1).all()
            # nodes sharing an own sphere and a level (one cluster) are selected alike
            key = {}
            for n in range(a.n_nodes):
                k = (int(a.node_level[n]),) + tuple(a.own_sphere[n].tolist()) + (int(a.node_parent[n] >= 0),)
                key.setdefault(k, set()).add(bool(sel[n]))
            assert all(len(v) == 1 for v in key.values())
