"""Checks of the synthetic hierarchy generator against the definitions it follows (Sec. 3.3-3.4)."""
import numpy as np

from synth import scenes
from synth.assets import BRANCH, LEAF_SIZE, make_asset


def test_tree_shape(small_asset):
    a = small_asset
    lv, par = a.node_level, a.node_parent
    assert (par[lv == lv.max()] == -1).all() and (lv[par < 0] == lv.max()).all()
    assert (lv[par[par >= 0]] == lv[par >= 0] + 1).all()
    assert (a.node_count >= 1).all() and (a.node_count <= LEAF_SIZE).all()
    # nodes' Gaussian ranges tile the Gaussian array in node order
    assert a.node_first[0] == 0
    assert (a.node_first[1:] == a.node_first[:-1] + a.node_count[:-1]).all()
    assert int(a.node_first[-1] + a.node_count[-1]) == a.n_gauss
    # 4-ary: at most BRANCH children per parent
    assert np.bincount(par[par >= 0]).max() <= BRANCH
    assert int((lv == 0).sum()) == (20_000 + LEAF_SIZE - 1) // LEAF_SIZE


def test_group_sphere_bounds_its_gaussians(small_asset):
    """Own sphere = sphere of the node's cluster group: it contains every Gaussian mean of the group."""
    a = small_asset
    for n in range(a.n_nodes):
        c, r = a.own_sphere[n, :3].astype(np.float64), float(a.own_sphere[n, 3])
        mu = a.means[a.node_first[n]:a.node_first[n] + a.node_count[n]].astype(np.float64)
        assert (np.linalg.norm(mu - c, axis=1) <= r).all()


def test_group_sphere_centre_is_mean_before_enlargement():
    a = make_asset(11, 3000)
    # a leaf group's centre is the mean of its members' Gaussians (Fig. 4)
    par = a.node_parent
    for p in np.unique(par[(a.node_level == 0) & (par >= 0)])[:10]:
        kids = np.nonzero(par == p)[0]
        mu = np.concatenate([a.means[a.node_first[k]:a.node_first[k] + a.node_count[k]] for k in kids])
        np.testing.assert_allclose(a.own_sphere[kids[0], :3], mu.astype(np.float64).mean(axis=0), rtol=0, atol=1e-6)
        assert (a.own_sphere[kids] == a.own_sphere[kids[0]]).all()


def test_containment(small_asset):
    """Each node's own sphere contains its children's own sphere (r_p > r_c, Sec. 3.4)."""
    a = small_asset
    ch = np.nonzero(a.node_parent >= 0)[0]
    p = a.node_parent[ch]
    d = np.linalg.norm(a.own_sphere[p, :3].astype(np.float64) - a.own_sphere[ch, :3].astype(np.float64), axis=1)
    assert (d + a.own_sphere[ch, 3] <= a.own_sphere[p, 3]).all()
    assert (a.own_sphere[p, 3] > a.own_sphere[ch, 3]).all()


def test_deterministic():
    a, b = make_asset(4, 5000), make_asset(4, 5000)
    for k in ("means", "sh", "own_sphere", "node_first"):
        assert (getattr(a, k) == getattr(b, k)).all()


def test_merged_gaussian_moments():
    """A parent Gaussian made of two equal-weight children has their mean as its mean."""
    from synth.assets import merge_pairs
    mu = np.array([[0.0, 0, 0], [1.0, 0, 0]], np.float32)
    ls = np.full((2, 3), np.log(0.1), np.float32)
    q = np.array([[1.0, 0, 0, 0], [1.0, 0, 0, 0]], np.float32)
    o = np.array([0.5, 0.5], np.float32)
    sh = np.zeros((2, 16, 3), np.float32)
    m, nls, nq, no, nsh = merge_pairs(mu, ls, q, o, sh, np.array([0]), np.array([1]))
    np.testing.assert_allclose(m[0], [0.5, 0, 0], atol=1e-7)
    # variance along x: 0.01 + 0.25, others 0.01; opacity 1 - 0.25
    np.testing.assert_allclose(np.sort(np.exp(2 * nls[0].astype(np.float64))), [0.01, 0.01, 0.26], rtol=1e-5)
    assert no[0] == np.float32(0.75)


def test_crowd_layout():
    inst = scenes.crowd_instances()
    assert inst.n == 1000
    r = np.linalg.norm(inst.trans[:, :2], axis=1)
    assert (np.abs(r - scenes.CROWD_RING) >= 3.5).all()
    assert (inst.scale >= 0.5).all() and (inst.scale <= 2.0).all()
    np.testing.assert_allclose(np.einsum("nij,nkj->nik", inst.rot, inst.rot), np.tile(np.eye(3), (1000, 1, 1)), atol=1e-12)
    cam = scenes.crowd_camera(0)
    assert np.allclose(cam.center, [60.0, 0.0, 1.7])
