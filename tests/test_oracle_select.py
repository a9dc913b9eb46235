"""Pins for the oracle's footprint and selection (Sec. 3.3 Fig. 4, Sec. 3.4)."""
import math
import os
import types

import numpy as np
import pytest

import oracle
from synth import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _identity_inst():
    return scenes.single_instance()


def _camera_looking_x(eye_x, f):
    # camera at (eye_x, 0, 0) looking along +x, world z up
    return scenes.look_at((eye_x, 0.0, 0.0), (eye_x + 1.0, 0.0, 0.0), 200, 200, 2 * math.degrees(math.atan(100.0 / f)))


def test_footprint_hand_value():
    # unit sphere 3 units in front of a 256x256 camera with a 60 deg horizontal fov
    cam = scenes.tiny_camera()
    m = oracle.compose(cam.world_to_cam, np.eye(3)[None], np.zeros((1, 3)), np.ones(1))[0]
    f = oracle.footprint(np.zeros((1, 3)), np.ones(1), m, 1.0, cam.fx, cam.fy)[0]
    # f = 128 / tan(30 deg) = 221.70250 px, F = pi * 1 * f^2 / 9
    assert cam.fx == pytest.approx(221.7025033688163, rel=1e-7)
    assert f == pytest.approx(17157.28, rel=1e-5)


def _raycast_area(c, r, f, half=64, sub=16):
    """Pixel area of a sphere's silhouette by casting sub x sub rays per pixel around its centre."""
    u0, v0 = f * c[0] / c[2], f * c[1] / c[2]
    n = 2 * half * sub
    g = (np.arange(n) + 0.5) / sub - half
    xs, ys = np.meshgrid(u0 + g, v0 + g)
    d = np.stack([xs / f, ys / f, np.ones_like(xs)], axis=-1)
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    cross = np.cross(np.broadcast_to(c, d.shape), d)
    hit = np.linalg.norm(cross, axis=-1) <= r
    return hit.sum() / (sub * sub)


@pytest.mark.parametrize("c,r", [((0.0, 0.0, 8.0), 1.0), ((2.0, 1.0, 8.0), 1.0), ((-1.5, 0.5, 5.0), 0.6)])
def test_footprint_against_raycast_area(c, r):
    """F = pi r^2 f^2 / z^2 approximates the silhouette area; the ratio is a closed form.

    The silhouette of a sphere at distance l (depth z) is an ellipse of area
    pi r^2 f^2 sqrt(l^2 - r^2) / (z^2 - r^2)^(3/2); ray casting measures that area directly.
    """
    f = 100.0
    c = np.array(c)
    m = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
    F = oracle.footprint(c[None], np.array([r]), m, 1.0, f, f)[0]
    area = _raycast_area(c, r, f)
    z, l2 = c[2], float(c @ c)
    ratio = (z * z - r * r) ** 1.5 / (z * z * math.sqrt(l2 - r * r))
    assert F / area == pytest.approx(ratio, rel=5e-3)


def test_footprint_instance_scale_equals_world_sphere():
    rng = np.random.default_rng(5)
    cam = scenes.orbit_camera(6.0)
    rot = scenes.random_rotations(rng, 1)
    t = np.array([[0.3, -0.2, 0.5]])
    s = np.array([1.7])
    c = rng.normal(size=(20, 3)) * 0.5
    r = rng.uniform(0.05, 0.3, 20)
    m = oracle.compose(cam.world_to_cam, rot, t, s)[0]
    f_inst = oracle.footprint(c, r, m, 1.7, cam.fx, cam.fy)
    cw = (s[0] * (rot[0] @ c.T)).T + t[0]
    m0 = oracle.compose(cam.world_to_cam, np.eye(3)[None], np.zeros((1, 3)), np.ones(1))[0]
    f_world = oracle.footprint(cw, s[0] * r, m0, 1.0, cam.fx, cam.fy)
    np.testing.assert_allclose(f_inst, f_world, rtol=1e-12)


def test_footprint_straddling_sphere_is_unbounded():
    m = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
    f = oracle.footprint(np.array([[0.0, 0.0, 0.5], [0.0, 0.0, -3.0]]), np.array([0.6, 1.0]), m, 1.0, 100.0, 100.0)
    assert np.isinf(f[0])
    # behind the camera the footprint mirrors the one in front (z enters squared)
    g = oracle.footprint(np.array([[0.0, 0.0, 3.0]]), np.array([1.0]), m, 1.0, 100.0, 100.0)
    assert f[1] == pytest.approx(g[0])


def _load_tree():
    nodes, foot, cuts = [], {}, []
    with open(os.path.join(GOLDEN, "select_tree8.txt")) as fh:
        for line in fh:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "node":
                nodes.append([float(x) for x in t[1:]])
            elif t[0] == "footprint":
                foot[t[1]] = float(t[2])
            elif t[0] == "cut":
                cuts.append((float(t[1]), [int(x) for x in t[2:]]))
    a = np.array(nodes)
    asset = types.SimpleNamespace(
        node_level=a[:, 1].astype(np.uint8), node_parent=a[:, 2].astype(np.int32),
        own_sphere=a[:, 3:7].astype(np.float32), gaussians_per_group=1)
    return asset, foot, cuts


def test_select_hand_worked_tree():
    asset, foot, cuts = _load_tree()
    cam = _camera_looking_x(-11.0, 100.0)
    assert cam.fx == pytest.approx(100.0, rel=1e-6)
    inst = _identity_inst()
    m = oracle.compose(cam.world_to_cam, inst.rot, inst.trans, inst.scale)[0]
    sph = asset.own_sphere
    for name, idx in (("GX", 8), ("GY", 10), ("GXY", 12), ("GR", 14)):
        f = oracle.footprint(sph[idx:idx + 1, :3], sph[idx:idx + 1, 3], m, 1.0, cam.fx, cam.fy)[0]
        assert f == pytest.approx(foot[name], rel=2e-6)
    for tau_f, expect in cuts:
        cut = oracle.select([asset], inst, cam, math.sqrt(tau_f))
        assert cut.node.tolist() == expect, tau_f
        assert len(cut.ties) == 0


def test_tau_zero_selects_all_leaves(tiny_asset):
    cam = scenes.tiny_camera()
    cut = oracle.select([tiny_asset], scenes.single_instance(), cam, 0.0)
    leaves = np.nonzero(tiny_asset.node_level == 0)[0]
    assert cut.node.tolist() == leaves.tolist()


def test_tau_infinite_selects_roots(tiny_asset):
    cam = scenes.orbit_camera(60.0, 640, 480)
    inst = scenes.subset(scenes.crowd_instances(8, n_assets=1), np.arange(8))
    inst.trans[:, :2] *= 0.05          # keep the instances in front, clear of the camera plane
    cut = oracle.select([tiny_asset], inst, cam, 1e18)
    root = int(np.nonzero(tiny_asset.node_parent < 0)[0][0])
    assert cut.node.tolist() == [root] * inst.n
    assert cut.inst.tolist() == list(range(inst.n))


@pytest.mark.parametrize("tau_px", [0.25, 0.5, 1.0, 2.0, 4.0, 16.0])
@pytest.mark.parametrize("dist", [1.5, 3.0, 8.0, 30.0])
def test_exact_cover(tiny_asset, tau_px, dist):
    """Every leaf has exactly one selected node on its path to the root."""
    cam = scenes.orbit_camera(dist, 640, 360)
    cut = oracle.select([tiny_asset], scenes.single_instance(), cam, tau_px)
    sel = np.zeros(tiny_asset.n_nodes, bool)
    sel[cut.node] = True
    cnt = oracle.cover_counts(tiny_asset, sel)
    assert (cnt == 1).all()


def test_siblings_selected_together(tiny_asset):
    cam = scenes.orbit_camera(4.0, 640, 360)
    cut = oracle.select([tiny_asset], scenes.single_instance(), cam, 1.0)
    sel = np.zeros(tiny_asset.n_nodes, bool)
    sel[cut.node] = True
    par = tiny_asset.node_parent
    for p in np.unique(par[sel & (par >= 0)]):
        kids = np.nonzero(par == p)[0]
        assert sel[kids].all()


def test_exact_cover_crowd_subset(tiny_asset, small_asset):
    inst = scenes.crowd_instances(60, n_assets=2)
    cam = scenes.crowd_camera(17)
    cut = oracle.select([tiny_asset, small_asset], inst, cam, 1.0)
    for i in range(inst.n):
        a = [tiny_asset, small_asset][int(inst.asset[i])]
        sel = np.zeros(a.n_nodes, bool)
        sel[cut.node[cut.inst == i]] = True
        assert (oracle.cover_counts(a, sel) == 1).all()
