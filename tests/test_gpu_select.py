"""GPU selection (Sec. 3.3-3.4) against the FP64 oracle: the cut is bit-exact, near ties excluded."""
import numpy as np
import pytest

import oracle
from synth import scenes
from v3dg_cases import assert_cut_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Context():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2505_06523_gb300 import Context
    return Context


@pytest.fixture(scope="module")
def orbit_asset():
    from synth.assets import cached_asset
    return cached_asset(1, 1_000_000)


def test_cut_tiny(Context, tiny_asset):
    cam = scenes.tiny_camera()
    inst = scenes.single_instance()
    with Context(0) as ctx:
        ctx.load_hierarchy(tiny_asset)
        ctx.set_instances(inst)
        ctx.select(cam, 1.0)
        got = ctx.get_cut()
        st = ctx.frame_stats()
    cut = oracle.select([tiny_asset], inst, cam, 1.0)
    assert_cut_parity(got, cut)
    assert st["cut_nodes"] == len(got)
    assert st["cut_gaussians"] == int(tiny_asset.node_count[got[:, 1]].sum())


@pytest.mark.parametrize("k", range(8))
def test_cut_orbit(Context, orbit_asset, k):
    d = scenes.orbit_distances()[k]
    cam = scenes.orbit_camera(d)
    inst = scenes.single_instance()
    with Context(0) as ctx:
        ctx.load_hierarchy(orbit_asset)
        ctx.set_instances(inst)
        for tau in (0.5, 1.0, 2.0, 4.0):
            ctx.select(cam, tau)
            got = ctx.get_cut()
            cut = oracle.select([orbit_asset], inst, cam, tau)
            assert_cut_parity(got, cut)


def test_tau_limits(Context, tiny_asset):
    inst = scenes.subset(scenes.crowd_instances(8, n_assets=1), np.arange(8))
    inst.trans[:, :2] *= 0.05
    cam = scenes.orbit_camera(60.0, 640, 480)
    root = int(np.nonzero(tiny_asset.node_parent < 0)[0][0])
    leaves = np.nonzero(tiny_asset.node_level == 0)[0]
    with Context(0) as ctx:
        ctx.load_hierarchy(tiny_asset)
        ctx.set_instances(inst)
        ctx.select(cam, 0.0)
        got = ctx.get_cut()
        assert len(got) == inst.n * len(leaves)
        assert (got[:, 1] == np.tile(leaves, inst.n)).all()
        ctx.select(cam, 1e18)
        got = ctx.get_cut()
        assert got[:, 1].tolist() == [root] * inst.n


def test_cut_crowd_decimated(Context, tiny_asset, small_asset):
    inst = scenes.crowd_instances(200, n_assets=2, half_extent=70.0)
    assets = [tiny_asset, small_asset]
    with Context(0) as ctx:
        for a in assets:
            ctx.load_hierarchy(a)
        ctx.set_instances(inst)
        for t in (0, 40, 150, 299):
            cam = scenes.crowd_camera(t)
            for tau in (0.5, 1.0, 4.0):
                ctx.select(cam, tau)
                assert_cut_parity(ctx.get_cut(), oracle.select(assets, inst, cam, tau))


def test_empty_scene(Context, tiny_asset):
    with Context(0) as ctx:
        ctx.load_hierarchy(tiny_asset)
        inst = scenes.single_instance()
        ctx.set_instances(scenes.subset(inst, np.zeros(0, np.int64)))
        ctx.select(scenes.tiny_camera(), 1.0)
        assert len(ctx.get_cut()) == 0
        rgb, T = ctx.render(want_T=True)
        assert float(rgb.abs().max()) == 0.0 and float(T.min()) == 1.0


def _cut_and_frame(Context, assets, inst, cams, tau, topdown):
    from paper_2505_06523_gb300._native import V3DG_OPT_SELECT_TOPDOWN
    out = []
    with Context(0) as ctx:
        ctx.set_option(V3DG_OPT_SELECT_TOPDOWN, int(topdown))
        for a in assets:
            ctx.load_hierarchy(a)
        ctx.set_instances(inst)
        for cam in cams:
            ctx.select(cam, tau)
            rgb, T = ctx.render(want_T=True)
            out.append((ctx.get_cut(), ctx.frame_stats(), rgb.cpu().numpy(), T.cpu().numpy()))
    return out


@pytest.mark.parametrize("tau", [0.5, 1.0, 4.0])
def test_topdown_equals_flat(Context, tiny_asset, small_asset, tau):
    """Top-down selection: the same cut (against the oracle too), the same render list size and
    the same image, bit for bit, as the flat kernel."""
    inst = scenes.crowd_instances(200, n_assets=2, half_extent=70.0)
    assets = [tiny_asset, small_asset]
    cams = [scenes.crowd_camera(t, 640, 360) for t in (0, 40, 150)] + [scenes.orbit_camera(2.0, 320, 200)]
    flat = _cut_and_frame(Context, assets, inst, cams, tau, False)
    td = _cut_and_frame(Context, assets, inst, cams, tau, True)
    for cam, (c0, s0, rgb0, t0), (c1, s1, rgb1, t1) in zip(cams, flat, td):
        assert np.array_equal(c0, c1)
        assert_cut_parity(c1, oracle.select(assets, inst, cam, tau))
        for k in ("cut_nodes", "cut_gaussians", "render_nodes", "visible", "pairs"):
            assert s0[k] == s1[k], k
        assert np.array_equal(rgb0, rgb1) and np.array_equal(t0, t1)


def test_topdown_tau_limits(Context, tiny_asset):
    """tau -> 0 selects every leaf and tau -> inf every root, walking the whole tree."""
    from paper_2505_06523_gb300._native import V3DG_OPT_SELECT_TOPDOWN
    inst = scenes.subset(scenes.crowd_instances(8, n_assets=1), np.arange(8))
    inst.trans[:, :2] *= 0.05
    cam = scenes.orbit_camera(60.0, 640, 480)
    root = int(np.nonzero(tiny_asset.node_parent < 0)[0][0])
    leaves = np.nonzero(tiny_asset.node_level == 0)[0]
    with Context(0) as ctx:
        ctx.set_option(V3DG_OPT_SELECT_TOPDOWN, 1)
        ctx.load_hierarchy(tiny_asset)
        ctx.set_instances(inst)
        ctx.select(cam, 0.0)
        got = ctx.get_cut()
        assert len(got) == inst.n * len(leaves) and (got[:, 1] == np.tile(leaves, inst.n)).all()
        ctx.select(cam, 1e18)
        assert ctx.get_cut()[:, 1].tolist() == [root] * inst.n
