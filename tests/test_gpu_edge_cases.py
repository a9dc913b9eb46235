"""Degenerate cases of the splatting path and the bounded device-side waits.

* Near-singular 2D covariances (Sec. 5.1 renders without the 2D dilation, eps2d = 0): thin
  needles and an edge-on disc, on and off the optical axis, whose det(Sigma_2D) is far below
  1e-12 px^4.  The kernel forms and inverts those in FP64; records and image are compared with the
  FP64 oracle element by element, and the frame counter shows that the FP64 branch ran.
* The waits of the chained scans give up after a bounded number of polls: a look-back whose
  predecessor never publishes returns V3DG_ETIMEOUT, and the context keeps working.
"""
import math
import types

import numpy as np
import pytest

import oracle
from synth import scenes

pytestmark = pytest.mark.gpu

F32 = np.float32


@pytest.fixture(scope="module")
def Context():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2505_06523_gb300 import Context
    return Context


def _quat(axis, deg):
    ax = np.asarray(axis, float) / np.linalg.norm(axis)
    a = math.radians(deg) / 2
    return [math.cos(a), *(math.sin(a) * ax)]


# (mean, quaternion, log-scales): each mean projects exactly onto a pixel centre of the camera
# below (X/Z, Y/Z and f X/Z + c are exact in binary), so the screen position carries no rounding
# on either side and the image compares at the one pixel each Gaussian reaches.
NEEDLES = [
    ((0, 0, 4), _quat((0, 0, 1), 45), (math.log(5e-3), math.log(5e-7), math.log(5e-7))),
    ((2, 1, 4), _quat((0, 0, 1), 30), (math.log(5e-3), math.log(5e-7), math.log(5e-7))),
    ((-3, 2, 8), _quat((0, 0, 1), 60), (math.log(8e-3), math.log(4e-7), math.log(4e-7))),
    ((5.5, -1, 4), _quat((0, 0, 1), -20), (math.log(4e-3), math.log(5e-7), math.log(5e-7))),
    ((1, -2, 2), _quat((0, 0, 1), 75), (math.log(2e-3), math.log(2e-7), math.log(2e-7))),
    ((0, 0, 6), [1, 0, 0, 0], (math.log(5e-3), math.log(5e-7), math.log(5e-3))),        # disc seen edge-on
    ((2, 1, 8), _quat((1, 1, 0), 35), (math.log(6e-3), math.log(3e-7), math.log(3e-7))),  # tilted out of the image plane
]


def needle_asset():
    """One leaf per Gaussian (so each Gaussian is its node's centre) under a root that is never
    selected at tau = 0."""
    n = len(NEEDLES)
    means = [m for m, _, _ in NEEDLES] + [(0, 0, 100.0)]
    rng = np.random.default_rng(21)
    sh = rng.normal(0, 0.3, (n + 1, 16, 3))
    return types.SimpleNamespace(
        means=np.asarray(means, F32), log_scales=np.asarray([l for _, _, l in NEEDLES] + [(-5, -5, -5)], F32),
        quats=np.asarray([q for _, q, _ in NEEDLES] + [[1, 0, 0, 0]], F32),
        opacity=np.asarray(rng.uniform(0.3, 0.95, n + 1), F32), sh=sh.astype(F32),
        node_first=np.arange(n + 1, dtype=np.uint32), node_count=np.ones(n + 1, np.uint32),
        node_level=np.array([0] * n + [1], np.uint8), node_parent=np.array([n] * n + [-1], np.int32),
        own_sphere=np.array([[*m, 1e-3] for m in means[:n]] + [[0, 0, 5, 200.0]], F32), gaussians_per_group=256)


def test_near_singular_conics(Context):
    from paper_2505_06523_gb300._native import V3DG_OPT_COUNT_WORK
    asset = needle_asset()
    inst = scenes.single_instance()
    cam = scenes.Camera(np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1), 40.0, 40.0, 64.5, 48.5, 192, 128)
    with Context(0) as ctx:
        ctx.set_option(V3DG_OPT_COUNT_WORK, 1)
        ctx.load_hierarchy(asset)
        ctx.set_instances(inst)
        ctx.select(cam, 0.0)
        rgb, T = ctx.render(want_T=True)
        rgb, T = rgb.cpu().numpy().astype(np.float64), T.cpu().numpy().astype(np.float64)
        g = ctx.get_projected()
        st = ctx.frame_stats()
    cut = oracle.select([asset], inst, cam, 0.0)
    p = oracle.project([asset], inst, cam, cut)
    n = len(NEEDLES)
    det = p.cov[:, 0] * p.cov[:, 2] - p.cov[:, 1] ** 2
    assert len(cut.inst) == n and (det < 1e-12).all() and p.visible.all()
    # every Gaussian took the FP64 inverse
    assert st["conic_fp64"] == n, st
    # records, element by element (the screen means are exact, so no Gaussian sits near a tile edge)
    assert g["local"].tolist() == list(range(n))
    assert np.abs(g["u"].astype(np.float64) - p.u).max() <= 1e-6
    rel = np.abs(g["conic"].astype(np.float64) - p.conic).max(axis=1) / np.abs(p.conic).max(axis=1)
    assert rel.max() <= 1e-5, rel
    assert np.abs(g["rgb"].astype(np.float64) - p.rgb).max() <= 2e-6
    assert (g["depth_key"] == p.depth_key).all()
    # the image: each Gaussian reaches exactly the pixel under its mean
    C, To, B = oracle.render_image(p, cam.width, cam.height)
    assert (To < 1).sum() == n - 1   # two Gaussians share the pixel on the optical axis
    assert np.abs(rgb - C).max() <= 1e-6 and np.abs(T - To).max() <= 1e-6


def test_bounded_wait_gives_up(Context, small_asset):
    """A look-back whose predecessor never publishes gives up after the poll limit: the kernel
    returns, the call reports V3DG_ETIMEOUT, and the next frame renders normally."""
    from paper_2505_06523_gb300 import _native as N
    cam = scenes.look_at((0.3, -2.4, 0.5), (0.0, 0.0, 0.0), 128, 96, 60.0)
    with Context(0) as ctx:
        assert N.v3dg_check_wait(ctx.ctx, 1000, True) == 1000
        with pytest.raises(N.V3dgError) as e:
            N.v3dg_check_wait(ctx.ctx, 1000, False)
        assert e.value.status == N.V3DG_ETIMEOUT
        with pytest.raises(N.V3dgError) as e:
            N.v3dg_check_wait(ctx.ctx, 0, False)
        assert e.value.status == N.V3DG_EINVAL
        ctx.load_hierarchy(small_asset)
        ctx.set_instances(scenes.single_instance())
        ctx.select(cam, 1.0)
        a = ctx.render()[0].cpu().numpy()
        st = ctx.frame_stats()
        assert not st["timeout"] and not st["overflow"] and float(np.abs(a).sum()) > 0
        assert N.v3dg_check_wait(ctx.ctx, 1 << 20, True) == 1000
