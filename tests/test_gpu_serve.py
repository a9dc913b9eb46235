"""Request server (v3dg_server_start / v3dg_submit / v3dg_poll) on a GPU.

Each request repeats the per-frame path (selection, Sec. 3.4; splatting, Sec. 2.1) for its own
scene, camera and tolerance.  The kernels make no result depend on timing (stable sorts, fixed
blend order), so a frame rendered alone through the plain API and the same frame rendered while
others run on the server's slots must agree bit for bit; one of them is also checked against the
oracle.
"""
import numpy as np
import pytest

import oracle
from synth import scenes
from v3dg_cases import IMG_ABS, PSNR_MIN, image_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2505_06523_gb300 import Context, _native
    return Context, _native


def _requests():
    """Mixed requests: instance subsets of one crowd layout, several resolutions, cameras and tau."""
    crowd = scenes.crowd_instances(200, n_assets=2, half_extent=70.0)
    rng = np.random.default_rng(11)
    out = []
    sizes = [(160, 96), (320, 180), (96, 64), (256, 144)]
    for k in range(10):
        n = [1, 40, 200, 120][k % 4]
        idx = np.sort(rng.choice(200, size=n, replace=False))
        w, h = sizes[k % len(sizes)]
        if k % 5 == 0:
            inst = scenes.single_instance()
            cam = scenes.look_at((0.0, -2.6 - 0.3 * k, 0.4), (0.0, 0.0, 0.0), w, h, 60.0)
        else:
            inst = scenes.subset(crowd, idx)
            cam = scenes.crowd_camera(int(rng.integers(0, 300)), width=w, height=h)
        out.append((inst, cam, [0.5, 1.0, 2.0, 4.0][k % 4]))
    return out


def _alone(Context, assets, reqs):
    imgs = []
    with Context(0) as ctx:
        for a in assets:
            ctx.load_hierarchy(a)
        for inst, cam, tau in reqs:
            ctx.set_instances(inst)
            ctx.select(cam, tau)
            rgb, T = ctx.render_host(want_T=True)
            imgs.append((rgb.copy(), T.copy(), ctx.frame_stats()))
    return imgs


@pytest.mark.parametrize("slots,budget,merge", [(3, 0, 1), (2, 1, 1), (3, 0, 4)])
def test_same_alone_and_in_the_mix(api, tiny_asset, small_asset, slots, budget, merge):
    """Every request's image equals the image of the same frame rendered alone (budget 1 byte
    admits one request at a time; budget 0 lets all slots overlap; merge 4 renders waiting
    requests of one image size together)."""
    Context, N = api
    assets = [tiny_asset, small_asset]
    reqs = _requests()
    alone = _alone(Context, assets, reqs)
    with Context(0) as ctx:
        ctx.set_option(N.V3DG_OPT_SERVE_MERGE, merge)
        for a in assets:
            ctx.load_hierarchy(a)
        ctx.server_start(slots, budget)
        tickets = [ctx.submit(inst, cam, tau, want_T=True) for inst, cam, tau in reqs]
        got = {}
        while len(got) < len(tickets):
            for t in tickets:
                if t not in got:
                    r = ctx.poll(t, 2000)
                    if r is not None:
                        got[t] = r
        ctx.server_stop()
    for k, t in enumerate(tickets):
        rec, rgb, T = got[t]
        a_rgb, a_T, st = alone[k]
        assert rec["status"] == N.V3DG_OK
        assert rec["submit_ms"] <= rec["start_ms"] <= rec["done_ms"]
        if rec["batch_views"] == 1:   # merged frames report the counters of all their views
            assert rec["visible"] == st["visible"] and rec["pairs"] == st["pairs"], k
        assert np.array_equal(rgb, a_rgb), k
        assert np.array_equal(T, a_T), k


@pytest.mark.parametrize("merge", [8, 3])
def test_merged_requests_equal_alone(api, tiny_asset, small_asset, merge):
    """Requests of one image size that wait together are rendered as the views of one frame (each
    its own instances, camera and tau); each image equals the one its request gives alone."""
    Context, N = api
    assets = [tiny_asset, small_asset]
    crowd = scenes.crowd_instances(200, n_assets=2, half_extent=70.0)
    rng = np.random.default_rng(5)
    reqs = []
    for k in range(12):
        idx = np.sort(rng.choice(200, size=[200, 30, 90, 1][k % 4], replace=False))
        reqs.append((scenes.subset(crowd, idx), scenes.crowd_camera(int(rng.integers(0, 300)), width=240, height=136),
                     [0.5, 1.0, 2.0, 4.0][k % 4]))
    alone = _alone(Context, assets, reqs)
    with Context(0) as ctx:
        ctx.set_option(N.V3DG_OPT_SERVE_MERGE, merge)
        for a in assets:
            ctx.load_hierarchy(a)
        ctx.server_start(1)
        tickets = [ctx.submit(inst, cam, tau, want_T=True) for inst, cam, tau in reqs]
        got = {}
        while len(got) < len(tickets):
            for t in tickets:
                if t not in got:
                    r = ctx.poll(t, 2000)
                    if r is not None:
                        got[t] = r
        ctx.server_stop()
    views = [got[t][0]["batch_views"] for t in tickets]
    assert max(views) > 1 and max(views) <= merge, views
    for k, t in enumerate(tickets):
        rec, rgb, T = got[t]
        assert rec["status"] == N.V3DG_OK
        assert np.array_equal(rgb, alone[k][0]) and np.array_equal(T, alone[k][1]), (k, rec["batch_views"])


def test_served_frame_matches_oracle(api, small_asset):
    Context, _ = api
    inst = scenes.single_instance()
    cam = scenes.look_at((0.0, -2.6, 0.4), (0.0, 0.0, 0.0), 96, 80, 60.0)
    with Context(0) as ctx:
        ctx.load_hierarchy(small_asset)
        ctx.server_start(2)
        t = ctx.submit(inst, cam, 1.0)
        r = None
        while r is None:
            r = ctx.poll(t, 100000)
        ctx.server_stop()
    _, rgb, _ = r
    cut = oracle.select([small_asset], inst, cam, 1.0)
    p = oracle.project([small_asset], inst, cam, cut)
    C, _, B = oracle.render_image(p, cam.width, cam.height)
    err, ps, _ = image_errors(rgb, C, B)
    assert err <= IMG_ABS and ps >= PSNR_MIN


def test_server_errors(api, small_asset):
    Context, N = api
    inst = scenes.single_instance()
    cam = scenes.tiny_camera()
    with Context(0) as ctx:
        with pytest.raises(N.V3dgError) as e:
            ctx.server_start(2)
        assert e.value.status == N.V3DG_ENOTFOUND          # no asset loaded yet
        ctx.load_hierarchy(small_asset)
        with pytest.raises(N.V3dgError) as e:
            ctx.server_start(0)
        assert e.value.status == N.V3DG_EINVAL
        with pytest.raises(N.V3dgError) as e:
            ctx.submit(inst, cam, 1.0)
        assert e.value.status == N.V3DG_ENOTFOUND          # no server running
        ctx.server_start(2)
        with pytest.raises(N.V3dgError) as e:
            ctx.server_start(2)
        assert e.value.status == N.V3DG_EBUSY
        with pytest.raises(N.V3dgError) as e:
            ctx.set_option(N.V3DG_OPT_SPLIT_PAIRS, 4096)
        assert e.value.status == N.V3DG_EBUSY
        with pytest.raises(N.V3dgError) as e:
            ctx.load_hierarchy(small_asset)
        assert e.value.status == N.V3DG_EBUSY
        bad = scenes.single_instance()
        bad.asset[0] = 5
        with pytest.raises(N.V3dgError) as e:
            ctx.submit(bad, cam, 1.0)
        assert e.value.status == N.V3DG_ENOTFOUND
        bad = scenes.single_instance()
        bad.scale[0] = -1.0
        with pytest.raises(N.V3dgError) as e:
            ctx.submit(bad, cam, 1.0)
        assert e.value.status == N.V3DG_EINVAL
        with pytest.raises(N.V3dgError) as e:
            ctx.submit(inst, cam, -1.0)
        assert e.value.status == N.V3DG_EINVAL
        with pytest.raises(N.V3dgError) as e:
            N.v3dg_poll(ctx.ctx, 12345, 0)
        assert e.value.status == N.V3DG_ENOTFOUND
        t = ctx.submit(inst, cam, 1.0)
        r = None
        while r is None:
            r = ctx.poll(t, 100000)
        with pytest.raises(N.V3dgError) as e:
            N.v3dg_poll(ctx.ctx, t, 0)                     # already reported
        assert e.value.status == N.V3DG_ENOTFOUND
        # the plain API still works beside a running server
        ctx.set_instances(inst)
        ctx.select(cam, 1.0)
        rgb, _ = ctx.render_host()
        assert np.array_equal(rgb, r[1])
        ctx.server_stop()
        ctx.set_option(N.V3DG_OPT_SPLIT_PAIRS, 4096)        # allowed again


def test_stop_drains_the_queue(api, small_asset):
    """server_stop finishes queued requests (their images are written) before it returns."""
    Context, _ = api
    inst = scenes.single_instance()
    cams = [scenes.look_at((0.0, -2.0 - 0.2 * k, 0.3), (0.0, 0.0, 0.0), 128, 96, 60.0) for k in range(8)]
    with Context(0) as ctx:
        ctx.load_hierarchy(small_asset)
        ctx.server_start(1)
        tickets = [ctx.submit(inst, c, 1.0) for c in cams]
        outs = [ctx._requests[t][0] for t in tickets]
        ctx.server_stop()
        ref = []
        ctx.set_instances(inst)
        for c in cams:
            ctx.select(c, 1.0)
            ref.append(ctx.render_host()[0].copy())
    for o, r in zip(outs, ref):
        assert np.array_equal(o.numpy(), r)
