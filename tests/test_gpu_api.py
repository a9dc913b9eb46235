"""Error behaviour of the C ABI on a GPU (statuses, unchanged state, no CPU fallback)."""
import numpy as np
import pytest

from synth import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2505_06523_gb300 import _native
    return _native


def test_render_without_select(native, small_asset):
    from paper_2505_06523_gb300 import Context, V3dgError
    with Context(0) as ctx:
        ctx.load_hierarchy(small_asset)
        ctx.set_instances(scenes.single_instance())
        ctx.cam = scenes.tiny_camera()
        with pytest.raises(V3dgError) as e:
            ctx.render()
        assert e.value.status == native.V3DG_ENOTFOUND


def test_select_without_assets(native):
    from paper_2505_06523_gb300 import Context, V3dgError
    with Context(0) as ctx:
        with pytest.raises(V3dgError) as e:
            ctx.select(scenes.tiny_camera(), 1.0)
        assert e.value.status == native.V3DG_ENOTFOUND


def test_bad_hierarchy_rejected(native, small_asset):
    import copy
    from paper_2505_06523_gb300 import Context, V3dgError
    with Context(0) as ctx:
        for mutate in ("count", "parent", "sphere", "range", "roots"):
            a = copy.deepcopy(small_asset)
            if mutate == "count":
                a.node_count[3] = 65
            elif mutate == "parent":
                a.node_parent[0] = 0
            elif mutate == "sphere":
                a.own_sphere[5, 3] = np.nan
            elif mutate == "range":
                a.node_first[-1] = a.n_gauss
            else:
                a.node_parent[np.nonzero(a.node_level == a.node_level.max())[0]] = -1
                a.node_parent[0] = -1
            with pytest.raises(V3dgError) as e:
                ctx.load_hierarchy(a)
            assert e.value.status == native.V3DG_EINVAL, mutate
        # a good one still loads with id 0: the failures changed nothing
        assert ctx.load_hierarchy(small_asset) == 0


def test_bad_instances_and_camera(native, small_asset):
    from paper_2505_06523_gb300 import Context, V3dgError
    with Context(0) as ctx:
        ctx.load_hierarchy(small_asset)
        inst = scenes.single_instance()
        inst.asset[0] = 3
        with pytest.raises(V3dgError) as e:
            ctx.set_instances(inst)
        assert e.value.status == native.V3DG_ENOTFOUND
        inst = scenes.single_instance()
        inst.scale[0] = 0.0
        with pytest.raises(V3dgError) as e:
            ctx.set_instances(inst)
        assert e.value.status == native.V3DG_EINVAL
        ctx.set_instances(scenes.single_instance())
        cam = scenes.tiny_camera()
        cam.width = 0
        with pytest.raises(V3dgError) as e:
            ctx.select(cam, 1.0)
        assert e.value.status == native.V3DG_EINVAL
        with pytest.raises(V3dgError):
            ctx.select(scenes.tiny_camera(), -1.0)


def test_launch_counter_and_stage_times(native, small_asset):
    from paper_2505_06523_gb300 import Context
    with Context(0) as ctx:
        ctx.set_option(native.V3DG_OPT_STAGE_TIMING, 1)
        ctx.load_hierarchy(small_asset)
        ctx.set_instances(scenes.single_instance())
        n0 = ctx.launches()
        ctx.select(scenes.tiny_camera(), 1.0)
        ctx.render()
        ms, n1 = ctx.stage_times()
        assert n1 - n0 >= 10
        assert all(m >= 0 for m in ms) and sum(ms) > 0


def test_work_counting_changes_nothing(native, small_asset):
    from paper_2505_06523_gb300 import Context
    cam = scenes.look_at((0.0, -2.6, 0.4), (0.0, 0.0, 0.0), 160, 120, 60.0)
    with Context(0) as ctx:
        ctx.load_hierarchy(small_asset)
        ctx.set_instances(scenes.single_instance())
        ctx.select(cam, 1.0)
        a, _ = ctx.render()
        a = a.cpu().numpy()
        st0 = ctx.frame_stats()
        ctx.set_option(native.V3DG_OPT_COUNT_WORK, 1)
        ctx.select(cam, 1.0)
        b, _ = ctx.render()
        st = ctx.frame_stats()
    assert (a == b.cpu().numpy()).all()
    assert st0["blend_evals"] == 0
    assert 0 < st["blend_contribs"] <= st["blend_evals"] <= st["pairs"] * 256
