"""Host arithmetic of bench.py: the roofline fields of the JSON line and the clock record.

Every figure here is recomputed by hand from the stated unit costs (236 B read per slot, a 48-byte
record, 8-byte pixel box and 4-byte key written per visible Gaussian, 4 B per culled slot, ...),
so a change to the reported arithmetic has to change this file too.
"""
import math

import pytest

import bench

PEAKS = {"hbm_gbs": 1000.0, "sm_max_mhz": 2000.0}
FS = {"visible": 1000.0, "pairs": 3000.0, "render_nodes": 20.0, "blend_evals": 5.0e6, "blend_contribs": 2.0e6}
STAGE_MS = {"select": 0.01, "project": 1.0, "depth_sort": 0.5, "bin": 0.2, "tile_sort": 0.4, "ranges": 0.05,
            "blend": 2.0}


def _bytes():
    slots = 20 * 64
    vis, pairs = 1000, 3000
    return {
        "select": 8 * 20,
        "project": 236 * slots + (48 + 8 + 4) * vis + 4 * (slots - vis),
        "depth_sort": slots * (4 * 16 + 4),
        "bin": vis * 12 + pairs * 8,
        "tile_sort": pairs * (2 * 16 + 4),
        "ranges": pairs * 4 + 8 * 8160,
    }


def test_hbm_stage_fields():
    r = bench.roofline_for("project", STAGE_MS, FS, PEAKS, "measured")
    want_gbs = _bytes()["project"] / 1e-3 / 1e9
    assert r["kernel"] == "k_project" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(want_gbs, rel=1e-12)
    assert r["frac"] == pytest.approx(want_gbs / 1000.0, rel=1e-12)
    assert r["peak"] == 1000.0 and r["peak_source"] == "measured"
    # traffic: the ncu bytes per slot of the committed capture times the frame's slots
    per, unit, src = bench.NCU_DRAM_PER_UNIT["project"]
    assert unit == "slot" and src.startswith("profiles/")
    assert r["traffic"] == pytest.approx(per * 20 * 64)


def test_select_is_labelled_by_its_own_bound():
    r = bench.roofline_for("project", STAGE_MS, FS, PEAKS, "measured")
    assert r["per_stage"]["select"]["bound"] == "latency" and "profiles/" in r["per_stage"]["select"]["note"]
    assert all(r["per_stage"][k]["bound"] == "hbm" for k in ("project", "depth_sort", "bin", "tile_sort", "ranges"))


def test_project_bytes_grouped_by_cluster():
    """With the render list projected grouped by cluster (render_clusters counted), the projection
    reads each distinct cluster's 64 x 236 B once plus 44 B per entry (entry, FP64 reference,
    order); the writes are unchanged."""
    fs = dict(FS, render_clusters=5.0)
    r = bench.roofline_for("project", STAGE_MS, fs, PEAKS, "measured")
    slots, vis = 20 * 64, 1000
    want = 236 * 64 * 5 + 44 * 20 + (48 + 8 + 4) * vis + 4 * (slots - vis)
    assert r["achieved"] == pytest.approx(want / 1e-3 / 1e9, rel=1e-12)
    # the other stages do not depend on the grouping
    r0 = bench.roofline_for("project", STAGE_MS, FS, PEAKS, "measured")
    for k in ("depth_sort", "bin", "tile_sort", "ranges", "blend"):
        assert r["per_stage"][k] == r0["per_stage"][k], k


def test_every_stage_and_the_frame():
    r = bench.roofline_for("project", STAGE_MS, FS, PEAKS, "measured")
    ps = r["per_stage"]
    for k, b in _bytes().items():
        gbs = b / (STAGE_MS[k] / 1000.0) / 1e9
        assert ps[k]["gbs"] == pytest.approx(gbs, rel=1e-12), k
        assert ps[k]["frac"] == pytest.approx(gbs / 1000.0, rel=1e-12), k
    alu_peak = 152 * 128 * 2000e6 / 1e12
    tflops = (8 * 5.0e6 + 10 * 2.0e6) / 2e-3 / 1e12
    assert ps["blend"]["tflops"] == pytest.approx(tflops, rel=1e-12)
    assert ps["blend"]["frac"] == pytest.approx(tflops / alu_peak, rel=1e-12)
    # the frame: each stage at its own bound, summed, against the sum of the measured stages
    ideal = sum(b / (1000.0 * 1e9) * 1e3 for b in _bytes().values()) + (8 * 5.0e6 + 10 * 2.0e6) / (alu_peak * 1e12) * 1e3
    assert r["frame"]["ideal_ms"] == pytest.approx(ideal, rel=1e-12)
    assert r["frame"]["measured_ms"] == pytest.approx(sum(STAGE_MS.values()), rel=1e-12)
    assert r["frame"]["frac"] == pytest.approx(ideal / sum(STAGE_MS.values()), rel=1e-12)


def test_blend_as_dominant_stage():
    r = bench.roofline_for("blend", STAGE_MS, FS, PEAKS, "measured")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["kernel"] == "k_blend"
    assert r["peak"] == pytest.approx(152 * 128 * 2000e6 / 1e12)
    assert r["work"]["evals"] == 5.0e6 and r["work"]["ops_per_eval"] == 8
    per, unit, _ = bench.NCU_DRAM_PER_UNIT["blend"]
    assert unit == "pair" and r["traffic"] == pytest.approx(per * 3000)


def test_stage_without_capture_has_no_traffic():
    r = bench.roofline_for("tile_sort", STAGE_MS, FS, PEAKS, "measured")
    assert r["kernel"] == "k_onesweep" and r["traffic"] is None and r["traffic_source"] is None


def test_clock_record_summary():
    c = bench.ClockSampler(0)
    c.lines = [
        "1965, 2070, 900.1, Not Active, Not Active, Not Active, Not Active",
        "2070, 2070, 1100.5, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 1200.0, Not Active, Not Active, Not Active, Not Active",
        "[N/A], 2070, 0, Not Active, Not Active, Not Active, Not Active",   # unreadable sample: skipped
        "garbage",
    ]
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    c.lines = ["1500, 2070, 800, Active, Not Active, Active, Not Active"]
    s = c.summary()
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and math.isclose(s["sm_mhz"], 1500.0)
    assert bench.ClockSampler(0).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_request_mix_draws_the_configured_classes():
    """Config 5's request mix: every draw is one of 100 / 1000 / 5000 instances, 720p / 1080p / 4K,
    tau 0.5 / 1 / 2 / 4 and a walk frame; the draws are seeded, and 2,000 of them reach every
    combination of scene size and resolution."""
    a = bench.mix_requests(2000, seed=7)
    assert a == bench.mix_requests(2000, seed=7) and a != bench.mix_requests(2000, seed=8)
    sizes, res, taus, frames = zip(*a)
    assert set(sizes) == {100, 1000, 5000}
    assert set(res) == {(1280, 720), (1920, 1080), (3840, 2160)}
    assert set(taus) == {0.5, 1.0, 2.0, 4.0}
    assert min(frames) >= 0 and max(frames) < 300
    assert len({(n, r) for n, r, _, _ in a}) == 9


def test_request_mix_scenes():
    """The mix's scenes: the first 100 crowd instances, the crowd, and the crowd extended to 5000."""
    from synth import scenes
    crowd = scenes.crowd_instances(1000, n_assets=3)
    sc = bench.mix_scenes(crowd, 3)
    assert {k: v.n for k, v in sc.items()} == {100: 100, 1000: 1000, 5000: 5000}
    assert (sc[100].trans == crowd.trans[:100]).all() and (sc[5000].trans[:1000] == crowd.trans).all()
    assert sc[5000].asset.max() < 3
