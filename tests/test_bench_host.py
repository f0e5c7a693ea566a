"""Host-side accounting of bench.py (no GPU): stage weights in a gated
iteration, the roofline of the dominant stage, and the guard that reports
stored DRAM traffic only for the CUDA sources it was captured from."""
import types

import pytest
import torch

import bench


def test_stage_weights_and_shares():
    out = {k: {"ms": ms} for k, ms in (("project", 0.15), ("bin_sort", 0.70), ("render_fwd", 0.33),
                                        ("loss", 0.07), ("loss_bwd", 0.05), ("raster_bwd", 0.75),
                                        ("project_bwd", 0.32), ("adam", 0.75), ("project_bwd_adam", 0.73))}
    w = bench.weigh_stages(out, b_frac=0.66)
    assert w["bin_sort"]["weight"] == 1.0 and w["loss"]["weight"] == 1.0
    assert w["raster_bwd"]["weight"] == 0.66 and w["project_bwd_adam"]["weight"] == 0.66
    assert w["project_bwd"]["weight"] == 0.0 and w["adam"]["weight"] == 0.0  # the loop runs the fused stage
    assert sum(v["share"] for v in w.values()) == pytest.approx(1.0)
    tot = 0.15 + 0.70 + 0.33 + 0.07 + 0.66 * (0.05 + 0.75 + 0.73)
    assert w["bin_sort"]["share"] == pytest.approx(0.70 / tot)


def _fake_loop(n=1000, pairs=12000, evals=50000.0, pixels=640 * 480, tiles=1200, n_params=59 * 1000):
    views = types.SimpleNamespace(n=1, total_pixels=pixels, total_tiles=tiles)
    r = types.SimpleNamespace(n=n, views=views, pair_count=torch.tensor([pairs]),
                              n_last=torch.full((int(evals) // 100,), 100, dtype=torch.int32))
    return types.SimpleNamespace(renderer=r, model=types.SimpleNamespace(flat=torch.zeros(n_params)))


def test_roofline_names_the_largest_share_and_divides_algorithmic_work_by_time():
    loop = _fake_loop()
    stages = {k: {"ms": 1.0, "share": s} for k, s in (("project", 0.1), ("bin_sort", 0.2), ("render_fwd", 0.1),
                                                      ("loss", 0.05), ("loss_bwd", 0.05),
                                                      ("raster_bwd", 0.3), ("project_bwd", 0.0), ("adam", 0.0),
                                                      ("project_bwd_adam", 0.2))}
    census = dict(sum_n_last=50000, evaluated=30000, contributing=20000, tile_pairs=4000, staged=6000)
    rf = bench.roofline_of(stages, loop, None, census, atomic_peak=8e9)
    assert rf["kernel"] == "raster_bwd" and rf["bound"] == "alu" and rf["unit"] == "TFLOP/s"
    # 13 FLOP per evaluated pair + 61 per contributing pair, over 1 ms
    assert rf["achieved"] == pytest.approx((13 * 30000 + 61 * 20000) / 1e-3 / 1e12)
    assert rf["frac"] == pytest.approx(rf["achieved"] / rf["peak"])
    fwd = rf["all_stages"]["render_fwd"]
    assert fwd["achieved"] == pytest.approx((13 * 30000 + 10 * 20000) / 1e-3 / 1e12)
    at = rf["all_stages"]["raster_bwd"]["atomic"]
    assert at["updates_per_s"] == pytest.approx(4000 / 1e-3)
    assert at["frac"] == pytest.approx(4000 / 1e-3 / 8e9)
    assert rf["all_stages"]["raster_bwd"]["pair_bytes_per_launch"] == pytest.approx(40 * 6000 + 36 * 4000)
    stages["raster_bwd"]["share"] = 0.0
    stages["project_bwd_adam"].update(ms=2.0, share=0.25)
    rf = bench.roofline_of(stages, loop, None, census)
    assert rf["kernel"] == "project_bwd_adam" and rf["bound"] == "hbm" and rf["unit"] == "GB/s"
    want = (1000 * 48 + 24 * 59 * 1000) / 2e-3 / 1e9  # 2D gradients + (p, m, v) read and written
    assert rf["achieved"] == pytest.approx(want)


def test_alu_peak_follows_the_device():
    assert bench.peak_alu_tflops(152, 2070.0) == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
    assert bench.peak_alu_tflops(76, 2070.0) == pytest.approx(bench.peak_alu_tflops(152, 2070.0) / 2)


def test_plan_times_the_last_steps_of_the_whole_loop():
    p = bench.plan_loop(5000, 20)
    assert p["start"] == 4980 and p["K"] == 20 and p["marks"][-1] == 5000
    assert p["evals"] == [4250, 4500, 4750, 5000]
    assert 4980 in p["marks"] and all(m > 0 for m in p["marks"]) and p["marks"] == sorted(set(p["marks"]))
    # a window longer than one checkpoint segment is split at the checkpoints inside it
    p = bench.plan_loop(5000, 1000)
    assert p["start"] == 4000 and p["marks"] == [4000, 4250, 4500, 4750, 5000]
    # the whole loop timed
    p = bench.plan_loop(100, 500)
    assert p["start"] == 0 and p["K"] == 100 and p["marks"] == [25, 50, 75, 100]


def test_backward_split_needs_skipped_backward_passes():
    # every iteration ran the backward pass: the split is undetermined, not noise / 1
    assert bench.backward_split(1000.0, 1002.0, 20, 20) == (None, None)
    assert bench.backward_split(1000.0, 990.0, 100, 95) == (None, None)  # 5% skipped < 10%
    f, b = bench.backward_split(5000 * 2.7, 5000 * 1.24 + 3300 * 1.46, 5000, 3300)
    assert b == pytest.approx(1.46) and f == pytest.approx(1.24)


def test_stored_traffic_only_for_matching_sources(monkeypatch):
    import json
    import os
    stored = json.load(open(os.path.join(bench.ROOT, "profiles", "stage_traffic_3M.json")))
    monkeypatch.setattr(bench, "sources_sha256", lambda: stored["sources_sha256"])
    got, note = bench.stage_traffic("bin_sort")
    assert got == float(stored["per_launch_bytes"]["bin_sort"]) and got > 0, note
    monkeypatch.setattr(bench, "sources_sha256", lambda: "0" * 64)
    got, note = bench.stage_traffic("bin_sort")
    assert got is None and "changed" in note


def test_coarse_pairs_count_super_tiles_of_each_rectangle():
    """(entry, 4x4-tile super-tile) pairs from packed tile rectangles
    (x0, y0, width, height): a rectangle inside one super-tile counts 1, one
    straddling a super-tile edge in x and y counts 4; empty ones count 0."""
    rect16 = torch.tensor([[0, 0, 4, 4], [3, 3, 2, 2], [5, 1, 8, 1], [0, 0, 0, 0], [7, 7, 1, 1]],
                          dtype=torch.int16)
    r = types.SimpleNamespace(aux_valid=True, rect16=rect16.view(-1))
    # [0,3]x[0,3]: 1; [3,4]x[3,4]: 4; x [5,12] -> super-tiles 1..3, y 1 -> 0: 3; empty: 0; (7,7): 1
    assert bench.coarse_pairs(r, 999) == 1 + 4 + 3 + 0 + 1
    assert bench.coarse_pairs(types.SimpleNamespace(aux_valid=False), 999) == 999
