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
    rf = bench.roofline_of(stages, loop, None)
    assert rf["kernel"] == "raster_bwd" and rf["bound"] == "alu" and rf["unit"] == "TFLOP/s"
    # 40 FLOP per evaluated pair over 1 ms
    assert rf["achieved"] == pytest.approx(40.0 * 50000.0 / 1e-3 / 1e12)
    assert rf["frac"] == pytest.approx(rf["achieved"] / rf["peak"])
    stages["raster_bwd"]["share"] = 0.0
    stages["project_bwd_adam"].update(ms=2.0, share=0.25)
    rf = bench.roofline_of(stages, loop, None)
    assert rf["kernel"] == "project_bwd_adam" and rf["bound"] == "hbm" and rf["unit"] == "GB/s"
    want = (1000 * 48 + 24 * 59 * 1000) / 2e-3 / 1e9  # 2D gradients + (p, m, v) read and written
    assert rf["achieved"] == pytest.approx(want)


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
