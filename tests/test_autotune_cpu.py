"""Autotuner host logic (no GPU): workload signatures and the cache."""
import json

from paper_2603_08997_gb300 import autotune
from paper_2603_08997_gb300.raster import RasterSettings


def test_signature_depends_on_workload_only():
    c = autotune.DEFAULT_CANDIDATES
    a = autotune.signature(1000, 3, [(64, 64), (32, 16)], 2, c)
    assert a == autotune.signature(1000, 3, [(32, 16), (64, 64)], 2, c)  # view order does not matter
    assert a != autotune.signature(1001, 3, [(64, 64), (32, 16)], 2, c)
    assert a != autotune.signature(1000, 3, [(64, 64), (32, 16)], 1, c)
    assert a != autotune.signature(1000, 3, [(64, 64), (32, 16)], 2, c[:3])


def test_candidates_cover_the_launch_shapes():
    tiles = {t for t, _, _, _ in autotune.DEFAULT_CANDIDATES}
    batches = {b for _, b, _, _ in autotune.DEFAULT_CANDIDATES}
    assert tiles == {8, 16, 32} and batches == {64, 128, 256}
    s = autotune.settings_of(RasterSettings(lambda_ssim=0.3), (8, 64, 2, 1))
    assert (s.tile, s.batch, s.pixels_per_thread_fwd, s.pixels_per_thread, s.lambda_ssim) == (8, 64, 2, 1, 0.3)


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "tune.json")
    autotune._cache.clear()
    autotune._cache["k"] = [16, 256, 1, 2]
    autotune.save_cache(p)
    autotune._cache.clear()
    autotune.load_cache(p)
    assert autotune._cache["k"] == [16, 256, 1, 2]
    assert json.load(open(p)) == {"k": [16, 256, 1, 2]}
    autotune._cache.clear()
