"""gs_bin_sort_noalloc: the binning/sort entry point for callers that cannot
allocate device memory (work issued during CUDA-graph capture, plugins whose
host owns all device memory, loops that must not block on the allocator).
Its scratch is a fixed array inside the library; its results must equal
gs_bin_sort's (bit-exact, like every sort in this suite) on consecutive calls,
so nothing left in the shared array from one call leaks into the next."""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from paper_2603_08997_gb300 import gsr, raster
from tests import gpu_util

pytestmark = pytest.mark.gpu


def _case(sizes, n, seed, tile=16):
    cams = [synth.camera_pinhole(50, 50, w / 2, h / 2, w, h) for w, h in sizes]
    recs = [synth.projected_records(n, w, h, seed=seed + v) for v, (w, h) in enumerate(sizes)]
    views = raster.Views(cams, tile)
    r = raster.Renderer(n, 0, views, raster.RasterSettings(tile=tile), pair_capacity=1 << 20, keep_keys=True)
    dev, _ = gpu_util.records(recs, cams, tile)
    gpu_util.set_projected(r, dev)
    return r


def _sorted(r):
    torch.cuda.synchronize()
    P = int(r.pair_count.item())
    return (P, r.keys[:P].cpu().numpy().copy(), r.vals[:P].cpu().numpy().copy(), r.ranges.cpu().numpy().copy(),
            int(r.status.item()))


def _noalloc(r):
    L = gsr.lib()
    proj = r.c_proj()
    r.status.zero_()
    code = L.gs_bin_sort_noalloc(C.byref(proj), gsr.ptr(r.views.dev), r.views.n, r.n, r.views.total_tiles,
                                 r.views.max_view_tiles, C.byref(r.cfg), gsr.ptr(r.keys), gsr.ptr(r.vals), r.cap, gsr.ptr(r.ranges),
                                 gsr.ptr(r.pair_count), gsr.ptr(r.status), gsr.stream_handle())
    assert code == gsr.GS_OK, gsr.status_string(code)
    return _sorted(r)


def _reference(r):
    r.status.zero_()
    r.bin_sort()
    return _sorted(r)


def test_noalloc_matches_bin_sort_on_consecutive_calls():
    gpu_util.lib()
    # a large call, then a smaller one: the second must not see the first's leftovers
    cases = [_case([(300, 200), (160, 90)], 20_000, seed=3), _case([(97, 61)], 3_000, seed=9)]
    got = [_noalloc(r) for r in cases]
    want = [_reference(r) for r in cases]
    for g, w in zip(got, want):
        assert g[4] == 0 and w[4] == 0
        assert g[0] == w[0] > 0
        assert np.array_equal(g[1], w[1])
        assert np.array_equal(g[2], w[2])
        assert np.array_equal(g[3], w[3])


def test_noalloc_rejects_sizes_beyond_its_array():
    gpu_util.lib()
    r = _case([(64, 64)], 1_000, seed=1)
    L = gsr.lib()
    proj = r.c_proj()
    r.ranges.fill_(7)
    code = L.gs_bin_sort_noalloc(C.byref(proj), gsr.ptr(r.views.dev), r.views.n, (1 << 18) + 1, r.views.total_tiles,
                                 r.views.max_view_tiles, C.byref(r.cfg), None, gsr.ptr(r.vals), 1024, gsr.ptr(r.ranges),
                                 gsr.ptr(r.pair_count), gsr.ptr(r.status), gsr.stream_handle())
    assert code == gsr.GS_ERR_WORKSPACE
    # a tile count whose count matrix would not fit the array (checked on the
    # host from the sizes alone, before anything reads the cameras)
    assert L.gs_bin_sort_workspace_size(r.n, r.views.n, 1024, 1 << 22) > 16 << 20
    code = L.gs_bin_sort_noalloc(C.byref(proj), gsr.ptr(r.views.dev), r.views.n, r.n, 1 << 22,
                                 r.views.max_view_tiles, C.byref(r.cfg), None, gsr.ptr(r.vals), 1024,
                                 gsr.ptr(r.ranges), gsr.ptr(r.pair_count), gsr.ptr(r.status), gsr.stream_handle())
    assert code == gsr.GS_ERR_WORKSPACE
    torch.cuda.synchronize()
    assert int(r.ranges.min().item()) == 7  # nothing was launched
