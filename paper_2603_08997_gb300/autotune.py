"""Launch-shape search for the compositing kernels.

The tile side (8, 16, 32), the staging batch (64, 128, 256) and the pixels
per thread of the forward and adjoint kernels change how the work maps to
the GPU but not what it computes: the contribution set is tile-size
invariant (conservative support rectangles) and every configuration gives
the same images and gradients up to the order of float atomics.  So the
choice is made on speed alone, by gs_autotune (the C ABI): each candidate
runs a few forward + loss + adjoint iterations on the caller's workload and
the fastest wins.  This module sizes its workspace and caches the choice per
workload signature (Gaussian count, SH degree, view sizes, views per step,
candidate set), in memory and optionally in a JSON file.
"""
from __future__ import annotations

import dataclasses
import hashlib
import json
import os

import torch

from . import gsr
from .raster import GaussianModel, RasterSettings, Renderer, Views

DEFAULT_CANDIDATES = tuple((t, b, pf, pb) for t in (8, 16, 32) for b in (64, 128, 256)
                           for pf, pb in ((1, 2), (1, 1), (2, 2)))

_cache: dict = {}


def signature(n: int, sh_degree: int, sizes, views_per_step: int, candidates) -> str:
    """Key of a workload: equal keys may share a tuned configuration."""
    blob = json.dumps([int(n), int(sh_degree), sorted([int(w), int(h)] for w, h in sizes), int(views_per_step),
                       [list(c) for c in candidates]])
    return hashlib.sha256(blob.encode()).hexdigest()[:24]


def load_cache(path: str) -> None:
    if path and os.path.exists(path):
        _cache.update(json.load(open(path)))


def save_cache(path: str) -> None:
    if path:
        json.dump(_cache, open(path, "w"), indent=1, sort_keys=True)


def settings_of(base: RasterSettings, cand) -> RasterSettings:
    t, b, pf, pb = cand
    return dataclasses.replace(base, tile=int(t), batch=int(b), pixels_per_thread_fwd=int(pf),
                               pixels_per_thread=int(pb))


def time_candidates(model: GaussianModel, cams: list, targets, base: RasterSettings, candidates, reps: int,
                    pair_capacity: int, stream=None) -> list:
    """gs_autotune over the candidates: ms per iteration of each (inf where the
    workload cannot use the shape), all views of `cams` rendered in one call.
    targets: one [3, H_v, W_v] device tensor per camera."""
    import ctypes as C
    from .raster import camera_struct
    n = len(candidates)
    shapes = (gsr.gs_launch_shape * n)(*[gsr.gs_launch_shape(*map(int, c)) for c in candidates])
    hcams = (gsr.gs_camera * len(cams))(*[camera_struct(c) for c in cams])
    flat = torch.cat([t.contiguous().view(-1) for t in targets]).to(model.flat.device)
    L = gsr.lib()
    cap = int(pair_capacity)
    ws_bytes = int(L.gs_autotune_workspace_size(model.n, model.sh_degree, hcams, len(cams), cap, shapes, n))
    ws = torch.empty(ws_bytes + 256, dtype=torch.uint8, device=model.flat.device)
    ws_ptr = (ws.data_ptr() + 255) // 256 * 256
    ms = (C.c_float * n)()
    best = C.c_int32(-1)
    cfg = base.struct(model.sh_degree)
    code = L.gs_autotune(C.byref(model.c_params()), hcams, len(cams), gsr.ptr(flat), C.byref(cfg),
                         float(base.lambda_ssim), shapes, n, int(reps), cap, C.c_void_p(ws_ptr), ws_bytes, ms,
                         C.byref(best), gsr.stream_handle(stream))
    if code == gsr.GS_ERR_UNSUPPORTED:
        raise RuntimeError("autotune: no candidate launch shape runs this workload")
    gsr.check("gs_autotune", code)
    del ws
    return [float(ms[i]) for i in range(n)]


def choose_list_form(model: GaussianModel, cams: list, targets, base: RasterSettings | None = None, reps: int = 5,
                     pair_capacity: int | None = None):
    """Which list form is faster for this workload: per-tile lists, or
    super-tile lists that the compositing kernels filter (RasterSettings.
    coarse_lists).  The super-tile form skips writing the tile lists and
    reads only the prefix of each list a tile composites, so it wins where
    pixels reach the transmittance floor early (dense scenes); where tiles
    composite their whole lists it pays for the filtering.  Both forms give
    the same images and the same gradients up to float-atomic order, so the
    choice is made on time alone: `reps` iterations of binning, forward,
    loss with its gradient and the raster adjoint over all `cams` in one
    call (projection once, outside the timing), CUDA events on the current
    stream.  targets: one [3, H_v, W_v] device tensor per camera.  Returns
    (settings with the faster form, {"tile": ms, "coarse": ms})."""
    base = base or RasterSettings()
    flat = torch.cat([t.contiguous().view(-1) for t in targets]).to(model.flat.device)
    k = len(cams)
    cap = int(pair_capacity) if pair_capacity else max(1 << 16, 24 * model.n * k)
    times = {}
    for form in ("tile", "coarse"):
        st = dataclasses.replace(base, coarse_lists=form == "coarse")
        r = Renderer(model.n, model.sh_degree, Views(cams, st.tile, model.flat.device), st, pair_capacity=cap)
        p = model.c_params()
        r.project(p)

        def one():
            r.bin_sort()
            r.render_fwd()
            r.compute_loss(flat, with_grad=True)
            r.raster_bwd()

        one()
        torch.cuda.synchronize()
        if int(r.status.item()) != 0:
            times[form] = float("inf")  # e.g. more pairs than the capacity
            continue
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(max(int(reps), 1)):
            one()
        e1.record()
        torch.cuda.synchronize()
        times[form] = e0.elapsed_time(e1) / max(int(reps), 1)
        del r
    torch.cuda.empty_cache()
    if min(times.values()) == float("inf"):
        raise RuntimeError("choose_list_form: neither list form runs this workload (capacity)")
    best = min(times, key=times.get)
    return dataclasses.replace(base, coarse_lists=best == "coarse"), times


def autotune(model: GaussianModel, cams: list, targets, base: RasterSettings | None = None,
             candidates=DEFAULT_CANDIDATES, views_per_step: int = 1, reps: int = 3, pair_capacity=None,
             cache_path: str | None = None):
    """Fastest launch shape for this workload.  targets: one [3, H_v, W_v]
    tensor per camera (device).  Returns (settings, {candidate: ms per
    iteration}); a cached choice returns ({}) timings."""
    base = base or RasterSettings()
    load_cache(cache_path)
    key = signature(model.n, model.sh_degree, [(c.width, c.height) for c in cams], views_per_step, candidates)
    if key in _cache:
        return settings_of(base, tuple(_cache[key])), {}
    # one multi-view call over the first views_per_step views stands for an iteration
    k = max(1, min(int(views_per_step), len(cams)))
    cap = int(pair_capacity) if pair_capacity else max(1 << 16, 24 * model.n * k)
    ms = time_candidates(model, cams[:k], targets[:k], base, candidates, reps, cap)
    times = {tuple(c): t for c, t in zip(candidates, ms)}
    torch.cuda.empty_cache()
    best = min(times, key=times.get)
    _cache[key] = list(best)
    save_cache(cache_path)
    return settings_of(base, best), times
