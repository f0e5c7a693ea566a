"""Launch-shape search for the compositing kernels.

The tile side (8, 16, 32), the staging batch (64, 128, 256) and the pixels
per thread of the forward and adjoint kernels change how the work maps to
the GPU but not what it computes: the contribution set is tile-size
invariant (conservative support rectangles) and every configuration gives
the same images and gradients up to the order of float atomics.  So the
choice is made on speed alone: each candidate runs a few forward + loss +
adjoint iterations on the caller's workload and the fastest wins.  Results
are cached per workload signature (Gaussian count, SH degree, view sizes,
views per step, candidate set), in memory and optionally in a JSON file.
"""
from __future__ import annotations

import copy
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


def _time_candidate(model: GaussianModel, cams: list, flat_targets, offsets, settings: RasterSettings,
                    views_per_step: int, reps: int, pair_capacity) -> float:
    wmax, hmax = max(c.width for c in cams), max(c.height for c in cams)
    slot_cam = copy.copy(cams[0])
    slot_cam.width, slot_cam.height = wmax, hmax
    slots = Views([slot_cam] * views_per_step, settings.tile)
    poses = Views(cams, settings.tile)
    r = Renderer(model.n, model.sh_degree, slots, settings, pair_capacity)
    r.sizes_on_device = True
    dev = model.flat.device
    seq = torch.arange(len(cams), dtype=torch.int32, device=dev)
    it = torch.zeros(1, dtype=torch.int64, device=dev)
    vid = torch.zeros(views_per_step, dtype=torch.int32, device=dev)
    grad = torch.zeros_like(model.flat)
    params, grads = model.c_params(), model.c_grads(grad)

    def once():
        gsr.call("gs_select_views", gsr.ptr(seq), len(cams), gsr.ptr(it), views_per_step, gsr.ptr(vid),
                 gsr.ptr(poses.dev), gsr.ptr(slots.dev), None)
        r.forward(params)
        r.compute_loss(flat_targets, offsets, vid, with_grad=True)
        r.backward(params, grads, accumulate=False)

    once()
    torch.cuda.synchronize()
    if int(r.status.item()) != 0:
        return float("inf")  # e.g. over the pair capacity: not a usable configuration
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        once()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


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
    sizes = [int(t.numel()) for t in targets]
    flat = torch.cat([t.contiguous().view(-1) for t in targets])
    offs = torch.tensor([sum(sizes[:i]) for i in range(len(sizes))], dtype=torch.int64, device=flat.device)
    times = {}
    for cand in candidates:
        try:
            times[tuple(cand)] = _time_candidate(model, cams, flat, offs, settings_of(base, cand), views_per_step,
                                                 reps, pair_capacity)
        except gsr.GsError:  # a shape this workload cannot use (e.g. too many tiles per view)
            times[tuple(cand)] = float("inf")
        torch.cuda.empty_cache()
    if all(t == float("inf") for t in times.values()):
        raise RuntimeError("autotune: no candidate launch shape runs this workload")
    best = min(times, key=times.get)
    _cache[key] = list(best)
    save_cache(cache_path)
    return settings_of(base, best), times
