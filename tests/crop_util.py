"""Oracle evaluation of one view restricted to a pixel window (test
infrastructure).

The oracle projects the scene with the full camera (culling, frustum clamp
of the Jacobian and colour direction exactly as for the whole view), keeps
the Gaussians whose inflated support box reaches the window, and bins,
composites and back-propagates on the window alone, with the means shifted
by the window's origin (an exact shift: integers in float64).  The window's
pixels, and the gradients of any loss supported on the window, equal those
of the whole view, because only Gaussians whose support reaches a pixel can
contribute to it and the kept ones are ordered as in the whole view."""
from __future__ import annotations

import numpy as np

import oracle
import synth


class WindowCam:
    def __init__(self, w: int, h: int):
        self.width, self.height = int(w), int(h)


def widen(scene) -> "synth.Scene":
    """float64 copy (the oracle then reads it without converting per call)."""
    return synth.Scene(*(np.asarray(getattr(scene, k), np.float64) for k in
                         ("means", "log_scales", "quats", "opacity_logit", "sh")))


def subset(scene, idx) -> "synth.Scene":
    return synth.Scene(*(getattr(scene, k)[idx] for k in ("means", "log_scales", "quats", "opacity_logit", "sh")))


def select(proj: dict, x0: int, y0: int, w: int, h: int, margin_px: float = 2.0) -> np.ndarray:
    """Indices (ascending) of the Gaussians whose support box reaches the
    window's pixel centres, widened by margin_px."""
    m, r = proj["mean2d"], proj["radius"]
    lo_x, hi_x = x0 + 0.5 - margin_px, x0 + w - 0.5 + margin_px
    lo_y, hi_y = y0 + 0.5 - margin_px, y0 + h - 0.5 + margin_px
    keep = ((proj["touched"] > 0) & (m[:, 0] + r[:, 0] >= lo_x) & (m[:, 0] - r[:, 0] <= hi_x)
            & (m[:, 1] + r[:, 1] >= lo_y) & (m[:, 1] - r[:, 1] <= hi_y))
    return np.nonzero(keep)[0]


def window_proj(proj: dict, idx, x0: int, y0: int, w: int, h: int, tile: int) -> dict:
    """The kept Gaussians' records in window coordinates, with rectangles and
    tile counts for the window's tile grid."""
    out = {k: proj[k][idx] for k in ("mean2d", "conic", "rgb", "opacity", "depth_bits", "radius", "flags")}
    out["mean2d"] = out["mean2d"] - np.array([x0, y0], np.float64)
    m, r = out["mean2d"], out["radius"]
    xa = np.maximum(np.ceil(m[:, 0] - r[:, 0] - 0.5), 0)
    xb = np.minimum(np.floor(m[:, 0] + r[:, 0] - 0.5), w - 1)
    ya = np.maximum(np.ceil(m[:, 1] - r[:, 1] - 0.5), 0)
    yb = np.minimum(np.floor(m[:, 1] + r[:, 1] - 0.5), h - 1)
    ok = (xa <= xb) & (ya <= yb)
    rect = np.zeros((len(idx), 4), np.int32)
    rect[:, 0] = np.where(ok, xa // tile, 0)
    rect[:, 1] = np.where(ok, ya // tile, 0)
    rect[:, 2] = np.where(ok, xb // tile, -1)
    rect[:, 3] = np.where(ok, yb // tile, -1)
    out["rect"] = rect
    out["touched"] = np.where(ok, (rect[:, 2] - rect[:, 0] + 1) * (rect[:, 3] - rect[:, 1] + 1), 0).astype(np.int32)
    return out


def window_pass(scene64, cam, rc, x0: int, y0: int, w: int, h: int, weights=None, idx=None,
                margin_rel: float = 1e-4) -> dict:
    """Window image (and, with weights [3, h, w], the gradients of
    L = <weights, window image> for the kept Gaussians).  idx: the kept
    Gaussians when already known (the scene may then be just those)."""
    proj = oracle.project(scene64, cam, rc)
    if idx is None:  # whole scene given: keep the Gaussians reaching the window
        idx = select(proj, x0, y0, w, h)
        sub_scene = subset(scene64, idx)
        rows = idx
    else:  # the scene is already the kept Gaussians (idx indexes it)
        sub_scene = scene64
        rows = np.asarray(idx)
    wp = window_proj(proj, rows, x0, y0, w, h, rc.tile)
    wc = WindowCam(w, h)
    _, vals, ranges, _ = oracle.bin_sort([wp], [wc], rc.tile)
    f = oracle.render(wp, wc, vals, ranges, rc, 0, margin_rel)
    out = dict(image=f["image"], margin=f["margin"], idx=idx, hash=f["hash"], flags=wp["flags"])
    if weights is not None:
        g2d = oracle.raster_bwd(wp, wc, vals, ranges, rc, np.asarray(weights, np.float64))
        out["grads"] = oracle.project_bwd(sub_scene, cam, rc, g2d)
    return out
