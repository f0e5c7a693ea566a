"""Shared helpers of the GPU parity tests: convert seeded inputs to the
library's layouts and to the oracle's, and compare results."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2603_08997_gb300 import build, gsr, raster

_built = False


def lib():
    global _built
    if not _built:
        build.build()
        oracle.core.build()
        _built = True
    return gsr.lib()


def records(rec: dict, cams: list, tile: int):
    """Synthetic screen-space records (synth.projected_records, one list per
    view) -> (device rec/rect/touched tensors, per-view oracle dicts).

    Both sides get the same quadratic form: the conic factor U (upper Cholesky
    of Q = Sigma2D^-1) is rounded to float32 once and the oracle uses
    Q = U^T U evaluated exactly in float64."""
    V = len(cams)
    n = rec[0]["mean2d"].shape[0]
    R = np.zeros((V, n, 12), np.float32)
    rect = np.zeros((V, n, 4), np.int32)
    touched = np.zeros((V, n), np.int32)
    orc = []
    for v, (r, cam) in enumerate(zip(rec, cams)):
        c, s = np.cos(r["theta"].astype(np.float64)), np.sin(r["theta"].astype(np.float64))
        s1, s2 = r["sigma1"].astype(np.float64), r["sigma2"].astype(np.float64)
        # Sigma2D = Rot diag(s1^2, s2^2) Rot^T ; Q = inverse
        a = c * c * s1 ** 2 + s * s * s2 ** 2
        b = c * s * (s1 ** 2 - s2 ** 2)
        d = s * s * s1 ** 2 + c * c * s2 ** 2
        det = a * d - b * b
        Qa, Qb, Qc = d / det, -b / det, a / det
        u00 = np.sqrt(Qa)
        u01 = Qb / u00
        u11 = np.sqrt(np.maximum(Qc - u01 * u01, 1e-30))
        U = np.stack([u00, u01, u11], 1).astype(np.float32)
        Uf = U.astype(np.float64)
        conic = np.stack([Uf[:, 0] ** 2, Uf[:, 0] * Uf[:, 1], Uf[:, 1] ** 2 + Uf[:, 2] ** 2], 1)
        R[v, :, 0:2] = r["mean2d"]
        R[v, :, 2:4] = U[:, 0:2]
        R[v, :, 4] = U[:, 2]
        R[v, :, 5] = r["opacity"]
        R[v, :, 6:9] = r["rgb"]
        R[v, :, 9] = r["depth"]
        # support bound: alpha' >= 1/255 needs dp^T Q dp <= 2 ln 255 < 3.5^2, and
        # the x (y) extent of that ellipse is at most 3.5 sigma1
        R[v, :, 10] = 3.5 * r["sigma1"]
        R[v, :, 11] = 3.5 * r["sigma1"]
        box = r["box"].astype(np.float64)
        x0 = np.maximum(np.ceil(box[:, 0] - 0.5), 0)
        x1 = np.minimum(np.floor(box[:, 1] - 0.5), cam.width - 1)
        y0 = np.maximum(np.ceil(box[:, 2] - 0.5), 0)
        y1 = np.minimum(np.floor(box[:, 3] - 0.5), cam.height - 1)
        ok = (x0 <= x1) & (y0 <= y1) & ~r["culled"]
        rect[v, :, 0] = np.where(ok, x0 // tile, 0)
        rect[v, :, 1] = np.where(ok, y0 // tile, 0)
        rect[v, :, 2] = np.where(ok, x1 // tile, -1)
        rect[v, :, 3] = np.where(ok, y1 // tile, -1)
        touched[v] = np.where(ok, (rect[v, :, 2] - rect[v, :, 0] + 1) * (rect[v, :, 3] - rect[v, :, 1] + 1), 0)
        orc.append(dict(mean2d=r["mean2d"].astype(np.float64), conic=conic,
                        rgb=r["rgb"].astype(np.float64), opacity=r["opacity"].astype(np.float64),
                        depth_bits=r["depth"].view(np.uint32).copy(), rect=rect[v].copy(),
                        touched=touched[v].copy()))
    dev = dict(rec=torch.from_numpy(R.ravel()).cuda(), rect=torch.from_numpy(rect.ravel()).cuda(),
               touched=torch.from_numpy(touched.ravel()).cuda())
    return dev, orc


def set_projected(renderer: raster.Renderer, dev: dict) -> None:
    renderer.rec.copy_(dev["rec"])
    renderer.rect.copy_(dev["rect"])
    renderer.touched.copy_(dev["touched"])
    renderer.aux_valid = False  # bin_sort derives depth keys and rectangles from these records


def rel_err(a, b) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def cosine(a, b) -> float:
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300))


def gpu_grads(model: raster.GaussianModel, flat: torch.Tensor) -> dict:
    v = model.group_views(flat)
    return {k: t.double().cpu().numpy() for k, t in v.items()}


def l1_tie_mask(oracle_image, target, margin=None, tau: float = 1e-4) -> np.ndarray:
    """Values [3,H,W] where the L1 derivative sign(C - C_hat) is not determined
    at the render's float32 precision: |C - C_hat| <= tau in the oracle's own
    image (tau = the end-to-end per-pixel reach of float32 rendering), plus
    every channel of the pixels the oracle flags near a cut-off.  Both sides
    of an end-to-end gradient test zero dL/dimage there, so the comparison
    covers what is unique (the oracle's input never comes from the GPU)."""
    m = np.abs(np.asarray(oracle_image, np.float64) - np.asarray(target, np.float64)) <= tau
    if margin is not None:
        m |= np.asarray(margin, bool)[None]
    return m
