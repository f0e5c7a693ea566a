"""Adaptive density control (the densification phase before T_d, and the
opacity-threshold prune) in plain numpy.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the bench's CPU
arms may use it; the product path never does.

The paper's Sec. 3 (Preliminaries) states the scheme qualitatively: during
iterations 0..T_d the Gaussians with a high view-space positional gradient
are cloned when small and split when large, and near-transparent ones
(alpha_i < eps_alpha) are pruned; after T_d the set is fixed.  Everything
else is a reading, the vanilla 3DGS convention where there is one:

  D1 statistic: after each backward pass, for each view v it covered and each
     Gaussian i visible in v (tile count > 0), accum_i += || dL/dmean2D_i,v ||_2
     (pixel units) and denom_i += 1.
  D2 decision (float32, so both sides decide alike): avg_i = accum_i / denom_i
     (0 when denom_i = 0); prune when the opacity logit < logit(eps_alpha)
     (the opacity test sigma(logit) < eps_alpha, thresholds given in logit
     units); else, when avg_i >= tau_grad: split when max_k log s_ik >
     log_size_thr (scales given in log units), clone otherwise; else keep.
     Prune wins over clone and split (vanilla densifies, then prunes the
     copies too, which share the opacity: the same outcome).
  D3 outputs, in input order with each Gaussian's outputs consecutive: keep
     -> the Gaussian (its Adam moments kept); clone -> the Gaussian (moments
     kept) then an identical copy (moments zero); split -> two children
     (moments zero); prune -> nothing.
  D4 split child k in {0, 1}: mean = mu + R(q / |q|) (s * z_k), s =
     exp(log s), z_k ~ N(0, I3) drawn by the caller and passed in; log-scales
     reduced by log(1.6) (scales / (0.8 * 2)); rotation, opacity and SH copied.
  D5 every output's statistics start at zero; the Adam step count carries on.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

KEEP, CLONE, SPLIT, PRUNE = 0, 1, 2, 3
OUTPUTS = np.array([1, 2, 2, 0], np.int64)  # outputs per action (D3)
GROUPS = ("means", "log_scales", "quats", "opacity_logit", "sh")


@dataclass
class DensifyConfig:
    """Thresholds in the units the decision compares (D2).  Defaults: the
    vanilla opacity threshold 0.005; tau_grad and the size threshold are set
    per scene by the caller."""
    grad_thr: float = 2e-7
    log_size_thr: float = float(np.log(0.01))
    logit_prune_thr: float = float(np.log(0.005 / 0.995))
    log_split_shrink: float = float(np.log(1.6))


def accumulate(accum: np.ndarray, denom: np.ndarray, g_mean2d: np.ndarray, visible: np.ndarray):
    """D1 for one view: g_mean2d [N,2] (dL/dmean2D), visible [N] bool.
    Returns new (accum, denom) in float64 / int64."""
    g = np.asarray(g_mean2d, np.float64)
    norm = np.sqrt(g[:, 0] * g[:, 0] + g[:, 1] * g[:, 1])
    vis = np.asarray(visible, bool)
    accum = np.asarray(accum, np.float64) + np.where(vis, norm, 0.0)
    denom = np.asarray(denom, np.int64) + vis.astype(np.int64)
    return accum, denom


def decide(accum, denom, log_scales, opacity_logit, cfg: DensifyConfig) -> np.ndarray:
    """D2 in float32: one action per Gaussian."""
    f32 = np.float32
    a = np.asarray(accum, f32)
    d = np.asarray(denom, np.int64)
    avg = np.zeros(a.shape, f32)
    seen = d > 0
    avg[seen] = a[seen] / d[seen].astype(f32)  # one correctly rounded float32 division
    ls = np.asarray(log_scales, f32)
    big = np.max(ls, axis=1) > f32(cfg.log_size_thr)
    high = avg >= f32(cfg.grad_thr)
    prune = np.asarray(opacity_logit, f32) < f32(cfg.logit_prune_thr)
    act = np.full(a.shape, KEEP, np.uint8)
    act[high & ~big] = CLONE
    act[high & big] = SPLIT
    act[prune] = PRUNE
    return act


def quat_rotation(q: np.ndarray) -> np.ndarray:
    """Rotation matrices [N,3,3] of quaternions (w, x, y, z), normalised."""
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = np.empty((q.shape[0], 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - w * z)
    R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y)
    R[:, 2, 1] = 2 * (y * z + w * x)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def apply(params: dict, m: dict, v: dict, action: np.ndarray, noise: np.ndarray, cfg: DensifyConfig):
    """D3-D5: the densified parameter and moment groups (float64).
    params / m / v: dicts of the groups (means [N,3], log_scales [N,3], quats
    [N,4], opacity_logit [N], sh [N,K,3]); noise [N,2,3] (D4's z, used for
    split Gaussians only).  Returns (params, m, v) of the output set."""
    act = np.asarray(action)
    n = act.shape[0]
    counts = OUTPUTS[act]
    src = np.repeat(np.arange(n), counts)           # source Gaussian of every output
    k = np.arange(src.shape[0]) - np.repeat(np.cumsum(counts) - counts, counts)  # 0 or 1 within a source
    a_out = act[src]
    out = {g: np.asarray(params[g], np.float64)[src].copy() for g in GROUPS}
    keep_moments = (a_out == KEEP) | ((a_out == CLONE) & (k == 0))
    mo = {g: np.where(_bcast(keep_moments, m[g]), np.asarray(m[g], np.float64)[src], 0.0) for g in GROUPS}
    vo = {g: np.where(_bcast(keep_moments, v[g]), np.asarray(v[g], np.float64)[src], 0.0) for g in GROUPS}
    sp = a_out == SPLIT
    if sp.any():
        i = src[sp]
        R = quat_rotation(np.asarray(params["quats"], np.float64)[i])
        s = np.exp(np.asarray(params["log_scales"], np.float64)[i])
        z = np.asarray(noise, np.float64)[i, k[sp]]
        out["means"][sp] = np.asarray(params["means"], np.float64)[i] + np.einsum("nij,nj->ni", R, s * z)
        out["log_scales"][sp] = np.asarray(params["log_scales"], np.float64)[i] - cfg.log_split_shrink
    return out, mo, vo


def _bcast(mask: np.ndarray, like) -> np.ndarray:
    like = np.asarray(like)
    return mask.reshape((-1,) + (1,) * (like.ndim - 1))


def output_count(action: np.ndarray) -> int:
    return int(OUTPUTS[np.asarray(action)].sum())
