"""Adam (Kingma & Ba, bias-corrected) in FP64: the optimizer step that runs
only when the gate lets the backward pass run (Algorithm 1).

Test infrastructure only.  Readings (the paper says "standard 3DGS optimizer"):
beta1 = 0.9, beta2 = 0.999, eps = 1e-15, constant per-group learning rates,
dense update of every parameter, the step counter counts executed steps.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

GROUPS = ("means", "log_scales", "quats", "opacity_logit", "sh_dc", "sh_rest")


@dataclass
class AdamConfig:
    lr_means: float = 1.6e-5
    lr_log_scales: float = 5e-3
    lr_quats: float = 1e-3
    lr_opacity: float = 2.5e-2
    lr_sh_dc: float = 2.5e-3
    lr_sh_rest: float = 1.25e-4
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15

    def lrs(self):
        return (self.lr_means, self.lr_log_scales, self.lr_quats, self.lr_opacity, self.lr_sh_dc,
                self.lr_sh_rest)


def param_groups(n: int, K: int):
    """[start, end) offsets of the six groups in the flat parameter vector
    means | log_scales | quats | opacity_logit | sh (sh = [N,K,3]; DC first)."""
    o_means, o_scales, o_quats, o_opac, o_sh = 0, 3 * n, 6 * n, 10 * n, 11 * n
    # DC and higher bands are interleaved per Gaussian ([N,K,3]); expressed as masks.
    return dict(means=(o_means, o_scales), log_scales=(o_scales, o_quats), quats=(o_quats, o_opac),
                opacity_logit=(o_opac, o_sh), sh=(o_sh, o_sh + 3 * K * n))


def lr_vector(n: int, K: int, cfg: AdamConfig) -> np.ndarray:
    g = param_groups(n, K)
    lr = np.empty(g["sh"][1])
    lr[g["means"][0]:g["means"][1]] = cfg.lr_means
    lr[g["log_scales"][0]:g["log_scales"][1]] = cfg.lr_log_scales
    lr[g["quats"][0]:g["quats"][1]] = cfg.lr_quats
    lr[g["opacity_logit"][0]:g["opacity_logit"][1]] = cfg.lr_opacity
    sh = lr[g["sh"][0]:g["sh"][1]].reshape(n, K, 3)
    sh[:, 0, :] = cfg.lr_sh_dc
    sh[:, 1:, :] = cfg.lr_sh_rest
    return lr


def adam_step(p: np.ndarray, g: np.ndarray, m: np.ndarray, v: np.ndarray, step: int, lr: np.ndarray,
              cfg: AdamConfig):
    """One executed step (step = number of steps already executed).  Returns
    (p, m, v, step + 1) as new FP64 arrays."""
    p = np.asarray(p, np.float64)
    g = np.asarray(g, np.float64)
    t = step + 1
    m = cfg.beta1 * np.asarray(m, np.float64) + (1.0 - cfg.beta1) * g
    v = cfg.beta2 * np.asarray(v, np.float64) + (1.0 - cfg.beta2) * g * g
    mhat = m / (1.0 - cfg.beta1 ** t)
    vhat = v / (1.0 - cfg.beta2 ** t)
    p = p - lr * mhat / (np.sqrt(vhat) + cfg.eps)
    return p, m, v, t
