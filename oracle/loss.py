"""Eq. (loss): L = (1 - lambda) L1 + lambda (1 - SSIM), lambda = 0.2, in FP64.

Test infrastructure only.  Readings (the paper names only Wang et al.'s SSIM):
11x11 Gaussian window with sigma 1.5 normalised to sum 1, C1 = 0.01^2,
C2 = 0.03^2 (data range 1), zero padding with 'same' output size, SSIM = mean
of the SSIM map over all 3HW values; L1 = mean |C - C_hat| over 3HW; the
derivative of |x| at 0 is taken as 0.
"""
from __future__ import annotations

import numpy as np

C1 = 0.01 ** 2
C2 = 0.03 ** 2
HALF = 5


def gaussian_window(size: int = 11, sigma: float = 1.5) -> np.ndarray:
    r = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-(r * r) / (2.0 * sigma * sigma))
    g /= g.sum()
    return np.outer(g, g)


def _filter(a: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Zero-padded 'same' correlation of each channel of a [C,H,W] array with the
    11x11 window, written as the plain double sum over the window's taps."""
    Cn, H, W = a.shape
    p = np.zeros((Cn, H + 2 * HALF, W + 2 * HALF))
    p[:, HALF:HALF + H, HALF:HALF + W] = a
    out = np.zeros_like(a, dtype=np.float64)
    for dy in range(2 * HALF + 1):
        for dx in range(2 * HALF + 1):
            out += w[dy, dx] * p[:, dy:dy + H, dx:dx + W]
    return out


def ssim_map(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    w = gaussian_window()
    mx, my = _filter(x, w), _filter(y, w)
    sxx = _filter(x * x, w) - mx * mx
    syy = _filter(y * y, w) - my * my
    sxy = _filter(x * y, w) - mx * my
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))


def loss_and_grad(image: np.ndarray, target: np.ndarray, lam: float = 0.2, need_grad: bool = True):
    """Loss of one view ([3,H,W] arrays) and dL/dimage.

    SSIM-map terms per pixel: A1 = 2 mx my + C1, A2 = 2 sxy + C2,
    B1 = mx^2 + my^2 + C1, B2 = sxx + syy + C2, m = A1 A2 / (B1 B2), with
    sxx = E[x^2] - mx^2 and sxy = E[xy] - mx my.  Taking mx, E[x^2], E[xy] as
    the variables that depend on x, the chain rule through the (self-adjoint,
    symmetric) window filter gives
      d mean(m) / dx = (1/n) [ F(dm/dmx) + 2 x F(dm/dEx2) + y F(dm/dExy) ].
    """
    x = np.asarray(image, np.float64)
    y = np.asarray(target, np.float64)
    n = x.size
    w = gaussian_window()
    mx, my = _filter(x, w), _filter(y, w)
    ex2, ey2, exy = _filter(x * x, w), _filter(y * y, w), _filter(x * y, w)
    sxx, syy, sxy = ex2 - mx * mx, ey2 - my * my, exy - mx * my
    A1, A2 = 2 * mx * my + C1, 2 * sxy + C2
    B1, B2 = mx * mx + my * my + C1, sxx + syy + C2
    D = B1 * B2
    m = A1 * A2 / D
    l1 = np.abs(x - y).mean()
    ssim = m.mean()
    L = (1.0 - lam) * l1 + lam * (1.0 - ssim)
    if not need_grad:
        return L, None
    dm_dmx = (2 * my * A2 - 2 * my * A1) / D - m * (2 * mx * B2 - 2 * mx * B1) / D
    dm_dex2 = -m / B2
    dm_dexy = 2 * A1 / D
    dssim = (_filter(dm_dmx, w) + 2 * x * _filter(dm_dex2, w) + y * _filter(dm_dexy, w)) / n
    dl1 = np.sign(x - y) / n
    return L, (1.0 - lam) * dl1 - lam * dssim
