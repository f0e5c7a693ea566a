"""Pins of the loss oracle, Eq. (loss) with lambda = 0.2, against SSIM's
closed-form special cases and an independent torch conv2d implementation
(value via F.conv2d, gradient via autograd) in FP64."""
import numpy as np
import torch
import torch.nn.functional as F

from oracle.loss import C1, C2, gaussian_window, loss_and_grad, ssim_map


def _torch_loss(x, y, lam=0.2):
    w = torch.tensor(gaussian_window(), dtype=torch.float64).expand(3, 1, 11, 11)

    def filt(a):
        return F.conv2d(a.unsqueeze(0), w, padding=5, groups=3)[0]

    mx, my = filt(x), filt(y)
    sxx = filt(x * x) - mx * mx
    syy = filt(y * y) - my * my
    sxy = filt(x * y) - mx * my
    m = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    return (1 - lam) * (x - y).abs().mean() + lam * (1 - m.mean()), m


def test_ssim_identity():
    rng = np.random.default_rng(0)
    x = rng.uniform(size=(3, 20, 17))
    np.testing.assert_allclose(ssim_map(x, x), 1.0, rtol=0, atol=1e-13)
    L, g = loss_and_grad(x, x)
    assert abs(L) < 1e-13


def test_ssim_constant_images():
    """Constant a, b: away from the border all variances vanish, so the map is
    (2ab + C1) / (a^2 + b^2 + C1)."""
    a, b = 0.3, 0.7
    m = ssim_map(np.full((3, 30, 30), a), np.full((3, 30, 30), b))
    np.testing.assert_allclose(m[:, 5:-5, 5:-5], (2 * a * b + C1) / (a * a + b * b + C1), rtol=1e-12)


def test_window():
    w = gaussian_window()
    assert w.shape == (11, 11) and abs(w.sum() - 1) < 1e-15
    r = np.arange(11) - 5.0
    g = np.exp(-r * r / 4.5)
    np.testing.assert_allclose(w, np.outer(g, g) / g.sum() ** 2, rtol=1e-14)


def test_value_and_grad_vs_torch_autograd():
    rng = np.random.default_rng(1)
    x = rng.uniform(size=(3, 23, 31))
    y = np.clip(x + rng.normal(0, 0.1, size=x.shape), 0, 1)
    L, g = loss_and_grad(x, y)
    xt = torch.tensor(x, requires_grad=True)
    Lt, m = _torch_loss(xt, torch.tensor(y))
    Lt.backward()
    np.testing.assert_allclose(ssim_map(x, y), m.detach().numpy(), rtol=1e-12, atol=1e-14)
    assert abs(L - Lt.item()) <= 1e-13 * abs(L)
    np.testing.assert_allclose(g, xt.grad.numpy(), rtol=1e-10, atol=1e-15)


def test_grad_finite_difference():
    rng = np.random.default_rng(2)
    x = rng.uniform(size=(3, 12, 12))
    y = rng.uniform(size=(3, 12, 12))
    _, g = loss_and_grad(x, y)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 5, 6), (2, 11, 3), (0, 6, 11), (1, 3, 3)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (loss_and_grad(xp, y, need_grad=False)[0] - loss_and_grad(xm, y, need_grad=False)[0]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * abs(g[idx]) + 1e-12
