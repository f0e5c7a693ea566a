"""Pin of the oracle's analytic adjoint against central finite differences of
the oracle's own forward (FP64), on tiny scenes, skipping coordinates whose
perturbation changes a discrete decision (contribution set, order, clamp,
stop, frustum clamp, colour clamp) - the places where the loss has a jump or
a kink."""
import numpy as np
import pytest

import oracle
import synth

RC = oracle.RasterConfig()
NAMES = ("means", "log_scales", "quats", "opacity_logit", "sh")


def _fd_check(scene, cam, loss_fn, h, rtol, floor):
    f0 = oracle.forward(scene, cam, RC)
    L0, dL = loss_fn(f0["image"])
    grads = oracle.backward(scene, cam, RC, f0, dL)
    checked = skipped = 0
    worst = 0.0
    for nm in NAMES:
        arr = getattr(scene, nm)
        for i in range(arr.size):
            outs = []
            for sgn in (1.0, -1.0):
                s = scene.copy()
                a = getattr(s, nm).astype(np.float64).reshape(-1)
                a[i] += sgn * h
                setattr(s, nm, a.reshape(arr.shape))
                outs.append(oracle.forward(s, cam, RC))
            if any(o["hash"] != f0["hash"] or (o["proj"]["flags"] != f0["proj"]["flags"]).any() for o in outs):
                skipped += 1
                continue
            fd = (loss_fn(outs[0]["image"])[0] - loss_fn(outs[1]["image"])[0]) / (2 * h)
            an = grads[nm].reshape(-1)[i]
            # per-coordinate relative error, floored at `floor` x the group's largest gradient
            err = abs(fd - an) / max(abs(an), floor * np.abs(grads[nm]).max())
            worst = max(worst, err)
            checked += 1
            assert err <= rtol, (nm, i, fd, an)
    return checked, skipped, worst


@pytest.mark.parametrize("seed,deg", [(3, 3), (7, 1), (11, 0)])
def test_fd_linear_functional(seed, deg):
    """L = <Wt, C>: isolates the rasterizer adjoint from the loss."""
    scene, cam = synth.scene_tiny(10, seed=seed, sh_degree=deg)
    Wt = np.random.default_rng(seed).normal(size=(3, cam.height, cam.width))
    checked, skipped, worst = _fd_check(scene, cam, lambda img: ((img * Wt).sum(), Wt), 1e-5, 1e-4, 1e-4)
    assert checked > 0.9 * (checked + skipped)


def test_fd_full_loss():
    """L = 0.8 L1 + 0.2 (1 - SSIM) against a random target, chained through the loss oracle."""
    scene, cam = synth.scene_tiny(8, seed=5, sh_degree=2)
    target = np.random.default_rng(9).uniform(size=(3, cam.height, cam.width))
    checked, skipped, worst = _fd_check(scene, cam, lambda img: oracle.loss_and_grad(img, target), 1e-5,
                                        1e-4, 1e-4)
    assert checked > 0.9 * (checked + skipped)


def test_frustum_clamped_gaussian_fd():
    """A Gaussian outside 1.3x the field of view uses the clamped J (true derivative)."""
    cam = synth.camera_pinhole(32.0, 32.0, 16.0, 16.0, 32, 32)
    scene, _ = synth.scene_tiny(3, seed=2, sh_degree=0)
    scene.means[0] = np.array([1.8, 0.1, 2.0], np.float32)     # x/z = 0.9 > 1.3 * 0.5
    scene.log_scales[0] = np.log(np.array([0.6, 0.3, 0.2], np.float32))
    scene.opacity_logit[0] = 3.0
    pr = oracle.project(scene, cam, RC)
    assert pr["flags"][0] & 1 and pr["touched"][0] > 0
    Wt = np.random.default_rng(0).normal(size=(3, 32, 32))
    checked, skipped, worst = _fd_check(scene, cam, lambda img: ((img * Wt).sum(), Wt), 1e-5, 1e-4, 1e-4)
    assert checked > 0
