"""The refinement loop's own backward path against the FP64 oracle, and
stress cases of the adjoint's transmittance rebuild.

* gs_render_bwd_adam - the raster adjoint followed by the projection adjoint
  fused with Adam, the loop's backward branch - against oracle.backward then
  oracle.adam_step, after 1 and 3 steps at C1 (2,000 Gaussians, 64x64) and at
  the full C2 size (200,000 Gaussians SH3, 980x545).  Adam's first step moves
  every parameter with a non-zero gradient by exactly its learning rate in
  the gradient's direction, so an element whose gradient is smaller than the
  float32 gradient error can move the other way, and one whose gradient is
  below 1e-10 (near Adam's eps = 1e-15) moves by an amount that depends on
  |g| itself: those elements (the GPU's own float32 gradient, from
  gs_render_bwd on the same state, differs in sign from the oracle's, or
  |g| < 1e-10) are counted and bounded by two learning rates per step.
  dL/dimage is zeroed on both sides where the L1 sign is a float32 tie
  (gpu_util.l1_tie_mask, decided from the oracle's own image).
  Every other parameter must agree within 2e-6 relative (normwise per group,
  and per element against 2e-6 of the group's RMS); the moments within the
  gradient bar (m 1e-4, v 2e-4 normwise).
  Both list forms (tile lists; super-tile lists filtered by the kernels, the
  bench's form) at C1 and at the full C2 size.
* The raster adjoint on near-opaque stacks: 600 Gaussians over a 32x32 image,
  alpha' reaching the 0.99 clamp at positions 40 and 230; with both, every
  pixel has 230 contributors inside the first 256-record batch and stops
  there; with one, the transmittance floor is reached in the second batch.
  The in-batch rebuild T_k = T_(k+1) / (1 - alpha'_k) divides by 0.01 at the
  clamped records.  g2d within 1e-4 normwise, cosine >= 0.9999.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle.adam import AdamConfig, adam_step
from paper_2603_08997_gb300 import raster
from tests import gpu_util

pytestmark = pytest.mark.gpu

GROUPS = ("means", "log_scales", "quats", "opacity_logit", "sh")


def _lr(cfg: AdamConfig, n: int, K: int) -> dict:
    sh = np.empty((n, K, 3))
    sh[:, 0, :] = cfg.lr_sh_dc
    sh[:, 1:, :] = cfg.lr_sh_rest
    return {"means": cfg.lr_means, "log_scales": cfg.lr_log_scales, "quats": cfg.lr_quats,
            "opacity_logit": cfg.lr_opacity, "sh": sh.ravel()}


def _scene64(p: dict, like) -> synth.Scene:
    """The oracle's parameters as a float64 scene (its projection takes them as they are)."""
    return synth.Scene(p["means"].reshape(-1, 3), p["log_scales"].reshape(-1, 3), p["quats"].reshape(-1, 4),
                       p["opacity_logit"].reshape(-1), p["sh"].reshape(like.sh.shape))


def _grad_vec(g: dict) -> dict:
    return {k: np.asarray(g[k], np.float64).ravel() for k in GROUPS}


@pytest.mark.parametrize("case,steps,coarse", [("c1", 1, False), ("c1", 3, False), ("c2", 1, False),
                                               ("c2", 3, False), ("c1", 3, True), ("c2", 3, True)])
def test_fused_backward_adam_against_oracle(case, steps, coarse):
    gpu_util.lib()
    rc = oracle.RasterConfig()
    if case == "c1":
        scene, cam, target = synth.case_c1()
    else:
        scene, tscene, cam, noise = synth.case_c2()  # the full 200,000-Gaussian size
        target = (oracle.forward(tscene, cam, rc)["image"] + noise).astype(np.float32)
    cfg = AdamConfig()
    views = raster.Views([cam], 16)
    r = raster.Renderer(scene.n, scene.sh_degree, views, raster.RasterSettings(coarse_lists=coarse))
    model = raster.GaussianModel.from_scene(scene)
    adam = raster.AdamState(model, lr=cfg.lrs(), beta1=cfg.beta1, beta2=cfg.beta2, eps=cfg.eps)
    grad = torch.zeros_like(model.flat)
    tgt = torch.from_numpy(target.ravel()).cuda()
    n, K = scene.n, scene.sh.shape[1]
    lr = _lr(cfg, n, K)
    p = {k: getattr(scene, k).astype(np.float64).ravel() for k in GROUPS}
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(x) for k, x in p.items()}
    ambiguous = {k: np.zeros(p[k].shape, bool) for k in GROUPS}
    flipped = {k: np.zeros(p[k].shape, bool) for k in GROUPS}
    for step in range(steps):
        s64 = _scene64(p, scene)
        f = oracle.forward(s64, cam, rc, margin_rel=1e-4)
        L, dL = oracle.loss_and_grad(f["image"], target)
        # the L1 sign is a float32 tie where the oracle's image is within 1e-4
        # of the target: dL/dimage zeroed there on both sides
        tie = gpu_util.l1_tie_mask(f["image"], target, f["margin"])
        dL[tie] = 0.0
        g_orc = _grad_vec(oracle.backward(s64, cam, rc, f, dL))
        r.forward(model.c_params())
        r.compute_loss(tgt, with_grad=True)
        r.dL_dimage.view(3, cam.height, cam.width)[torch.from_numpy(tie).cuda()] = 0.0
        # the GPU's own float32 gradient of the current state (unfused path),
        # only to find the elements whose gradient sign float32 cannot resolve
        r.backward(model.c_params(), model.c_grads(grad))
        g_gpu = _grad_vec(gpu_util.gpu_grads(model, grad))
        # the loop's backward branch: raster adjoint, projection adjoint + Adam
        r.backward_adam(model, adam)
        torch.cuda.synchronize()
        assert int(r.status.item()) == 0
        for k in GROUPS:
            # Adam's step is a function of the gradient's sign only where
            # |g| >> eps (first step: g / (|g| + eps)); below 1e-10 it also
            # depends on |g|, which float32 does not resolve
            # (a gradient exactly zero on both sides leaves the element in place)
            tiny = (np.abs(g_orc[k]) < 1e-10) & ((g_orc[k] != 0) | (g_gpu[k] != 0))
            flip = (np.sign(g_gpu[k]) != np.sign(g_orc[k])) & ~tiny
            flipped[k] |= flip
            ambiguous[k] |= flip | tiny
            p[k], m[k], v[k], _ = adam_step(p[k], g_orc[k], m[k], v[k], step, lr[k], cfg)
    assert int(adam.step_count.item()) == steps
    got_p = _grad_vec(gpu_util.gpu_grads(model, model.flat))
    got_m = _grad_vec(gpu_util.gpu_grads(model, adam.m))
    got_v = _grad_vec(gpu_util.gpu_grads(model, adam.v))
    for k in GROUPS:
        amb = ambiguous[k]
        # unresolved elements (sign or magnitude below float32's reach): each
        # within two learning rates per step; sign flips of gradients above
        # 1e-10 are rare (< 0.1%); the tiny ones are near-invisible Gaussians
        assert flipped[k].mean() < 1e-3, (k, int(flipped[k].sum()))
        assert amb.mean() < 0.1, (k, int(amb.sum()))
        lr_k = np.broadcast_to(lr[k], p[k].shape)
        assert np.all(np.abs(got_p[k] - p[k])[amb] <= 2.0 * steps * lr_k[amb] * (1 + 1e-3)), k
        ok = ~amb
        ref, got = p[k][ok], got_p[k][ok]
        assert gpu_util.rel_err(got, ref) <= 2e-6, (k, gpu_util.rel_err(got, ref))
        if steps == 1:
            # one step moves every resolved element by exactly +-lr on both
            # sides: per element, within 2e-6 of the larger of |p| and the RMS
            rms = np.sqrt(np.mean(ref ** 2))
            bad = np.abs(got - ref) > 2e-6 * np.maximum(np.abs(ref), rms)
            if bad.any():
                j = int(np.argmax(np.abs(got - ref) / np.maximum(np.abs(ref), rms)))
                idx = np.nonzero(ok)[0][j]
                raise AssertionError((k, int(bad.sum()), int(idx), float(got[j]), float(ref[j]),
                                      float(g_orc[k][idx]), float(g_gpu[k][idx])))
        if np.linalg.norm(m[k][ok]) > 0:
            assert gpu_util.rel_err(got_m[k][ok], m[k][ok]) <= 1e-4, (k, gpu_util.rel_err(got_m[k][ok], m[k][ok]))
            assert gpu_util.rel_err(got_v[k][ok], v[k][ok]) <= 2e-4, (k, gpu_util.rel_err(got_v[k][ok], v[k][ok]))


def _stack_case(clamp_at, tile=16, batch=256, ppt=2, coarse=False):
    gpu_util.lib()
    cam = synth.camera_pinhole(50, 50, 16, 16, 32, 32)
    rec = synth.opaque_stack_records(600, 32, 32, clamp_at=clamp_at, seed=3)
    views = raster.Views([cam], tile)
    r = raster.Renderer(600, 0, views, raster.RasterSettings(tile=tile, batch=batch, pixels_per_thread=ppt,
                                                              pixels_per_thread_fwd=ppt, coarse_lists=coarse))
    dev, orc = gpu_util.records([rec], [cam], tile)
    gpu_util.set_projected(r, dev)
    r.bin_sort()
    r.render_fwd()
    return cam, r, orc[0]


@pytest.mark.parametrize("clamp_at", [(40, 230), (40,)])
@pytest.mark.parametrize("tile,batch,ppt,coarse", [(16, 256, 2, False), (16, 128, 1, False), (8, 256, 2, False),
                                                   (32, 256, 2, False), (16, 256, 2, True), (8, 128, 1, True)])
def test_raster_bwd_near_opaque_stack(clamp_at, tile, batch, ppt, coarse):
    cam, r, orc = _stack_case(clamp_at, tile, batch, ppt, coarse)
    dl = synth.dl_dimage(cam.width, cam.height, seed=9)
    g2d = r.raster_bwd(dL_dimage=torch.from_numpy(dl.ravel()).cuda()).double().cpu().numpy()[0]
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0
    rc = oracle.RasterConfig(tile=tile)
    _, ovals, oranges, _ = oracle.bin_sort([orc], [cam], tile)
    o = oracle.render(orc, cam, ovals, oranges, rc, 0)
    nl = r.n_last.view(cam.height, cam.width).cpu().numpy()
    agree = (nl == o["n_last"]) | o["margin"].astype(bool)
    assert agree.all()
    if clamp_at == (40, 230):
        # 230 contributors, all inside the first 256-record batch, then the stop
        assert (o["n_contrib"] == 230).all() and (o["n_last"] == 230).all()
    else:
        assert o["n_last"].min() > 256  # the floor is reached in the second batch
    og = oracle.raster_bwd(orc, cam, ovals, oranges, rc, dl.astype(np.float64))
    for name, sl in (("mean2d", slice(0, 2)), ("conic", slice(2, 5)), ("opacity", slice(5, 6)), ("rgb", slice(6, 9))):
        a, b = g2d[:, sl], og[:, sl]
        assert gpu_util.rel_err(a, b) < 1e-4, (name, gpu_util.rel_err(a, b))
        assert gpu_util.cosine(a, b) > 0.9999, name
    # record 40 is clamped at every pixel: alpha' = 0.99 passes no gradient to
    # its opacity, mean or conic on either side; record 230 (when present) is
    # never composited
    assert np.all(og[40, 0:6] == 0.0) and np.all(g2d[40, 0:6] == 0.0)
    assert np.any(og[40, 6:9] != 0.0)
    if 230 in clamp_at:
        assert np.all(og[230] == 0.0) and np.all(g2d[230] == 0.0)
    img = r.image_of(0).cpu().numpy()
    np.testing.assert_allclose(img, o["image"], rtol=1e-5, atol=1e-5 * np.abs(o["image"]).max())
