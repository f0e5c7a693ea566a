"""GPU loss, backward and Adam against the FP64 oracle.

Tolerances: loss within 1e-5 relative; gradients per parameter group within
1e-4 normwise relative error with cosine >= 0.9999; Adam within 1e-6."""
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


def _setup(scene, cam, tile=16, batch=256, ppt=2, coarse=False):
    gpu_util.lib()
    views = raster.Views([cam], tile)
    r = raster.Renderer(scene.n, scene.sh_degree, views,
                        raster.RasterSettings(tile=tile, batch=batch, pixels_per_thread=ppt,
                                              pixels_per_thread_fwd=ppt, coarse_lists=coarse))
    model = raster.GaussianModel.from_scene(scene)
    return r, model


def test_loss_multi_view():
    sizes = [(64, 64), (97, 41), (33, 120)]
    cams = [synth.camera_pinhole(50, 50, w / 2, h / 2, w, h) for w, h in sizes]
    gpu_util.lib()
    views = raster.Views(cams, 16)
    r = raster.Renderer(10, 0, views)
    rng = np.random.default_rng(0)
    imgs = [rng.uniform(0, 1, (3, h, w)).astype(np.float32) for w, h in sizes]
    tgts = [np.clip(i + rng.normal(0, 0.1, i.shape), 0, 1).astype(np.float32) for i in imgs]
    r.image.copy_(torch.from_numpy(np.concatenate([i.ravel() for i in imgs])))
    tgt = torch.from_numpy(np.concatenate([t.ravel() for t in tgts])).cuda()
    r.compute_loss(tgt, with_grad=True)
    torch.cuda.synchronize()
    for v in range(3):
        L, dL = oracle.loss_and_grad(imgs[v], tgts[v])
        assert abs(float(r.loss[v].item()) - L) <= 1e-5 * abs(L)
        g = r.views.image_view(r.dL_dimage, v).cpu().numpy()
        assert gpu_util.rel_err(g, dL) < 1e-4


def test_loss_full_view():
    """The 1297 x 840 view: flat regions (SSIM's variances near zero, where the
    window sums' centre shift matters), smooth ramps and noise, over 41 x 27
    output tiles with ragged right and bottom edges."""
    w, h = 1297, 840
    cam = synth.camera_pinhole(900, 900, w / 2, h / 2, w, h)
    gpu_util.lib()
    views = raster.Views([cam], 16)
    r = raster.Renderer(10, 0, views)
    rng = np.random.default_rng(5)
    yy, xx = np.mgrid[0:h, 0:w]
    img = np.empty((3, h, w), np.float32)
    img[0] = 0.5 + 0.4 * np.sin(xx / 37.0) * np.cos(yy / 23.0)
    img[1] = np.where(xx < w // 2, 0.25, 0.75)  # flat halves
    img[2] = rng.uniform(0, 1, (h, w))
    tgt = np.clip(img + rng.normal(0, 0.05, img.shape) * (xx % 3 > 0), 0, 1).astype(np.float32)
    r.image.copy_(torch.from_numpy(img.ravel()))
    t = torch.from_numpy(tgt.ravel()).cuda()
    r.compute_loss(t, with_grad=True)
    torch.cuda.synchronize()
    L, dL = oracle.loss_and_grad(img, tgt)
    assert abs(float(r.loss[0].item()) - L) <= 1e-5 * abs(L)
    g = r.views.image_view(r.dL_dimage, 0).cpu().numpy()
    assert gpu_util.rel_err(g, dL) < 1e-4


def _check_grads(gg, og, tol=1e-4):
    for k in GROUPS:
        a, b = gg[k], og[k]
        if np.linalg.norm(b) == 0:
            assert np.linalg.norm(a) == 0
            continue
        assert gpu_util.rel_err(a, b) < tol, (k, gpu_util.rel_err(a, b))
        assert gpu_util.cosine(a, b) > 0.9999, (k, gpu_util.cosine(a, b))


@pytest.mark.parametrize("seed,deg", [(3, 3), (7, 1), (11, 0), (5, 2)])
def test_backward_linear_functional_tiny(seed, deg):
    scene, cam = synth.scene_tiny(40, seed=seed, sh_degree=deg)
    dl = synth.dl_dimage(cam.width, cam.height, seed)
    r, model = _setup(scene, cam)
    adam = raster.AdamState(model)
    r.forward(model.c_params())
    r.backward(model.c_params(), model.c_grads(adam.grad), dL_dimage=torch.from_numpy(dl.ravel()).cuda())
    torch.cuda.synchronize()
    rc = oracle.RasterConfig()
    f = oracle.forward(scene, cam, rc)
    og = oracle.backward(scene, cam, rc, f, dl.astype(np.float64))
    _check_grads(gpu_util.gpu_grads(model, adam.grad), og)


@pytest.mark.parametrize("tile,batch,ppt", [(16, 256, 2), (8, 64, 2), (32, 128, 2), (16, 128, 1)])
def test_backward_full_loss_c1(tile, batch, ppt):
    scene, cam, target = synth.case_c1()
    r, model = _setup(scene, cam, tile, batch, ppt)
    adam = raster.AdamState(model)
    r.forward(model.c_params())
    r.compute_loss(torch.from_numpy(target.ravel()).cuda(), with_grad=True)
    r.backward(model.c_params(), model.c_grads(adam.grad))
    torch.cuda.synchronize()
    rc = oracle.RasterConfig(tile=tile)
    f = oracle.forward(scene, cam, rc)
    L, dL = oracle.loss_and_grad(f["image"], target)
    assert abs(float(r.loss.item()) - L) <= 1e-5 * L
    og = oracle.backward(scene, cam, rc, f, dL)
    _check_grads(gpu_util.gpu_grads(model, adam.grad), og)


@pytest.mark.parametrize("coarse", [False, True])
def test_backward_c2(coarse):
    """The full C2 scene (200,000 Gaussians SH3, 980x545) through the loss,
    with tile lists and with super-tile lists.  dL/dimage is zeroed on both
    sides where the L1 sign is a float32 tie (gpu_util.l1_tie_mask, from the
    oracle's image); everywhere else each side uses its own loss gradient."""
    scene, tscene, cam, noise = synth.case_c2()
    rc = oracle.RasterConfig()
    target = (oracle.forward(tscene, cam, rc)["image"] + noise).astype(np.float32)
    r, model = _setup(scene, cam, coarse=coarse)
    adam = raster.AdamState(model)
    r.forward(model.c_params())
    r.compute_loss(torch.from_numpy(target.ravel()).cuda(), with_grad=True)
    f = oracle.forward(scene, cam, rc, margin_rel=1e-4)
    L, dL = oracle.loss_and_grad(f["image"], target)
    tie = gpu_util.l1_tie_mask(f["image"], target, f["margin"])
    assert tie.mean() < 0.02
    dL[tie] = 0.0
    r.dL_dimage.view(3, cam.height, cam.width)[torch.from_numpy(tie).cuda()] = 0.0
    r.backward(model.c_params(), model.c_grads(adam.grad))
    torch.cuda.synchronize()
    assert abs(float(r.loss.item()) - L) <= 1e-5 * L
    og = oracle.backward(scene, cam, rc, f, dL)
    _check_grads(gpu_util.gpu_grads(model, adam.grad), og)


def test_adam_against_oracle():
    gpu_util.lib()
    scene, _ = synth.scene_tiny(37, seed=1, sh_degree=3)
    model = raster.GaussianModel.from_scene(scene)
    cfg = AdamConfig()
    adam = raster.AdamState(model, lr=cfg.lrs(), beta1=cfg.beta1, beta2=cfg.beta2, eps=cfg.eps)
    rng = np.random.default_rng(4)
    o = model.offsets
    n, K = scene.n, scene.sh.shape[1]
    p = {k: getattr(scene, k).astype(np.float64).ravel() for k in GROUPS}
    m = {k: np.zeros_like(v) for k, v in p.items()}
    vv = {k: np.zeros_like(v) for k, v in p.items()}
    lr = {"means": cfg.lr_means, "log_scales": cfg.lr_log_scales, "quats": cfg.lr_quats,
          "opacity_logit": cfg.lr_opacity}
    sh_lr = np.where((np.arange(3 * K * n) % (3 * K)) < 3, cfg.lr_sh_dc, cfg.lr_sh_rest)
    do = torch.zeros(1, dtype=torch.int32, device="cuda")
    step = 0
    for it, on in enumerate([1, 1, 0, 1, 1, 0, 0, 1]):
        g = {k: rng.normal(size=v.shape) * 10.0 ** rng.uniform(-5, 0, v.shape) for k, v in p.items()}
        gv = model.group_views(adam.grad)
        for k in GROUPS:
            gv[k].copy_(torch.from_numpy(g[k].astype(np.float32).reshape(gv[k].shape)))
        do.fill_(on)
        adam.step(do_step=do, zero_grad=True)
        if on:
            for k in GROUPS:
                gk = g[k].astype(np.float32).astype(np.float64)
                p[k], m[k], vv[k], _ = adam_step(p[k], gk, m[k], vv[k], step, sh_lr if k == "sh" else lr[k], cfg)
            step += 1
    torch.cuda.synchronize()
    assert int(adam.step_count.item()) == step
    got = gpu_util.gpu_grads(model, model.flat)
    for k in GROUPS:
        np.testing.assert_allclose(got[k].ravel(), p[k], rtol=2e-6, atol=1e-7)
    assert float(adam.grad.abs().max().item()) == 0.0
    # padding between groups stays zero
    pad = torch.ones_like(model.flat, dtype=torch.bool)
    for k, (a, b) in {"means": (o[0], o[0] + 3 * n), "log_scales": (o[1], o[1] + 3 * n),
                      "quats": (o[2], o[2] + 4 * n), "opacity_logit": (o[3], o[3] + n),
                      "sh": (o[4], o[4] + 3 * K * n)}.items():
        pad[a:b] = False
    assert float(model.flat[pad].abs().max().item()) == 0.0


def test_autograd_function_matches_oracle():
    """render() and photometric_loss() as torch.autograd.Functions: gradients of
    the summed loss of two views against the oracle's."""
    from paper_2603_08997_gb300 import autograd
    gpu_util.lib()
    scene, cam0 = synth.scene_tiny(60, seed=9, sh_degree=2)
    cam1 = synth.camera_pinhole(28.0, 30.0, 20.0, 14.0, 40, 28)
    views = raster.Views([cam0, cam1], 16)
    r = raster.Renderer(scene.n, scene.sh_degree, views)
    model = raster.GaussianModel.from_scene(scene)
    rng = np.random.default_rng(1)
    tg = [rng.uniform(0, 1, (3, c.height, c.width)) for c in (cam0, cam1)]
    target = torch.from_numpy(np.concatenate([t.ravel() for t in tg]).astype(np.float32)).cuda()
    flat = model.flat.clone().requires_grad_(True)
    img = autograd.render(flat, model, r)
    losses = autograd.photometric_loss(img, target, r)
    losses.sum().backward()
    torch.cuda.synchronize()
    rc = oracle.RasterConfig()
    og = None
    for c, t in zip((cam0, cam1), tg):
        f = oracle.forward(scene, c, rc)
        L, dL = oracle.loss_and_grad(f["image"], t.astype(np.float32))
        og = oracle.backward(scene, c, rc, f, dL, og)
    _check_grads(gpu_util.gpu_grads(model, flat.grad), og)


@pytest.mark.parametrize("deg", [3, 0, 2])
def test_fused_backward_adam_equals_separate_calls(deg):
    """gs_render_bwd_adam, and gs_raster_bwd + gs_project_bwd_adam, equal
    gs_render_bwd followed by gs_adam_step over two steps, telemetry included.
    1500 Gaussians: full warps and a partial last warp of the fused sweep."""
    scene, cam = synth.scene_tiny(1500 + 13, seed=2, sh_degree=deg)
    target = torch.from_numpy(np.random.default_rng(3).uniform(0, 1, (3, cam.height, cam.width)).astype(np.float32))
    target = target.cuda().view(-1)
    out = []
    for form in ("separate", "fused", "split"):
        r, model = _setup(scene, cam)
        adam = raster.AdamState(model)
        norms = torch.zeros(2, dtype=torch.float64, device="cuda")
        for _ in range(2):
            r.forward(model.c_params())
            r.compute_loss(target, with_grad=True)
            if form == "fused":
                r.backward_adam(model, adam, norms2=norms)
            elif form == "split":
                r.raster_bwd()
                r.project_bwd_adam(model, adam, norms2=norms)
            else:
                r.backward(model.c_params(), model.c_grads(adam.grad))
                adam.step(norms2=norms)
        torch.cuda.synchronize()
        out.append((model.flat.clone(), adam.m.clone(), adam.v.clone(), int(adam.step_count.item()),
                    norms.cpu().numpy()))
    p0, m0, v0, s0, n0 = out[0]
    assert n0[0] > 0 and n0[1] > 0
    for p1, m1, v1, s1, n1 in out[1:]:
        assert s0 == s1 == 2
        torch.testing.assert_close(p1, p0, rtol=1e-6, atol=1e-7)
        torch.testing.assert_close(m1, m0, rtol=1e-5, atol=1e-10)
        torch.testing.assert_close(v1, v0, rtol=1e-5, atol=1e-14)
        np.testing.assert_allclose(n1, n0, rtol=1e-4)


@pytest.mark.parametrize("tile,ppt", [(16, 2), (8, 2), (32, 2), (16, 1), (16, 4), (32, 4)])
def test_raster_bwd_g2d_against_oracle(tile, ppt):
    """gs_raster_bwd alone, on synthetic records both sides share: the per-view
    per-Gaussian gradients wrt (mean2D, conic a b c, opacity, colour)."""
    sizes = [(150, 97), (64, 40)]
    cams = [synth.camera_pinhole(50, 50, w / 2, h / 2, w, h) for w, h in sizes]
    recs = [synth.projected_records(3000, w, h, seed=31 + v) for v, (w, h) in enumerate(sizes)]
    gpu_util.lib()
    views = raster.Views(cams, tile)
    r = raster.Renderer(3000, 0, views, raster.RasterSettings(tile=tile, pixels_per_thread=ppt, pixels_per_thread_fwd=ppt))
    dev, orc = gpu_util.records(recs, cams, tile)
    gpu_util.set_projected(r, dev)
    r.bin_sort()
    r.render_fwd()
    dls = [synth.dl_dimage(w, h, seed=5 + v) for v, (w, h) in enumerate(sizes)]
    dl = torch.from_numpy(np.concatenate([d.ravel() for d in dls])).cuda()
    g2d = r.raster_bwd(dL_dimage=dl).double().cpu().numpy()
    torch.cuda.synchronize()
    rc = oracle.RasterConfig(tile=tile)
    _, ovals, oranges, toff = oracle.bin_sort(orc, cams, tile)
    for v, cam in enumerate(cams):
        og = oracle.raster_bwd(orc[v], cam, ovals, oranges, rc, dls[v].astype(np.float64), int(toff[v]))
        for name, sl in (("mean2d", slice(0, 2)), ("conic", slice(2, 5)), ("opacity", slice(5, 6)), ("rgb", slice(6, 9))):
            a, b = g2d[v][:, sl], og[:, sl]
            assert gpu_util.rel_err(a, b) < 1e-4, (v, name, gpu_util.rel_err(a, b))
            assert gpu_util.cosine(a, b) > 0.9999


def test_split_backward_equals_render_bwd():
    scene, cam = synth.scene_tiny(200, seed=4, sh_degree=3)
    dl = torch.from_numpy(synth.dl_dimage(cam.width, cam.height, 2).ravel()).cuda()
    r, model = _setup(scene, cam)
    g1 = torch.zeros_like(model.flat)
    g2 = torch.zeros_like(model.flat)
    r.forward(model.c_params())
    r.backward(model.c_params(), model.c_grads(g1), dL_dimage=dl)
    r.raster_bwd(dL_dimage=dl)
    r.project_bwd(model.c_params(), model.c_grads(g2))
    torch.cuda.synchronize()
    # equal up to the order of the float atomics in the raster adjoint
    assert gpu_util.rel_err(g2.cpu().numpy(), g1.cpu().numpy()) < 1e-6


def test_backward_mixed_pixels_per_thread():
    """The checkpoint layout is independent of the thread mapping: a forward
    pass with 2 pixels per thread feeds a backward pass with 1 and the other
    way round, with the same gradients up to float atomic order."""
    scene, cam = synth.scene_tiny(300, seed=8, sh_degree=2)
    dl = torch.from_numpy(synth.dl_dimage(cam.width, cam.height, 3).ravel()).cuda()
    res = []
    for f_ppt, b_ppt in ((1, 1), (2, 1), (1, 2), (2, 2)):
        r, model = _setup(scene, cam, tile=8, batch=64, ppt=f_ppt)
        g = torch.zeros_like(model.flat)
        r.forward(model.c_params())
        r.cfg.pixels_per_thread = b_ppt
        r.backward(model.c_params(), model.c_grads(g), dL_dimage=dl)
        torch.cuda.synchronize()
        assert int(r.status.item()) == 0
        res.append(g.cpu().numpy())
    for g in res[1:]:
        assert gpu_util.rel_err(g, res[0]) < 1e-6


@pytest.mark.parametrize("t0", [0, 1, 99, 2999, 29999])
def test_adam_bias_correction_at_step_counts(t0):
    """One Adam step after t0 executed steps (random moments) against the FP64
    oracle: the bias corrections 1 - beta^t hold from t = 1, where they are
    small differences, to t = 30000, where they are 1."""
    gpu_util.lib()
    scene, _ = synth.scene_tiny(64, seed=5, sh_degree=1)
    model = raster.GaussianModel.from_scene(scene)
    cfg = AdamConfig()
    adam = raster.AdamState(model, lr=cfg.lrs(), beta1=cfg.beta1, beta2=cfg.beta2, eps=cfg.eps)
    # the kernel receives the betas as float32 (gs_adam_config): the oracle
    # takes the same values, so 1 - beta2 agrees beyond the 1e-5 that
    # float32(0.999) differs from 0.999 by
    cfg = AdamConfig(beta1=float(np.float32(cfg.beta1)), beta2=float(np.float32(cfg.beta2)), eps=cfg.eps)
    rng = np.random.default_rng(10 + t0)
    n, K = scene.n, scene.sh.shape[1]
    lr = {"means": cfg.lr_means, "log_scales": cfg.lr_log_scales, "quats": cfg.lr_quats,
          "opacity_logit": cfg.lr_opacity,
          "sh": np.where((np.arange(3 * K * n) % (3 * K)) < 3, cfg.lr_sh_dc, cfg.lr_sh_rest)}
    model.flat.zero_()  # p = 0: the float32 result carries the update to full relative precision
    pv, mv, vv, gv = (model.group_views(x) for x in (model.flat, adam.m, adam.v, adam.grad))
    state = {}
    for k in GROUPS:
        shape = tuple(pv[k].shape)
        g = rng.normal(0, 1e-3, shape).astype(np.float32)
        m = (rng.normal(0, 1e-3, shape) if t0 else np.zeros(shape)).astype(np.float32)
        v = (rng.uniform(1e-10, 1e-5, shape) if t0 else np.zeros(shape)).astype(np.float32)
        gv[k].copy_(torch.from_numpy(g))
        mv[k].copy_(torch.from_numpy(m))
        vv[k].copy_(torch.from_numpy(v))
        state[k] = (pv[k].double().cpu().numpy().ravel(), g.astype(np.float64).ravel(), m.astype(np.float64).ravel(),
                    v.astype(np.float64).ravel())
    adam.step_count.fill_(t0)
    adam.step()
    torch.cuda.synchronize()
    assert int(adam.step_count.item()) == t0 + 1
    for k in GROUPS:
        p0, g, m, v = state[k]
        p1, m1, v1, _ = adam_step(p0, g, m, v, t0, lr[k], cfg)
        got = pv[k].double().cpu().numpy().ravel()
        # moments: a few float32 roundings of the two terms (the sum may cancel)
        m_tol = 4e-7 * (cfg.beta1 * np.abs(m) + (1 - cfg.beta1) * np.abs(g))
        v_tol = 4e-7 * (cfg.beta2 * v + (1 - cfg.beta2) * g * g)
        # update: 2e-5 of itself (SFU square root and reciprocal, bias
        # corrections) plus what the first moment's rounding carries
        t = t0 + 1
        den = np.sqrt(v1 / (1 - cfg.beta2 ** t)) + cfg.eps
        p_tol = 2e-5 * np.abs(p1) + lr[k] * m_tol / (1 - cfg.beta1 ** t) / den
        assert np.all(np.abs(got - p1) <= p_tol)
        assert np.all(np.abs(mv[k].double().cpu().numpy().ravel() - m1) <= m_tol)
        assert np.all(np.abs(vv[k].double().cpu().numpy().ravel() - v1) <= v_tol)


def test_adam_norms_telemetry():
    """gs_adam_step's optional norms: sum g^2 and sum (p_new - p_old)^2."""
    gpu_util.lib()
    scene, _ = synth.scene_tiny(500, seed=9, sh_degree=3)
    model = raster.GaussianModel.from_scene(scene)
    adam = raster.AdamState(model)
    rng = np.random.default_rng(1)
    adam.grad.copy_(torch.from_numpy(rng.normal(0, 1e-3, adam.grad.numel()).astype(np.float32)))
    g = adam.grad.double().clone()
    p0 = model.flat.double().clone()
    norms = torch.zeros(2, dtype=torch.float64, device="cuda")
    adam.step(norms2=norms)
    torch.cuda.synchronize()
    want = [float((g * g).sum()), float(((model.flat.double() - p0) ** 2).sum())]
    got = norms.cpu().numpy()
    assert abs(got[0] - want[0]) <= 1e-5 * want[0] and abs(got[1] - want[1]) <= 1e-4 * want[1]


def test_adam_learning_rate_scaled_by_opened_views():
    """gs_adam_config.lr_scale_den: with the step-gate word holding the number
    of opened views k, the step's learning rates are lr * k / den (against
    the FP64 oracle with the scaled rates); k = 0 still skips the step."""
    gpu_util.lib()
    scene, _ = synth.scene_tiny(50, seed=3, sh_degree=2)
    model = raster.GaussianModel.from_scene(scene)
    cfg = AdamConfig()
    adam = raster.AdamState(model, lr=cfg.lrs(), beta1=cfg.beta1, beta2=cfg.beta2, eps=cfg.eps)
    adam.cfg.lr_scale_den = 8
    n, K = scene.n, scene.sh.shape[1]
    rng = np.random.default_rng(8)
    p = {k: getattr(scene, k).astype(np.float64).ravel() for k in GROUPS}
    m = {k: np.zeros_like(v) for k, v in p.items()}
    vv = {k: np.zeros_like(v) for k, v in p.items()}
    lr = {"means": cfg.lr_means, "log_scales": cfg.lr_log_scales, "quats": cfg.lr_quats,
          "opacity_logit": cfg.lr_opacity}
    sh_lr = np.where((np.arange(3 * K * n) % (3 * K)) < 3, cfg.lr_sh_dc, cfg.lr_sh_rest)
    do = torch.zeros(1, dtype=torch.int32, device="cuda")
    step = 0
    for k_open in (3, 0, 8, 1):
        g = {k: rng.normal(size=v.shape) for k, v in p.items()}
        gv = model.group_views(adam.grad)
        for k in GROUPS:
            gv[k].copy_(torch.from_numpy(g[k].astype(np.float32).reshape(gv[k].shape)))
        do.fill_(k_open)
        adam.step(do_step=do, zero_grad=True)
        if k_open:
            for k in GROUPS:
                gk = g[k].astype(np.float32).astype(np.float64)
                rate = (sh_lr if k == "sh" else lr[k]) * (k_open / 8.0)
                p[k], m[k], vv[k], _ = adam_step(p[k], gk, m[k], vv[k], step, rate, cfg)
            step += 1
    torch.cuda.synchronize()
    assert int(adam.step_count.item()) == step == 3
    got = gpu_util.gpu_grads(model, model.flat)
    for k in GROUPS:
        np.testing.assert_allclose(got[k].ravel(), p[k], rtol=2e-6, atol=1e-7)
