"""Adaptive density control on the GPU against the oracle (oracle/densify.py).

* The statistic after backward passes: view counts bit-exact; the summed
  gradient norms within 1e-4 normwise of the oracle's accumulation of its own
  FP64 2D gradients (the gradient bar), and within 1e-6 of the oracle's
  accumulation of the GPU's 2D gradients.
* Decisions and output offsets bit-exact given identical statistics (both
  sides decide in float32), on random statistics around the thresholds, on
  3M Gaussians (many scan blocks) and on edge cases (nothing changes,
  everything pruned, one Gaussian).
* The output set: copies and moments exact, split children within 1e-6 of
  the FP64 oracle given the same noise.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import densify as D
from paper_2603_08997_gb300 import gsr, raster
from paper_2603_08997_gb300.refine import densification_phase
from tests import gpu_util

pytestmark = pytest.mark.gpu

GROUPS = ("means", "log_scales", "quats", "opacity_logit", "sh")


def _cfg(grad_thr, log_size_thr, logit_thr):
    c = gsr.gs_densify_config()
    c.grad_thr, c.log_size_thr, c.logit_prune_thr, c.log_split_shrink = grad_thr, log_size_thr, logit_thr, np.log(1.6)
    return c


def _ocfg(c):
    return D.DensifyConfig(grad_thr=c.grad_thr, log_size_thr=c.log_size_thr, logit_prune_thr=c.logit_prune_thr,
                           log_split_shrink=float(np.float32(c.log_split_shrink)))


def _random_model(n, deg=1, seed=0):
    rng = np.random.default_rng(seed)
    K = (deg + 1) ** 2
    scene = synth.Scene(rng.normal(size=(n, 3)).astype(np.float32), rng.normal(-3, 0.6, (n, 3)).astype(np.float32),
                        rng.normal(size=(n, 4)).astype(np.float32), rng.normal(0, 2.5, n).astype(np.float32),
                        rng.normal(size=(n, K, 3)).astype(np.float32))
    return scene, raster.GaussianModel.from_scene(scene)


def _stats(n, seed=1):
    rng = np.random.default_rng(seed)
    st = raster.DensityStats(n)
    acc = (rng.exponential(1.0, n) * (rng.random(n) < 0.9)).astype(np.float32)
    den = rng.integers(0, 6, n).astype(np.int32)
    st.accum.copy_(torch.from_numpy(acc))
    st.denom.copy_(torch.from_numpy(den))
    return st, acc, den


@pytest.mark.parametrize("n", [1, 1000, 4097, 3_000_000])
def test_decide_and_offsets_bit_exact(n):
    gpu_util.lib()
    scene, model = _random_model(n, deg=0, seed=n)
    st, acc, den = _stats(n, seed=n + 1)
    c = _cfg(0.8, -2.9, -2.0)
    action, offsets = raster.densify_decide(model, st, c)
    torch.cuda.synchronize()
    want = D.decide(acc, den, scene.log_scales, scene.opacity_logit, _ocfg(c))
    got = action.cpu().numpy()
    assert np.array_equal(got, want)
    cnt = D.OUTPUTS[want]
    assert np.array_equal(offsets.cpu().numpy(), np.concatenate([[0], np.cumsum(cnt)]))
    if n >= 1000:
        assert all((want == a).any() for a in (D.KEEP, D.CLONE, D.SPLIT, D.PRUNE))


def test_decide_at_the_thresholds():
    """The hand-worked table of the oracle's pins, through the kernel."""
    import os
    t = []
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "densify_decisions.txt")):
        line = line.split("#")[0].strip()
        if line:
            t.append([float(x) for x in line.split()])
    t = np.array(t)
    n = t.shape[0]
    gpu_util.lib()
    model = raster.GaussianModel(n, 0)
    v = model.views
    v["log_scales"].copy_(torch.from_numpy(t[:, 2:5].astype(np.float32)))
    v["opacity_logit"].copy_(torch.from_numpy(t[:, 5].astype(np.float32)))
    st = raster.DensityStats(n)
    st.accum.copy_(torch.from_numpy(t[:, 0].astype(np.float32)))
    st.denom.copy_(torch.from_numpy(t[:, 1].astype(np.int32)))
    action, offsets = raster.densify_decide(model, st, _cfg(0.25, -2.0, -5.0))
    assert action.cpu().numpy().tolist() == t[:, 6].astype(int).tolist()


@pytest.mark.parametrize("deg", [0, 3])
def test_apply_against_oracle(deg):
    n = 3000
    gpu_util.lib()
    scene, model = _random_model(n, deg=deg, seed=5)
    adam = raster.AdamState(model)
    rng = np.random.default_rng(6)
    adam.m.copy_(torch.from_numpy(rng.normal(size=adam.m.numel()).astype(np.float32)))
    adam.v.copy_(torch.from_numpy(rng.uniform(0, 1, adam.v.numel()).astype(np.float32)))
    adam.step_count.fill_(17)
    st, acc, den = _stats(n, seed=7)
    c = _cfg(0.8, -2.9, -2.0)
    noise = rng.normal(size=(n, 2, 3)).astype(np.float32)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    old_m = gpu_util.gpu_grads(model, adam.m)
    old_v = gpu_util.gpu_grads(model, adam.v)
    new, new_adam, action = raster.densify(model, adam, st, c, torch.from_numpy(noise).cuda(), status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0 and int(new_adam.step_count.item()) == 17
    act = D.decide(acc, den, scene.log_scales, scene.opacity_logit, _ocfg(c))
    assert np.array_equal(action.cpu().numpy(), act)
    p = {k: getattr(scene, k).astype(np.float64) for k in GROUPS}
    m = {k: old_m[k] for k in GROUPS}
    v = {k: old_v[k] for k in GROUPS}
    op, om, ov = D.apply(p, m, v, act, noise.astype(np.float64), _ocfg(c))
    assert new.n == D.output_count(act) == op["means"].shape[0]
    gp = gpu_util.gpu_grads(new, new.flat)
    gm = gpu_util.gpu_grads(new, new_adam.m)
    gv = gpu_util.gpu_grads(new, new_adam.v)
    split_rows = np.repeat(act, D.OUTPUTS[act]) == D.SPLIT
    for k in GROUPS:
        assert np.array_equal(gm[k], om[k]) and np.array_equal(gv[k], ov[k]), k
        if k in ("means", "log_scales"):
            assert np.array_equal(gp[k][~split_rows], op[k][~split_rows]), k
            np.testing.assert_allclose(gp[k][split_rows], op[k][split_rows], rtol=1e-6, atol=1e-6)
        else:
            assert np.array_equal(gp[k], op[k]), k
    # padding between the groups of the new buffer stays zero
    o = new.offsets
    pad = torch.ones_like(new.flat, dtype=torch.bool)
    for a, w in ((0, 3), (1, 3), (2, 4), (3, 1), (4, 3 * (deg + 1) ** 2)):
        pad[o[a]:o[a] + w * new.n] = False
    assert float(new.flat[pad].abs().max().item()) == 0.0 if pad.any() else True


def test_apply_rejects_a_destination_of_the_wrong_size():
    n = 100
    gpu_util.lib()
    scene, model = _random_model(n, seed=8)
    adam = raster.AdamState(model)
    st, _, _ = _stats(n, seed=9)
    c = _cfg(0.8, -2.9, -2.0)
    action, offsets = raster.densify_decide(model, st, c)
    n_out = int(offsets[n].item())
    dst = raster.GaussianModel(n_out + 1, model.sh_degree)
    dm = torch.zeros_like(dst.flat)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    noise = torch.zeros((n, 2, 3), device="cuda")
    gsr.call("gs_densify_apply", gsr.ptr(model.flat), gsr.ptr(adam.m), gsr.ptr(adam.v), n, model.sh_degree,
             gsr.ptr(action), gsr.ptr(offsets), gsr.ptr(noise), C_byref(c), gsr.ptr(dst.flat), gsr.ptr(dm),
             gsr.ptr(dm), n_out + 1, gsr.ptr(status), gsr.stream_handle())
    torch.cuda.synchronize()
    assert int(status.item()) == gsr.GS_ERR_INVALID_ARG
    assert float(dst.flat.abs().max().item()) == 0.0


def C_byref(c):
    import ctypes
    return ctypes.byref(c)


def test_statistic_after_backward_against_oracle():
    """Two backward passes over two views of a C1-like scene: the statistic
    against the oracle's accumulation of (a) its own FP64 2D gradients and (b)
    the GPU's 2D gradients."""
    gpu_util.lib()
    scene, cam0, target0 = synth.case_c1(n=1500)
    cam1 = synth.camera_pinhole(60.0, 60.0, 30.0, 28.0, 60, 56)
    target1 = np.random.default_rng(3).uniform(0, 1, (3, 56, 60)).astype(np.float32)
    model = raster.GaussianModel.from_scene(scene)
    st = raster.DensityStats(scene.n)
    rc = oracle.RasterConfig()
    acc_o, den_o = np.zeros(scene.n), np.zeros(scene.n, np.int64)
    acc_g, den_g = np.zeros(scene.n), np.zeros(scene.n, np.int64)
    grad = torch.zeros_like(model.flat)
    for cam, target in ((cam0, target0), (cam1, target1)):
        r = raster.Renderer(scene.n, scene.sh_degree, raster.Views([cam], 16))
        r.forward(model.c_params())
        r.compute_loss(torch.from_numpy(target.ravel()).cuda(), with_grad=True)
        r.backward(model.c_params(), model.c_grads(grad))
        st.accumulate(r)
        torch.cuda.synchronize()
        g2d = r.bwd_ws.view(torch.float32)[:12 * scene.n].view(scene.n, 12).double().cpu().numpy()
        vis = r.touched.cpu().numpy() > 0
        f = oracle.forward(scene, cam, rc)
        L, dL = oracle.loss_and_grad(f["image"], target)
        og = oracle.backward(scene, cam, rc, f, dL)["g2d"]
        # visibility is the kernels' tile count (the oracle's wider rectangle
        # inflation may keep a Gaussian whose support reaches no pixel centre;
        # its 2D gradient is zero)
        assert np.all(og[~vis, 0:2] == 0.0)
        acc_o, den_o = D.accumulate(acc_o, den_o, og[:, 0:2], vis)
        acc_g, den_g = D.accumulate(acc_g, den_g, g2d[:, 0:2], vis)
    got_a = st.accum.double().cpu().numpy()
    got_d = st.denom.cpu().numpy()
    assert np.array_equal(got_d, den_o) and den_o.max() == 2
    assert gpu_util.rel_err(got_a, acc_o) < 1e-4
    np.testing.assert_allclose(got_a, acc_g, rtol=1e-6, atol=1e-12)


def test_densification_phase_grows_and_keeps_rendering():
    """A short densification phase on a C1-like scene: the count follows the
    decisions, the optimizer's step count carries on, and the loop keeps
    rendering (status clean) after each resize."""
    gpu_util.lib()
    scene, cam, target = synth.case_c1(n=800)
    cams = [cam]
    targets = torch.from_numpy(target[None]).cuda()
    model = raster.GaussianModel.from_scene(scene)
    cfg = raster.densify_config(grad_thr=1e-12, max_scale=float(np.exp(-2.8)), eps_alpha=0.02)
    seq = np.zeros(200, np.int32)
    model2, adam2, hist = densification_phase(model, cams, targets, seq, iters=60, cfg=cfg, interval=20, start=20)
    assert len(hist) == 3
    for (it, n0, c, s, p, n1, q) in hist:
        assert n1 == n0 + c + s - p
    assert hist[0][2] > 0 and hist[-1][5] == model2.n and int(adam2.step_count.item()) == 60
