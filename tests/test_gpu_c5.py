"""Stress size: 6M Gaussians SH3, 4 views at 1920x1080 in one batched call
(about 5e8 pairs).  The GPU renders and back-propagates the full views; the
oracle evaluates windows of them (tests/crop_util.py).  Window pixels within
1e-5 relative (outside near-cut-off pixels the oracle flags), and the
gradients of L = sum over views of <weights, window> - computed by the GPU
from dL/dimage = weights on the windows and 0 elsewhere - within 1e-4
normwise per parameter group, cosine >= 0.9999."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2603_08997_gb300 import raster
from tests import crop_util, gpu_util

pytestmark = pytest.mark.gpu

RC = oracle.RasterConfig()
WINDOWS = [(940, 524, 48, 32), (600, 300, 40, 24), (1300, 700, 32, 32), (960, 180, 40, 24)]


def test_c5_windows_against_oracle():
    gpu_util.lib()
    scene, cams = synth.case_c5()
    views = raster.Views(cams, 16)
    r = raster.Renderer(scene.n, 3, views, raster.RasterSettings(), pair_capacity=200_000_000 * len(cams))
    model = raster.GaussianModel.from_scene(scene)
    grad = torch.zeros_like(model.flat)
    rng = np.random.default_rng(3)
    wts = [rng.normal(size=(3, h, w)) for (_, _, w, h) in WINDOWS]
    dl = torch.zeros_like(r.image)
    for v, ((x0, y0, w, h), wt) in enumerate(zip(WINDOWS, wts)):
        full = np.zeros((3, cams[v].height, cams[v].width), np.float32)
        full[:, y0:y0 + h, x0:x0 + w] = wt
        dl[3 * views.pix_offsets[v]:3 * views.pix_offsets[v] + full.size] = torch.from_numpy(full.ravel())
    r.forward(model.c_params())
    r.backward(model.c_params(), model.c_grads(grad), dL_dimage=dl)
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0
    assert int(r.pair_count.item()) > 3e8
    got = gpu_util.gpu_grads(model, grad)

    s64 = crop_util.widen(scene)
    want = {k: np.zeros(got[k].shape) for k in got}
    for v, ((x0, y0, w, h), wt) in enumerate(zip(WINDOWS, wts)):
        o = crop_util.window_pass(s64, cams[v], RC, x0, y0, w, h, weights=wt)
        img = r.image_of(v).cpu().numpy()[:, y0:y0 + h, x0:x0 + w].astype(np.float64)
        ref, mask = o["image"], o["margin"].astype(bool)[None].repeat(3, 0)
        assert mask.mean() < 0.01
        d = np.where(mask, 0.0, np.abs(img - ref))
        assert d.max() <= 1e-5 * np.abs(ref).max()
        for k in want:
            want[k][o["idx"]] += o["grads"][k].reshape(want[k][o["idx"]].shape)
    for k in ("means", "log_scales", "quats", "opacity_logit", "sh"):
        a, b = got[k], want[k]
        assert gpu_util.rel_err(a, b) < 1e-4, (k, gpu_util.rel_err(a, b))
        assert gpu_util.cosine(a, b) > 0.9999, (k, gpu_util.cosine(a, b))
