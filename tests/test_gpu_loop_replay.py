"""The refinement loop at the bench's workload (3M Gaussians SH3, 200 ring
views at 1297x840), run as the captured CUDA graph: the per-iteration log of
losses and gate decisions, replayed through the Algorithm 1 oracle, gives
the same decisions bit for bit; the logged gradient and update norms are
zero exactly on the skipped iterations.  A batched run (2 views per
iteration) is replayed the same way under reading (vii).  The bench's list
form (super-tile lists) and the tile lists both."""
import numpy as np
import pytest
import torch

import synth
from oracle.gate import Gate as OGate, GateConfig
from tests import gpu_util

pytestmark = pytest.mark.gpu

ITERS = 800


def _targets(gt, cams, raster, dev):
    mgt = raster.GaussianModel.from_scene(gt, dev)
    r = raster.Renderer(gt.n, 3, raster.Views([cams[0]], 16, dev), raster.RasterSettings(), 24 * gt.n, dev)
    out = torch.empty((len(cams), 3, cams[0].height, cams[0].width), dtype=torch.float32, device=dev)
    for v, cam in enumerate(cams):
        r.views = raster.Views([cam], 16, dev)
        r.forward(mgt.c_params())
        out[v].copy_(r.image.view(3, cam.height, cam.width))
    torch.cuda.synchronize()
    return out


def _replay(seq, log, B, W):
    cfg = GateConfig(W=W, beta=0.95, eps=1e-8, rho_lo=0.5, n_views=200)
    og = OGate(cfg)
    want = np.zeros_like(log["g"], dtype=int)
    for k in range(log["g"].shape[0]):
        items = [(int(seq[k * B + j]), float(log["loss"][k, j])) for j in range(B)]
        want[k] = [og.decide(v, L) for v, L in items]
        for v, L in items:
            og.update(v, L)
    return want


@pytest.mark.parametrize("B,coarse", [(1, True), (1, False), (2, True)])
def test_loop_decisions_replay_bit_exact(B, coarse):
    from paper_2603_08997_gb300 import raster
    from paper_2603_08997_gb300.refine import RefinementLoop
    gpu_util.lib()
    dev = torch.device("cuda")
    gt, start, cams, seq = synth.case_c3(n_iters=ITERS * B)
    targets = _targets(gt, cams, raster, dev)
    model = raster.GaussianModel.from_scene(start, dev)
    W = 500 if B == 1 else 300
    loop = RefinementLoop(model, cams, targets, seq, raster.RasterSettings(coarse_lists=coarse), gated=True, W=W,
                          views_per_step=B, pair_capacity=24 * gt.n * B, log_capacity=ITERS)
    loop.capture()
    for _ in range(ITERS):
        loop.step_graph()
    torch.cuda.synchronize()
    assert int(loop.renderer.status.item()) == 0
    log = loop.read_log(ITERS)
    loop.close()
    assert np.isfinite(log["loss"]).all() and (log["loss"] > 0).all()
    want = _replay(np.asarray(seq), log, B, W)
    assert np.array_equal(log["g"].astype(int), want)
    stepped = log["g"].any(axis=1)
    assert 0 < (~stepped).sum() < ITERS  # the gate skipped some iterations, not all
    assert (log["grad_sq"][~stepped] == 0).all() and (log["update_sq"][~stepped] == 0).all()
    assert (log["grad_sq"][stepped] > 0).all() and (log["update_sq"][stepped] > 0).all()
