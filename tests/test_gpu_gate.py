"""GPU gate kernels (skipgs_gate_*) against the Algorithm 1 oracle: decisions
bit-exact given identical float32 losses."""
import os

import numpy as np
import pytest
import torch

from oracle.gate import Gate as OGate, GateConfig
from tests import gpu_util

pytestmark = pytest.mark.gpu


def _run_gpu(cfg: GateConfig, views, losses, per_call=1):
    from paper_2603_08997_gb300 import raster
    gpu_util.lib()
    gate = raster.Gate(cfg.n_views, cfg.W, cfg.beta, cfg.eps, cfg.rho_lo)
    v = torch.as_tensor(np.asarray(views, np.int32)).cuda()
    L = torch.as_tensor(np.asarray(losses, np.float32)).cuda()
    g = torch.zeros(len(views), dtype=torch.uint8, device="cuda")
    for k in range(0, len(views), per_call):
        sl = slice(k, min(k + per_call, len(views)))
        gate.decide(v[sl], L[sl], g[sl])
        gate.update(v[sl], L[sl])
    torch.cuda.synchronize()
    return g.cpu().numpy().astype(int), gate.read(), int(gate.status.item())


def _run_oracle(cfg, views, losses, per_call=1):
    """Reading (vii) of the oracle gate: the losses of one launch are decided in
    order, each its own t, against the EMA as it stood before the launch; the
    EMA updates follow in order."""
    og = OGate(cfg)
    gs = []
    for k in range(0, len(views), per_call):
        items = [(int(v), float(np.float32(L))) for v, L in zip(views[k:k + per_call], losses[k:k + per_call])]
        gs += [og.decide(v, L) for v, L in items]
        for v, L in items:
            og.update(v, L)
    return np.array(gs), og


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("per_call", [1, 4])
def test_random_sequences_bit_exact(seed, per_call):
    rng = np.random.default_rng(seed)
    n_views = int(rng.integers(1, 7))
    cfg = GateConfig(W=int(rng.integers(0, 40)), beta=0.95, eps=1e-8, rho_lo=0.5, n_views=n_views)
    T = 600
    views = rng.integers(0, n_views, T)
    # slowly decreasing losses with noise: the regime where the gate skips
    losses = (np.exp(rng.normal(0, 0.05, T)) * np.linspace(0.3, 0.2, T)).astype(np.float32)
    g_gpu, st, status = _run_gpu(cfg, views, losses, per_call)
    g_orc, og = _run_oracle(cfg, views, losses, per_call)
    assert status == 0
    assert np.array_equal(g_gpu, g_orc)
    assert (st["t"], st["b"], st["n_w"], st["n_w1"]) == (og.t, og.b, og.n_w, og.n_w1)
    assert st["rho_min"] == og.rho_min
    assert 0 < g_gpu.sum() < T


def test_hand_trace():
    from tests.test_oracle_gate import _load_trace
    cfg, rows = _load_trace()
    g, st, _ = _run_gpu(cfg, [r[1] for r in rows], [r[2] for r in rows])
    assert list(g) == [r[3] for r in rows]
    assert st["b"] == 5 and st["rho_min"] == 0.5


def test_near_ties_bit_exact():
    """Losses one float32 ulp around the EMA: the decision depends on the last
    bit of the binary64 arithmetic, which both sides must share."""
    cfg = GateConfig(W=2, beta=0.5, eps=0.0, rho_lo=-1.0, n_views=1)
    base = np.float32(0.25)
    seq = [base, base]
    for k in range(200):
        seq.append(np.nextafter(base, np.float32(1 if k % 3 else -1), dtype=np.float32))
        seq.append(base)
    views = np.zeros(len(seq), np.int32)
    g_gpu, _, _ = _run_gpu(cfg, views, seq)
    g_orc, _ = _run_oracle(cfg, views, seq)
    assert np.array_equal(g_gpu, g_orc)


def test_no_budget_ablation():
    rng = np.random.default_rng(3)
    cfg = GateConfig(W=5, beta=0.9, eps=1e-8, rho_lo=-1.0, n_views=3)
    views = rng.integers(0, 3, 300)
    losses = np.linspace(1.0, 0.5, 300).astype(np.float32)
    g_gpu, _, _ = _run_gpu(cfg, views, losses)
    g_orc, _ = _run_oracle(cfg, views, losses)
    assert np.array_equal(g_gpu, g_orc) and g_gpu[cfg.W:].sum() < 30


def test_nonfinite_loss_reported_and_skipped():
    from paper_2603_08997_gb300 import gsr
    cfg = GateConfig(W=1, beta=0.5, eps=1e-8, rho_lo=0.5, n_views=2)
    views = [0, 1, 0, 1]
    losses = [1.0, 1.0, float("nan"), 0.5]
    g, st, status = _run_gpu(cfg, views, losses)
    assert status == gsr.GS_ERR_NONFINITE
    assert g[2] == 0 and st["errors"] == 1 and st["t"] == 3


def test_decide_reports_the_number_of_opened_views():
    """skipgs_gate_decide writes the number of g = 1 into dev_any (the
    batched step's learning-rate scale reads it)."""
    from paper_2603_08997_gb300 import raster
    gpu_util.lib()
    gate = raster.Gate(8, W=0)
    ids = torch.arange(4, dtype=torch.int32, device="cuda")
    g = torch.zeros(4, dtype=torch.uint8, device="cuda")
    any_out = torch.zeros(1, dtype=torch.int32, device="cuda")
    losses = torch.tensor([1.0, 1.0, 1.0, 1.0], device="cuda")
    gate.decide(ids, losses, g, any_out)  # no history: every view opens
    gate.update(ids, losses)
    torch.cuda.synchronize()
    assert int(any_out.item()) == 4 == int(g.sum().item())
    losses2 = torch.tensor([2.0, 0.5, 3.0, 0.25], device="cuda")  # two above their EMA, two below
    gate.decide(ids, losses2, g, any_out)
    torch.cuda.synchronize()
    assert int(any_out.item()) == int(g.sum().item())
