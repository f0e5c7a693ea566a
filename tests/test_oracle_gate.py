"""Pins of the gate oracle (Algorithm 1, Sec. 3.2-3.3) against a hand-worked
trace and the invariants the equations imply."""
import itertools
import math
import os

import numpy as np
import pytest

from oracle.gate import Gate, GateConfig

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gate_trace_w3.txt")


def _load_trace():
    cfg, rows = {}, []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        if parts[0].isalpha() or "_" in parts[0]:
            cfg[parts[0]] = float(parts[1])
        else:
            rows.append((int(parts[0]), int(parts[1]), float(parts[2]), int(parts[3])))
    return GateConfig(W=int(cfg["W"]), beta=cfg["beta"], eps=cfg["eps"], rho_lo=cfg["rho_lo"],
                      n_views=int(cfg["n_views"])), rows


def test_hand_trace():
    cfg, rows = _load_trace()
    gate = Gate(cfg)
    for t, v, L, g in rows:
        assert gate.step(v, L) == g, f"t={t}"
        assert gate.t == t
    assert gate.rho_min == 0.5 and gate.b == 5


def _run(cfg, views, losses):
    gate = Gate(cfg)
    gs, bs, rhos = [], [], []
    for v, L in zip(views, losses):
        gs.append(gate.step(int(v), float(L)))
        bs.append(gate.b)
        rhos.append(gate.rho_min)
    return gate, np.array(gs), np.array(bs), np.array(rhos)


@pytest.mark.parametrize("seed", range(8))
def test_invariants_random(seed):
    """g = 1 during warmup; rho_min in [rho_lo, 1]; budget invariant
    b(t) >= rho_min * t - 1 for every t after calibration (Eq. rhocum_check:
    whenever b/(t-1) < rho_min the iteration is forced, so b cannot fall more
    than one step below the line rho_min * t)."""
    rng = np.random.default_rng(seed)
    n_views = int(rng.integers(1, 6))
    cfg = GateConfig(W=int(rng.integers(1, 30)), beta=0.95, eps=1e-8, rho_lo=0.5, n_views=n_views)
    T = 400
    views = rng.integers(0, n_views, size=T)
    losses = np.exp(rng.normal(0, 0.3, size=T)) * np.linspace(1.0, 0.5, T)
    gate, gs, bs, rhos = _run(cfg, views, losses)
    assert gs[:cfg.W].all()
    assert cfg.rho_lo <= gate.rho_min <= 1.0
    for t in range(1, T + 1):
        assert bs[t - 1] >= gate.rho_min * t - 1 - 1e-12
        assert bs[t - 1] == gs[:t].sum()


def test_rho_lo_one_skips_at_most_once():
    """rho_lo = 1 gives rho_min = 1.  The budget test is strict (Eq. rhocum_check),
    so the first post-warmup iteration, where rho_cum = W/W = 1 ties rho_min, may
    skip; from then on rho_cum < 1 and every iteration is forced."""
    rng = np.random.default_rng(1)
    cfg = GateConfig(W=5, beta=0.9, eps=1e-8, rho_lo=1.0, n_views=3)
    _, gs, _, _ = _run(cfg, rng.integers(0, 3, 200), rng.uniform(0.1, 1.0, 200))
    assert (1 - gs).sum() <= 1 and gs[cfg.W + 1:].all()


def test_increasing_losses_never_skip():
    """Strictly increasing per-view losses keep s > 1 (the EMA is a convex
    combination of earlier, smaller losses), so the skip test never proposes a skip."""
    rng = np.random.default_rng(2)
    cfg = GateConfig(W=3, beta=0.95, eps=1e-8, rho_lo=0.5, n_views=4)
    views = rng.integers(0, 4, 300)
    losses = np.arange(1, 301) * 0.01
    _, gs, _, _ = _run(cfg, views, losses)
    assert gs.all()


def test_calibration_formula():
    """Eq. (rhohat)/(rhomincalib) on a controlled warmup: one view, losses
    alternating up/down so that exactly half of the recorded tests give g=1."""
    cfg = GateConfig(W=9, beta=0.5, eps=0.0, rho_lo=0.5, n_views=1)
    gate = Gate(cfg)
    seq = [1.0, 2.0, 1.0, 2.0, 1.0, 2.0, 1.0, 2.0, 1.0]
    for L in seq:
        gate.step(0, L)
    # recorded: t=2..9 (8 iterations); s>1 exactly when the loss went up:
    rec = [1 if seq[i] > e else 0 for i, e in enumerate(_emas(seq, 0.5)) if i > 0]
    gate.step(0, 1.5)  # t = W+1 calibrates
    rho_hat = sum(rec) / len(rec)
    assert gate.n_w == 8 and gate.n_w1 == sum(rec)
    assert gate.rho_min == 0.5 + 0.5 * rho_hat


def _emas(seq, beta):
    out, e = [], None
    for L in seq:
        out.append(e if e is not None else -math.inf)
        e = L if e is None else beta * e + (1 - beta) * L
    return out


def test_no_history_in_warmup_keeps_rho_lo():
    """Reading (iii): every warmup iteration hits a fresh view -> rho_min = rho_lo."""
    cfg = GateConfig(W=4, beta=0.5, eps=0.0, rho_lo=0.5, n_views=8)
    gate = Gate(cfg)
    for v in range(4):
        gate.step(v, 1.0)
    gate.step(0, 0.5)
    assert gate.calibrated and gate.n_w == 0 and gate.rho_min == 0.5


def test_nonfinite_loss_leaves_state():
    cfg = GateConfig(W=2, n_views=2)
    gate = Gate(cfg)
    gate.step(0, 1.0)
    before = gate.state()
    assert gate.decide(0, float("nan")) == 0
    gate.update(0, float("inf"))
    assert gate.state() == before and gate.errors == 1


def test_no_budget_ablation_only_skip_test():
    """rho_lo < 0 (Table 4 ablation): after warmup g is the bare skip test."""
    cfg = GateConfig(W=2, beta=0.5, eps=0.0, rho_lo=-1.0, n_views=1)
    gate = Gate(cfg)
    gs = [gate.step(0, L) for L in [1.0, 0.9, 0.8, 0.7, 0.6, 0.5, 0.4, 0.3]]
    assert gs == [1, 1, 0, 0, 0, 0, 0, 0]


def test_exhaustive_tiny_orderings():
    """Brute force: every ordering of 6 distinct losses over 2 views and every
    view pattern; the budget invariant and warmup rule hold in each."""
    losses = [0.5, 0.7, 0.9, 1.1, 1.3, 1.5]
    cfg = GateConfig(W=2, beta=0.5, eps=1e-8, rho_lo=0.5, n_views=2)
    for perm in itertools.permutations(losses):
        for pattern in range(0, 64, 7):
            views = [(pattern >> i) & 1 for i in range(6)]
            gate, gs, bs, _ = _run(cfg, views, perm)
            assert gs[:2].all()
            for t in range(1, 7):
                assert bs[t - 1] >= gate.rho_min * t - 1 - 1e-12


def test_batch_reading_equals_sequential_for_distinct_views():
    """Reading (vii): a launch's losses are decided against the EMA from before
    the launch; with distinct views in each launch that is the sequential
    algorithm exactly."""
    rng = np.random.default_rng(5)
    cfg = GateConfig(W=6, beta=0.9, eps=1e-8, rho_lo=0.5, n_views=8)
    seq_gate, batch_gate = Gate(cfg), Gate(cfg)
    for _ in range(60):
        views = rng.permutation(8)[:4]
        losses = rng.uniform(0.1, 1.0, 4)
        g_seq = [seq_gate.step(int(v), float(L)) for v, L in zip(views, losses)]
        g_bat = batch_gate.decide_batch(views, losses)
        batch_gate.update_batch(views, losses)
        assert g_seq == g_bat
    assert seq_gate.state() == batch_gate.state()
