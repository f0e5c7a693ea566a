"""Algorithm 1 (SkipGS post-densification backward gating), in Python floats.

Test infrastructure only.  Python floats are IEEE binary64 and every operation
below rounds once (no fused multiply-add), which is the arithmetic the CUDA
gate kernel pins with explicit round-to-nearest double intrinsics.

Readings where the paper is silent or the algorithm listing and the text differ:
  (i)   first observation of a view: EMA = L (beta * empty is undefined);
  (ii)  warmup records the skip test only when the view already has an EMA
        history (Sec. 3.3, Eq. rhohat; the listing records unconditionally);
  (iii) no recorded warmup iteration at calibration: rho_min stays rho_lo, its
        initial value in the listing;
  (iv)  s == 1 skips (strict test, Eq. gate); a budget tie
        rho_cum(t-1) == rho_min does not force (strict test, Eq. rhocum_check);
  (v)   an unseen view after warmup has s = +inf, so g = 1;
  (vi)  a non-finite loss: g = 0, the state is left untouched and the call
        reports an error;
  (vii) several views of one batched launch are decided one after another,
        each as its own iteration t, all against the EMA as it stood before the
        launch (their losses come from the same parameters); the EMA updates
        of the launch follow, in order.  decide_batch / update_batch.
  rho_lo < 0 selects the ablation without budget control (Table 4): the skip
  test alone decides after warmup.
"""
from __future__ import annotations

import math
from dataclasses import dataclass


@dataclass
class GateConfig:
    W: int = 500
    beta: float = 0.95
    eps: float = 1e-8
    rho_lo: float = 0.5
    n_views: int = 1


class Gate:
    def __init__(self, cfg: GateConfig):
        self.cfg = cfg
        self.ema = [0.0] * cfg.n_views
        self.hist = [False] * cfg.n_views
        self.t = 0           # iterations decided so far
        self.b = 0           # backward count
        self.n_w = 0         # warmup iterations with history (|T_W|)
        self.n_w1 = 0        # ... of which the skip test gave g = 1
        self.rho_min = cfg.rho_lo if cfg.rho_lo >= 0 else 0.0
        self.calibrated = False
        self.errors = 0

    def decide(self, v: int, L: float) -> int:
        """Deviation score, skip test, warmup recording, calibration, budget override."""
        cfg = self.cfg
        L = float(L)
        if not math.isfinite(L):
            self.errors += 1
            return 0
        self.t += 1
        t = self.t
        if self.hist[v]:
            s = L / (self.ema[v] + cfg.eps)    # Eq. (deviation)
            g = 1 if s > 1.0 else 0            # Eq. (gate)
        else:
            g = 1                              # s = +inf
        if t <= cfg.W:
            if self.hist[v]:                   # reading (ii)
                self.n_w += 1
                self.n_w1 += g
            g = 1
        else:
            if not self.calibrated:            # once, at t = W + 1: Eq. (rhohat), Eq. (rhomincalib)
                if cfg.rho_lo >= 0 and self.n_w > 0:
                    rho_hat = self.n_w1 / self.n_w
                    self.rho_min = cfg.rho_lo + (1.0 - cfg.rho_lo) * rho_hat
                self.calibrated = True
            if cfg.rho_lo >= 0:
                rho_cum = self.b / max(t - 1, 1)   # Eq. (rhocum) before iteration t
                if rho_cum < self.rho_min:         # Eq. (rhocum_check)
                    g = 1
        if g:
            self.b += 1
        return g

    def update(self, v: int, L: float) -> None:
        """Eq. (view-ema), unconditional after the decision."""
        L = float(L)
        if not math.isfinite(L):
            return
        if self.hist[v]:
            self.ema[v] = self.cfg.beta * self.ema[v] + (1.0 - self.cfg.beta) * L
        else:
            self.ema[v] = L
            self.hist[v] = True

    def decide_batch(self, views, losses) -> list:
        return [self.decide(int(v), float(L)) for v, L in zip(views, losses)]

    def update_batch(self, views, losses) -> None:
        for v, L in zip(views, losses):
            self.update(int(v), float(L))

    def step(self, v: int, L: float) -> int:
        g = self.decide(v, L)
        self.update(v, L)
        return g

    def state(self) -> dict:
        return dict(ema=list(self.ema), hist=list(self.hist), t=self.t, b=self.b, n_w=self.n_w,
                    n_w1=self.n_w1, rho_min=self.rho_min, calibrated=self.calibrated)
