"""Pins of the density-control oracle (oracle/densify.py), independent of it:
a decision table worked by hand (tests/golden/densify_decisions.txt), split
offsets against scipy's rotation of the scaled noise, exact copies for keep
and clone, the output count and order, and the statistic against a direct
per-Gaussian loop."""
import os

import numpy as np
import pytest

from oracle import densify as D

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "densify_decisions.txt")


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if line:
            rows.append([float(x) for x in line.split()])
    return np.array(rows)


def test_decisions_match_hand_worked_table():
    t = _golden()
    cfg = D.DensifyConfig(grad_thr=0.25, log_size_thr=-2.0, logit_prune_thr=-5.0)
    act = D.decide(t[:, 0], t[:, 1].astype(np.int64), t[:, 2:5], t[:, 5], cfg)
    assert act.tolist() == t[:, 6].astype(int).tolist()


def test_accumulate_against_a_loop():
    rng = np.random.default_rng(0)
    n = 50
    acc, den = np.zeros(n), np.zeros(n, np.int64)
    want_a, want_d = np.zeros(n), np.zeros(n, np.int64)
    for _ in range(4):
        g = rng.normal(size=(n, 2))
        vis = rng.random(n) < 0.6
        acc, den = D.accumulate(acc, den, g, vis)
        for i in range(n):
            if vis[i]:
                want_a[i] += float(np.hypot(g[i, 0], g[i, 1]))
                want_d[i] += 1
    np.testing.assert_allclose(acc, want_a, rtol=1e-15)
    assert np.array_equal(den, want_d)


def _params(n, K=4, seed=1):
    rng = np.random.default_rng(seed)
    q = rng.normal(size=(n, 4))
    return {"means": rng.normal(size=(n, 3)), "log_scales": rng.normal(-3, 0.5, (n, 3)), "quats": q,
            "opacity_logit": rng.normal(size=n), "sh": rng.normal(size=(n, K, 3))}


def test_apply_counts_order_copies_and_moments():
    n = 7
    p = _params(n)
    m = {k: np.full_like(v, 0.5) for k, v in p.items()}
    v = {k: np.full_like(x, 0.25) for k, x in p.items()}
    act = np.array([D.KEEP, D.CLONE, D.PRUNE, D.SPLIT, D.KEEP, D.PRUNE, D.CLONE], np.uint8)
    z = np.random.default_rng(2).normal(size=(n, 2, 3))
    out, mo, vo = D.apply(p, m, v, act, z, D.DensifyConfig())
    assert D.output_count(act) == 1 + 2 + 0 + 2 + 1 + 0 + 2 == out["means"].shape[0]
    src = [0, 1, 1, 3, 3, 4, 6, 6]  # stable: each Gaussian's outputs in place
    kept_moments = [True, True, False, False, False, True, True, False]
    for j, (i, km) in enumerate(zip(src, kept_moments)):
        for g in D.GROUPS:
            if act[i] != D.SPLIT or g not in ("means", "log_scales"):
                assert np.array_equal(out[g][j], p[g][i]), (j, g)
            assert np.all(mo[g][j] == (0.5 if km else 0.0)) and np.all(vo[g][j] == (0.25 if km else 0.0))


def test_split_children_against_scipy_rotation():
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    n = 64
    p = _params(n, seed=3)
    z = np.random.default_rng(4).normal(size=(n, 2, 3))
    act = np.full(n, D.SPLIT, np.uint8)
    cfg = D.DensifyConfig()
    out, _, _ = D.apply(p, {k: np.zeros_like(x) for k, x in p.items()},
                        {k: np.zeros_like(x) for k, x in p.items()}, act, z, cfg)
    q = p["quats"]
    rot = Rot.from_quat(np.stack([q[:, 1], q[:, 2], q[:, 3], q[:, 0]], 1))  # scipy: (x, y, z, w)
    s = np.exp(p["log_scales"])
    for k in range(2):
        want = p["means"] + rot.apply(s * z[:, k])
        np.testing.assert_allclose(out["means"][k::2], want, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(np.exp(out["log_scales"][k::2]), s / 1.6, rtol=1e-12)


def test_split_of_axis_aligned_gaussian_is_scaled_noise():
    p = _params(3, seed=5)
    p["quats"] = np.tile([2.0, 0.0, 0.0, 0.0], (3, 1))  # identity after normalisation
    z = np.random.default_rng(6).normal(size=(3, 2, 3))
    out, _, _ = D.apply(p, {k: np.zeros_like(x) for k, x in p.items()},
                        {k: np.zeros_like(x) for k, x in p.items()}, np.full(3, D.SPLIT, np.uint8), z,
                        D.DensifyConfig())
    np.testing.assert_allclose(out["means"].reshape(3, 2, 3), p["means"][:, None] + np.exp(p["log_scales"])[:, None] * z,
                               rtol=1e-14, atol=1e-15)


def test_prune_everything_and_nothing():
    p = _params(5)
    z = np.zeros((5, 2, 3))
    zero = {k: np.zeros_like(x) for k, x in p.items()}
    out, _, _ = D.apply(p, zero, zero, np.full(5, D.PRUNE, np.uint8), z, D.DensifyConfig())
    assert out["means"].shape[0] == 0
    out, _, _ = D.apply(p, zero, zero, np.zeros(5, np.uint8), z, D.DensifyConfig())
    for g in D.GROUPS:
        assert np.array_equal(out[g], p[g])
