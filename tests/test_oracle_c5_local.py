"""The oracle at the stress size (6M Gaussians SH3, 1920x1080): its window
evaluation (tests/crop_util.py) against central finite differences of the
same window evaluation, for sampled Gaussians under the window, all 59
coordinates each (h = 1e-3 on the loss L = <weights, window image>; the
mean denominators of a pixel loss are fixed, so the window loss is the
exact local part of the full-view loss).  Coordinates whose perturbation
changes a discrete decision (contribution set, order, clamps) are skipped."""
import numpy as np

import oracle
import synth
from tests import crop_util

RC = oracle.RasterConfig()
NAMES = ("means", "log_scales", "quats", "opacity_logit", "sh")


def test_window_gradients_match_finite_differences_at_6m():
    scene, cams = synth.case_c5()
    s64 = crop_util.widen(scene)
    cam = cams[1]
    x0, y0, w, h = 952, 530, 16, 12
    rng = np.random.default_rng(7)
    wts = rng.normal(size=(3, h, w))
    base = crop_util.window_pass(s64, cam, RC, x0, y0, w, h, weights=wts)
    idx = base["idx"]
    assert len(idx) > 1000
    sub = crop_util.subset(s64, idx)
    local = np.arange(len(idx))
    L0 = float((base["image"] * wts).sum())
    g = base["grads"]
    # sample Gaussians with a non-negligible effect on the window
    eff = np.abs(g["opacity_logit"])
    cand = np.nonzero(eff > 1e-3 * eff.max())[0]
    picks = rng.choice(cand, size=8, replace=False)
    hstep = 1e-3
    checked = skipped = 0
    for i in picks:
        for nm in NAMES:
            arr = getattr(sub, nm)
            per = arr[i].size
            for c in range(per):
                vals = []
                for sgn in (1.0, -1.0):
                    s = crop_util.subset(sub, local)
                    a = getattr(s, nm)
                    flat = a.reshape(len(idx), -1)
                    flat[i, c] += sgn * hstep
                    o = crop_util.window_pass(s, cam, RC, x0, y0, w, h, idx=local)
                    vals.append(o)
                if any(o["hash"] != base["hash"] or (o["flags"] != base["flags"]).any() for o in vals):
                    skipped += 1
                    continue
                fd = (float((vals[0]["image"] * wts).sum()) - float((vals[1]["image"] * wts).sum())) / (2 * hstep)
                an = g[nm].reshape(len(idx), -1)[i, c]
                floor = 1e-3 * np.abs(g[nm]).max()
                # h = 1e-3 central differences: truncation ~ h^2 f''' / 6
                assert abs(fd - an) <= 2e-3 * max(abs(an), floor), (nm, i, c, fd, an)
                checked += 1
    assert checked > 0.8 * (checked + skipped)
    assert L0 != 0.0
