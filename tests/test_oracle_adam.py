"""Pin of the Adam oracle against torch.optim.Adam (FP64, one param group per
learning rate), including steps skipped by the gate (the step counter only
advances on executed steps)."""
import numpy as np
import torch

import synth
from oracle.adam import AdamConfig, adam_step, lr_vector, param_groups


def test_adam_vs_torch():
    scene, _ = synth.scene_tiny(7, seed=0, sh_degree=3)
    n, K = scene.n, scene.sh.shape[1]
    cfg = AdamConfig()
    lr = lr_vector(n, K, cfg)
    p0 = scene.flat().astype(np.float64)
    rng = np.random.default_rng(0)
    # torch: one parameter tensor per distinct lr, gathered by mask
    masks = {v: lr == v for v in np.unique(lr)}
    tparams = {v: torch.tensor(p0[mk].copy(), requires_grad=True) for v, mk in masks.items()}
    opt = torch.optim.Adam([{"params": [tp], "lr": float(v)} for v, tp in tparams.items()],
                           betas=(cfg.beta1, cfg.beta2), eps=cfg.eps, foreach=False)
    p, m, v, step = p0.copy(), np.zeros_like(p0), np.zeros_like(p0), 0
    gate = [1, 1, 0, 1, 0, 0, 1, 1]
    for it, g_on in enumerate(gate):
        g = rng.normal(size=p0.shape) * 10.0 ** rng.uniform(-6, 0, size=p0.shape)
        if not g_on:
            continue
        p, m, v, step = adam_step(p, g, m, v, step, lr, cfg)
        for val, tp in tparams.items():
            tp.grad = torch.tensor(g[masks[val]])
        opt.step()
    assert step == sum(gate)
    for val, tp in tparams.items():
        np.testing.assert_allclose(p[masks[val]], tp.detach().numpy(), rtol=1e-13, atol=1e-16)


def test_param_groups_layout():
    g = param_groups(5, 16)
    assert g["means"] == (0, 15) and g["quats"] == (30, 50) and g["opacity_logit"] == (50, 55)
    assert g["sh"] == (55, 55 + 240) and 55 + 240 == 59 * 5
