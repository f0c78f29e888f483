"""Pins of the CPU MLP reference: finite differences of the FP64 form, the
bfloat16 rounding rule against torch's, and agreement of the mixed-precision
form with the FP64 one to bfloat16 accuracy."""
import numpy as np
import torch

from oracle import mlp
from workloads.mlp_init import mlp_init_params


def test_bf16_rounding_matches_torch():
    x = np.random.default_rng(1).normal(size=4096).astype(np.float32) * 10
    x[:4] = [1.0, -2.5, 3.0000002, 1e-30]
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), want)


def test_fp64_gradient_matches_finite_differences():
    rng = np.random.default_rng(7)
    p = mlp_init_params(3).astype(np.float64) * 0.5
    p[2048:2176] = rng.normal(size=128) * 0.1
    p[18560:18688] = rng.normal(size=128) * 0.1
    X = rng.normal(size=(24, 16))
    T = rng.normal(size=24)
    loss, g = mlp.loss_and_grad(p, X, T, use_bf16=False)
    idx = np.concatenate([rng.choice(2048, 12, replace=False), 2048 + rng.choice(128, 6, replace=False),
                          2176 + rng.choice(16384, 20, replace=False), 18560 + rng.choice(128, 6, replace=False),
                          18688 + rng.choice(128, 6, replace=False), [18816]])
    for i in idx:
        h = 1e-6
        pp = p.copy(); pp[i] += h
        pm = p.copy(); pm[i] -= h
        fd = (mlp.loss_and_grad(pp, X, T, False)[0] - mlp.loss_and_grad(pm, X, T, False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_bf16_form_close_to_fp64_form():
    rng = np.random.default_rng(9)
    p = mlp_init_params(5)
    X = rng.normal(size=(64, 16))
    T = rng.normal(size=64)
    l1, g1 = mlp.loss_and_grad(p, X, T, True)
    l2, g2 = mlp.loss_and_grad(p, X, T, False)
    assert abs(l1 - l2) < 0.05 * abs(l2)
    assert np.linalg.norm(g1 - g2) < 0.05 * np.linalg.norm(g2)
