"""Pins of the FP64 MLP oracle (the learned pre-screen network)."""
import math

import numpy as np
import pytest
import scipy.stats


def test_gelu_is_x_times_normal_cdf(orc):
    for z in [-6.0, -2.5, -1.0, -1e-3, 0.0, 0.3, 1.0, 2.0, 7.5]:
        assert orc.gelu(z) == pytest.approx(z * scipy.stats.norm.cdf(z), rel=1e-14, abs=1e-300)


def _theta(d, H, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(0, 0.3, orc_count(d, H))


def orc_count(d, H):
    from oracle import oracle
    return oracle.mlp_count(d, H)


def test_forward_against_numpy(orc):
    d, H, B = 5, 16, 7
    theta = _theta(d, H, 0)
    X = np.random.default_rng(1).random((B, d))
    W1, b1, W2, b2, W3, b3 = [p.reshape(s) for p, (_, s) in zip(orc.mlp_split(theta, d, H), orc.mlp_sizes(d, H))]
    g = lambda z: z * scipy.stats.norm.cdf(z)
    ref = g(g(X @ W1 + b1) @ W2 + b2) @ W3 + b3
    assert np.allclose(orc.mlp_forward(theta, X, d, H), ref, rtol=1e-12, atol=1e-12)


def test_gradients_against_central_differences(orc):
    d, H, B = 4, 8, 5
    theta = _theta(d, H, 2)
    rng = np.random.default_rng(3)
    X, T = rng.random((B, d)), rng.normal(size=(B, 2))
    loss, grad = orc.mlp_grad(theta, X, T, d, H)
    o = orc.mlp_forward(theta, X, d, H)
    assert loss == pytest.approx(0.5 * np.sum((o - T) ** 2) / B, rel=1e-13)
    eps = 1e-6
    fd = np.empty_like(theta)
    for i in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fd[i] = (orc.mlp_grad(tp, X, T, d, H)[0] - orc.mlp_grad(tm, X, T, d, H)[0]) / (2 * eps)
    scale = np.abs(fd).max()
    assert np.max(np.abs(grad - fd)) <= 1e-6 * scale
