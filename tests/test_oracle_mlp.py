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


def test_ensemble_one_member_and_identical_members(orc):
    """One member: mu_bar, sigma_bar are that member's de-standardised outputs and ei is the
    textbook EI for minimisation; identical members: the spread term vanishes."""
    d, H, B = 3, 8, 6
    theta = _theta(d, H, 4)
    X = np.random.default_rng(5).random((B, d))
    nm = (0.3, 1.7, -0.4, 0.6)
    tau, xi = 0.2, 0.01
    o = orc.mlp_forward(theta, X, d, H)
    m1, s1 = o[:, 0] * nm[1] + nm[0], np.exp(o[:, 1] * nm[3] + nm[2])
    mu, sg, ei = orc.mlp_ensemble(theta[None, :], X, d, H, nm, tau, xi)
    assert np.allclose(mu, m1, rtol=1e-14, atol=1e-14) and np.allclose(sg, s1, rtol=1e-14)
    z = (tau - m1 - xi) / s1
    ref = (tau - m1 - xi) * scipy.stats.norm.cdf(z) + s1 * scipy.stats.norm.pdf(z)
    assert np.allclose(ei, ref, rtol=1e-12, atol=1e-15)
    mu3, sg3, _ = orc.mlp_ensemble(np.stack([theta] * 3), X, d, H, nm, tau, xi)
    assert np.allclose(mu3, m1, rtol=1e-13) and np.allclose(sg3, s1, rtol=1e-13)


def test_ensemble_two_members_mixture_variance(orc):
    """Equal-weight mixture of two members: var = (s1^2 + s2^2)/2 + ((m1 - m2)/2)^2."""
    d, H, B = 4, 8, 5
    ta, tb = _theta(d, H, 6), _theta(d, H, 7)
    X = np.random.default_rng(8).random((B, d))
    oa, ob = orc.mlp_forward(ta, X, d, H), orc.mlp_forward(tb, X, d, H)
    mu, sg, _ = orc.mlp_ensemble(np.stack([ta, tb]), X, d, H)
    ma, mb, sa, sb = oa[:, 0], ob[:, 0], np.exp(oa[:, 1]), np.exp(ob[:, 1])
    assert np.allclose(mu, (ma + mb) / 2, rtol=1e-13, atol=1e-15)
    assert np.allclose(sg ** 2, (sa ** 2 + sb ** 2) / 2 + ((ma - mb) / 2) ** 2, rtol=1e-12)


def test_f16_tolerance_detects_planted_mistakes(orc):
    """The tolerance the GPU parity tests use for the FP16 ensemble is tight enough to fail
    plausible kernel mistakes: each is planted in the oracle's parameters (W2 used
    transposed, b1 dropped, the two output columns of W3 swapped, one member left out) and
    must move mu_bar or sigma_bar beyond the tolerance for most candidates."""
    from tests._util import f16_ensemble_tol
    d, H, E, B = 20, 256, 3, 200
    rng = np.random.default_rng(9)
    th = []
    for _ in range(E):
        parts = [rng.uniform(-1, 1, (d, H)) * np.sqrt(6 / (d + H)), rng.normal(0, 0.2, H),
                 rng.uniform(-1, 1, (H, H)) * np.sqrt(6 / (2 * H)), rng.normal(0, 0.2, H),
                 rng.uniform(-1, 1, (H, 2)) * np.sqrt(6 / (H + 2)), rng.normal(0, 0.2, 2)]
        th.append(np.concatenate([p.ravel() for p in parts]))
    th = np.array(th)
    X = rng.random((B, d))
    nm, tau = (0.1, 1.3, -0.5, 0.7), 0.0
    rm, rs, _ = orc.mlp_ensemble(th, X, d, H, nm, tau)
    tm, ts, _ = f16_ensemble_tol(orc, th, X, d, H, nm, tau)
    oW2, ob1, oW3 = d * H + H, d * H, d * H + H + H * H + H

    def mutate(f):
        t = th.copy()
        for e in range(E):
            f(t[e])
        return t

    def tr_w2(t):
        t[oW2:oW2 + H * H] = t[oW2:oW2 + H * H].reshape(H, H).T.ravel()

    def no_b1(t):
        t[ob1:ob1 + H] = 0.0

    def swap_w3(t):
        t[oW3:oW3 + 2 * H] = t[oW3:oW3 + 2 * H].reshape(H, 2)[:, ::-1].ravel()

    cases = {"W2 transposed": mutate(tr_w2), "b1 dropped": mutate(no_b1), "W3 columns swapped": mutate(swap_w3),
             "member left out": th[:E - 1]}
    for name, t in cases.items():
        mm, ms, _ = orc.mlp_ensemble(t, X, d, H, nm, tau)
        caught = (np.abs(mm - rm) > tm) | (np.abs(ms - rs) > ts)
        assert caught.mean() > 0.9, f"{name}: only {caught.mean():.2f} of candidates outside the tolerance"


def test_f16_round_matches_torch():
    """The tolerance's FP16 emulation rounds FP32 values like torch's CPU float32 -> float16 cast."""
    import torch
    from tests._util import f16_round
    x = np.random.default_rng(10).normal(0, 3, 100000).astype(np.float32)
    x[:5] = [1.0 + 2 ** -11, 1.0 + 3 * 2 ** -11, -0.0, 65504.0, 2 ** -20]
    ref = torch.from_numpy(x).to(torch.float16).to(torch.float64).numpy()
    assert np.array_equal(f16_round(x), ref)
