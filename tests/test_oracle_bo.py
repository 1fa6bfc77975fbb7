"""Pins of the paper's synthetic objective (a black box of the input generator) and of the
oracle's BO driver."""
import math

import numpy as np
import pytest
import scipy.stats

from paper_2403_08131_b300 import workloads as W


def _u(x):
    return (np.asarray(x, dtype=np.float64) + 50.0) / 100.0


@pytest.mark.parametrize("case", [1, 2, 3, 4, 5])
def test_synthetic_closed_form_at_ones(case):
    """At x = 1 everywhere: every (x_i - x_{i+1}) term vanishes and cos(2 pi (x - 1)) = 1, so
    G1 = G2 = 50; G3 = 10 (Cases 1-3: five ones plus five ones) or 5 (Cases 4-5); G4 = 5."""
    f = W.PaperSynthetic(case)
    g = f.group_values(_u(np.ones(20)))
    g3 = 10.0 if case <= 3 else 5.0
    assert np.allclose(g, [50.0, 50.0, g3, 5.0], rtol=1e-12)
    assert f(_u(np.ones(20))[None, :])[0] == pytest.approx(2 * math.log(50) + math.log(g3) + math.log(5), rel=1e-13)


def test_synthetic_group_structure():
    """Each group depends only on its own variables, except that Group 3 also reads Group 4's;
    in Cases 4-5 x_u pairs with x_{u+5} only."""
    rng = np.random.default_rng(0)
    for case in range(1, 6):
        f = W.PaperSynthetic(case)
        x = rng.uniform(-50, 50, 20)
        g0 = f.group_values(_u(x))
        for i in range(20):
            x2 = x.copy()
            x2[i] += 0.37
            g = f.group_values(_u(x2))
            owner = i // 5
            changed = set(np.flatnonzero(g != g0))  # groups not reading x_i are recomputed bit for bit
            expect = {owner} | ({2} if owner == 3 else set())
            assert changed == expect, (case, i, changed)
    f = W.PaperSynthetic(4)
    x = np.full(20, 2.0)
    x[15] = 3.0   # pairs with x_10 only
    g = f.group_values(_u(x))[2]
    assert g == pytest.approx((2 * 3 ** 4) ** 2 + 4 * (2 * 2 ** 4) ** 2, rel=1e-13)
    f5 = W.PaperSynthetic(5)
    assert f5.group_values(_u(x))[2] == pytest.approx((2 * 3 ** 8) ** 2 + 4 * (2 * 2 ** 8) ** 2, rel=1e-13)


def test_synthetic_singular_point_and_log_floor():
    f = W.PaperSynthetic(3)
    x = np.ones(20)
    x[15] = 0.0
    g = f.group_values(_u(x))
    assert g[3] == pytest.approx(4.0 + 1e3, rel=1e-12)  # 1/x at |x| < 1e-3 taken at 1e-3
    x = np.ones(20)
    x[10:15] = 0.0
    x[15:20] = -1.0    # Case 2: sum x_u^2 + sum x_v = -5;  Case 1: 0 + 5 cos(-2 pi) = 5
    assert W.PaperSynthetic(2).group_values(_u(x))[2] == pytest.approx(-5.0, abs=1e-12)
    assert W.PaperSynthetic(2).routines(_u(x))[2] == pytest.approx(math.log(5.0), rel=1e-13)


def test_synthetic_noise_is_twelve_independent_draws():
    f0, f1 = W.PaperSynthetic(3, 0.0), W.PaperSynthetic(3, 0.5, seed=7)
    U = np.tile(_u(np.full(20, 2.0)), (20000, 1))
    d = f1.group_values(U) - f0.group_values(U)
    # G1, G2 carry five eps each (inside A_i), G3 and G4 one each
    assert np.allclose(d.std(0), 0.5 * np.sqrt([5, 5, 1, 1]), rtol=0.03)
    assert np.all(np.abs(d.mean(0)) < 0.03)
    assert scipy.stats.pearsonr(d[:, 0], d[:, 1])[0] < 0.03


def _sklearn_ei_argmax(X, y, cand, ls, s2, sn2):
    from sklearn.gaussian_process import GaussianProcessRegressor
    from sklearn.gaussian_process.kernels import ConstantKernel, Matern
    ys = (y - y.mean()) / (y.std() or 1.0)
    k = ConstantKernel(s2, "fixed") * Matern(length_scale=ls, length_scale_bounds="fixed", nu=2.5)
    gp = GaussianProcessRegressor(kernel=k, alpha=sn2, optimizer=None, normalize_y=False).fit(X, ys)
    mu, sd = gp.predict(cand, return_std=True)
    imp = ys.min() - mu
    z = np.where(sd > 0, imp / np.where(sd > 0, sd, 1), 0)
    ei = np.where(sd > 0, imp * scipy.stats.norm.cdf(z) + sd * scipy.stats.norm.pdf(z), np.maximum(imp, 0))
    return ei


def test_oracle_bo_follows_its_definition(orc):
    """The first points are the initial design; every later point is the EI argmax over the
    seeded candidates of its step, recomputed here with scikit-learn and scipy."""
    def fn(u):
        return float(np.sum((u - np.array([0.3, 0.7, 0.55])) ** 2) + 0.1 * np.sin(9 * u[0]))

    x_init = W.uniform_points(3, W.STREAM_BO_INIT, 5, 3)
    ls, s2, sn2, M, seed = W.lengthscale_rule(3), 1.0, 1e-4, 2048, 41
    X, y, b = orc.bo_search(fn, x_init, 14, M, seed, ls, s2, sn2)
    assert np.array_equal(X[:5], x_init)
    assert np.array_equal(y, [fn(u) for u in X]) and y[b] == y.min()
    for t in range(5, 14):
        cand = W.uniform_points(seed + t, W.STREAM_CAND, M, 3).astype(np.float32).astype(np.float64)
        ei = _sklearn_ei_argmax(X[:t], y[:t], cand, ls, s2, sn2)
        pick = int(np.flatnonzero((cand == X[t]).all(1))[0])
        assert ei[pick] >= ei.max() * (1 - 1e-9), (t, ei[pick], ei.max())


def test_oracle_bo_improves_on_its_initial_design(orc):
    def fn(u):
        return float(np.sum((u - 0.62) ** 2))

    x_init = W.uniform_points(5, W.STREAM_BO_INIT, 5, 2)
    X, y, b = orc.bo_search(fn, x_init, 25, 4096, 77, W.lengthscale_rule(2), 1.0, 1e-6)
    assert y[b] < 1e-3 < y[:5].min()
