"""Pins of the FP64 oracle of the GP log marginal likelihood and its gradient over
theta = (log l_1..log l_d, log s2, log sn2) (the quantity maximised when the GP's
hyperparameters are fitted by type-II maximum likelihood, Sec. 2)."""
import math

import numpy as np
import pytest


def _data(n, d, seed):
    rng = np.random.default_rng(seed)
    X = rng.random((n, d))
    y = np.sin(5 * X[:, 0]) + (X[:, 1:] ** 2).sum(1) - 0.4 * X[:, 0] * X[:, -1] + 0.05 * rng.normal(size=n)
    return X, y - y.mean()


def _sklearn_lml(X, y, ls, s2, sn2):
    """scikit-learn's LML and its gradient, reordered to (log l, log s2, log sn2)."""
    from sklearn.gaussian_process import GaussianProcessRegressor
    from sklearn.gaussian_process.kernels import ConstantKernel, Matern, WhiteKernel
    k = ConstantKernel(s2) * Matern(ls, nu=2.5) + WhiteKernel(sn2)
    gp = GaussianProcessRegressor(k, alpha=0.0, optimizer=None, normalize_y=False).fit(X, y)
    lml, g = gp.log_marginal_likelihood(gp.kernel_.theta, eval_gradient=True)
    d = X.shape[1]
    # sklearn's theta order: log s2, log l_1..l_d, log sn2
    return lml, np.concatenate([g[1:1 + d], g[:1], g[1 + d:]])


@pytest.mark.parametrize("n,d,seed", [(25, 2, 0), (60, 4, 1), (120, 6, 2)])
def test_lml_and_gradient_against_sklearn(orc, n, d, seed):
    X, y = _data(n, d, seed)
    ls = np.linspace(0.25, 0.7, d)
    lml, g = orc.lml_grad(X, y, ls, 1.3, 2e-3)
    lml_s, g_s = _sklearn_lml(X, y, ls, 1.3, 2e-3)
    assert lml == pytest.approx(lml_s, rel=1e-10, abs=1e-9)
    assert np.allclose(g, g_s, rtol=1e-8, atol=1e-8 * np.abs(g_s).max())


def test_gradient_against_central_differences(orc):
    X, y = _data(40, 3, 3)
    th = np.log(np.array([0.3, 0.45, 0.6, 0.9, 5e-3]))

    def f(t):
        e = np.exp(t)
        return orc.lml_grad(X, y, e[:3], e[3], e[4])[0]

    _, g = orc.lml_grad(X, y, np.exp(th[:3]), np.exp(th[3]), np.exp(th[4]))
    h = 1e-5
    for j in range(5):
        dp = th.copy(); dp[j] += h
        dm = th.copy(); dm[j] -= h
        fd = (f(dp) - f(dm)) / (2 * h)
        assert fd == pytest.approx(g[j], rel=1e-6, abs=1e-6), j


def test_single_observation_closed_form(orc):
    """n = 1: y ~ N(0, s2 + sn2), so LML = -y^2/(2v) - log(v)/2 - log(2 pi)/2 with v = s2 + sn2;
    the lengthscales do not enter (zero gradient) and dLML/dlog s = s (y^2/v^2 - 1/v)/2."""
    X = np.array([[0.3, 0.8]])
    y = np.array([1.7])
    s2, sn2 = 0.9, 0.05
    v = s2 + sn2
    lml, g = orc.lml_grad(X, y, [0.4, 0.5], s2, sn2)
    assert lml == pytest.approx(-y[0] ** 2 / (2 * v) - 0.5 * math.log(v) - 0.5 * math.log(2 * math.pi), rel=1e-14)
    assert g[0] == 0.0 and g[1] == 0.0
    assert g[2] == pytest.approx(0.5 * s2 * (y[0] ** 2 / v ** 2 - 1 / v), rel=1e-13)
    assert g[3] == pytest.approx(0.5 * sn2 * (y[0] ** 2 / v ** 2 - 1 / v), rel=1e-13)


def test_far_apart_points_factor(orc):
    """Points far apart relative to the lengthscales give K = (s2 + sn2) I to within
    exp(-sqrt5 r): the LML is a sum of independent one-point terms."""
    X = np.array([[0.0], [50.0], [100.0]])
    y = np.array([0.5, -1.2, 2.0])
    s2, sn2 = 1.1, 0.1
    lml, g = orc.lml_grad(X, y, [0.5], s2, sn2)
    v = s2 + sn2
    ref = sum(-t * t / (2 * v) - 0.5 * math.log(v) - 0.5 * math.log(2 * math.pi) for t in y)
    assert lml == pytest.approx(ref, rel=1e-13)
    assert abs(g[0]) < 1e-30


def test_scale_equivariance(orc):
    """Multiplying y by c and both variances by c^2 shifts the LML by -n log c and leaves the
    gradient unchanged (the model is the same up to the units of y)."""
    X, y = _data(30, 3, 5)
    ls = [0.3, 0.5, 0.4]
    l1, g1 = orc.lml_grad(X, y, ls, 1.2, 3e-3)
    c = 3.5
    l2, g2 = orc.lml_grad(X, c * y, ls, 1.2 * c * c, 3e-3 * c * c)
    assert l2 == pytest.approx(l1 - 30 * math.log(c), rel=1e-11)
    assert np.allclose(g1, g2, rtol=1e-8, atol=1e-9)


def test_gradient_vanishes_at_scipy_optimum(orc):
    """The maximiser found by scipy's L-BFGS-B on the oracle's LML has a gradient that vanishes
    (relative to its size at the start) and matches scikit-learn's own optimiser's LML."""
    import scipy.optimize
    X, y = _data(50, 2, 6)

    def negf(t):
        e = np.exp(t)
        v, g = orc.lml_grad(X, y, e[:2], e[2], e[3])
        return -v, -g

    t0 = np.log([0.5, 0.5, 1.0, 1e-2])
    r = scipy.optimize.minimize(negf, t0, jac=True, method="L-BFGS-B",
                                bounds=[(-5, 3), (-5, 3), (-5, 5), (-14, 1)])
    g0 = np.abs(negf(t0)[1]).max()
    assert np.abs(r.jac).max() < 1e-4 * g0
    from sklearn.gaussian_process import GaussianProcessRegressor
    from sklearn.gaussian_process.kernels import ConstantKernel, Matern, WhiteKernel
    k = ConstantKernel(1.0, (math.exp(-5), math.exp(5))) * Matern([0.5, 0.5], (math.exp(-5), math.exp(3)), nu=2.5) \
        + WhiteKernel(1e-2, (math.exp(-14), math.exp(1)))
    gp = GaussianProcessRegressor(k, alpha=0.0, n_restarts_optimizer=0).fit(X, y)
    assert -r.fun == pytest.approx(gp.log_marginal_likelihood_value_, rel=1e-5, abs=1e-5)


@pytest.mark.parametrize("n,d,seed", [(1, 2, 7), (45, 3, 8), (130, 5, 9)])
def test_dense_form_equals_c_oracle(orc, n, d, seed):
    """The library-primitive form used at large sizes agrees with the C loops."""
    X, y = _data(n, d, seed) if n > 1 else (np.array([[0.2, 0.9]]), np.array([0.7]))
    ls = np.linspace(0.3, 0.8, d)
    l1, g1 = orc.lml_grad(X, y, ls, 0.8, 4e-3)
    l2, g2, kap = orc.lml_grad_dense(X, y, ls, 0.8, 4e-3)
    assert l2 == pytest.approx(l1, rel=1e-11, abs=1e-11)
    assert np.allclose(g2, g1, rtol=1e-9, atol=1e-9 * max(1.0, np.abs(g1).max()))
    assert kap >= 1.0 - 1e-12
