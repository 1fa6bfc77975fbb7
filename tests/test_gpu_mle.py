"""GPU log marginal likelihood, its gradient and the multi-start L-BFGS hyperparameter fit
against the FP64 oracle.

Tolerance (derived from the arithmetic): both sides compute alpha and K^-1 from an FP64
Cholesky, whose forward error is bounded by about n u kappa(K) relative to the quantity
(u = 2^-53; kappa bounded above by kappa_1 = |K|_1 |K^-1|_1).  A relative perturbation of that
size in alpha and K^-1 moves the LML by at most n u kappa times |y||alpha| + sum |log L_ii| + n
and gradient component j by at most n u kappa times 1/2 sum (|alpha_p alpha_q| + |K^-1_pq|)
|dK_pq/dtheta_j|; the bar allows that once for each side, plus 32 u for the roundings of each
term's own evaluation (sqrt, exp, the products) and the reordered sums, which do not grow
with kappa."""
import math

import numpy as np
import pytest

from paper_2403_08131_b300 import workloads as W

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


def _obs(n, d, seed, noise=0.0):
    X = W.uniform_points(seed, W.STREAM_OBS, n, d)
    obj = W.Objective([d], [W.FN_ACKLEY], noise, seed)
    y = obj(X)
    return X, (y - y.mean()) / (y.std() or 1.0)


def _check(orc, X, y, ls, s2, sn2, lml, g):
    n = X.shape[0]
    lo, go, kap, lscale, gscale = orc.lml_grad_dense(X, y, ls, s2, sn2, scales=True)
    bar = 2 * U64 * (n * kap + 32)
    assert abs(lml - lo) <= bar * lscale, (lml, lo, bar * lscale)
    err = np.abs(g - go)
    assert np.all(err <= bar * gscale + 1e-300), (err / gscale, bar)
    pos = gscale > 0                         # a constant dimension has gscale = err = 0
    return float(np.max(err[pos] / gscale[pos])) if pos.any() else 0.0, bar


@pytest.mark.parametrize("n,d", [(2, 3), (63, 4), (64, 5), (65, 6), (200, 20), (700, 8), (300, 64)])
def test_lml_and_gradient_match_oracle(ctx, orc, n, d):
    from tests._util import to_dev
    X, y = _obs(n, d, 3000 + n)
    ls = 1.3 * np.asarray(W.lengthscale_rule(d))
    lml, g = ctx.lml(to_dev(X), to_dev(y), ls, 0.9, 2e-3)
    _check(orc, X, y, ls, 0.9, 2e-3, lml, g)


@pytest.mark.parametrize("n,d,stretch", [(1600, 7, 1.0), (1530, 20, 1.0), (1560, 64, 1.0), (1600, 6, 3e4)])
def test_lml_fixed_point_distances_match_oracle(ctx, orc, n, d, stretch):
    """Models with n_pad >= 1536 take the pair terms' squared distances in fixed point (exact
    128-bit sums over the quantised scaled coordinates, as their kernel matrix does) and the
    gradient's per-dimension squares from coordinates quantised per dimension: n_pad 1600 takes
    K^-1 as FP64 tiles, 1536 (ragged, n = 1530) from the tensor cores, d = 64 the widest input;
    stretch gives dimension 2 a lengthscale 3e4 times the others', so its scaled coordinates
    sit 15 binary orders below the largest and its gradient component is checked against its
    own, much smaller scale."""
    from tests._util import to_dev
    X, y = _obs(n, d, 5000 + n, noise=0.01)
    ls = 1.1 * np.asarray(W.lengthscale_rule(d))
    ls[2] *= stretch
    lml, g = ctx.lml(to_dev(X), to_dev(y), ls, 0.8, 3e-3)
    _check(orc, X, y, ls, 0.8, 3e-3, lml, g)


def test_lml_fixed_point_constant_dimension_has_zero_gradient(ctx, orc):
    """A dimension on which every observation agrees: each (x_pk - x_qk)^2 is exactly zero, so
    its gradient component is exactly 0.0 on both sides (the per-dimension quantisation of a
    constant column gives equal integers); the other components stay within the bar."""
    from tests._util import to_dev
    n, d = 1600, 5
    X, y = _obs(n, d, 6100, noise=0.01)
    X[:, 3] = 0.37
    ls = W.lengthscale_rule(d)
    lml, g = ctx.lml(to_dev(X), to_dev(y), ls, 1.0, 2e-3)
    assert g[3] == 0.0
    _check(orc, X, y, ls, 1.0, 2e-3, lml, g)


@pytest.mark.parametrize("n", [300, 1600])
def test_lml_nan_coordinate_fails_like_the_fit(ctx, n):
    """A NaN coordinate fails the evaluation with the fit's error, whether the distances are
    FP64 (n = 300) or fixed point (n = 1600: the coordinate kernels write zeros instead of
    converting the NaN)."""
    from paper_2403_08131_b300 import gpbo
    from tests._util import to_dev
    X, y = _obs(n, 4, 6200 + n)
    X[n // 3, 1] = np.nan
    with pytest.raises(gpbo.GpboError) as e:
        ctx.lml(to_dev(X), to_dev(y), W.lengthscale_rule(4), 1.0, 1e-3)
    assert e.value.code == gpbo.GPBO_ENOTSPD
    X[n // 3, 1] = 0.5                      # the context stays usable
    lml, g = ctx.lml(to_dev(X), to_dev(y), W.lengthscale_rule(4), 1.0, 1e-3)
    assert np.isfinite(lml) and np.all(np.isfinite(g))


def test_lml_single_observation_closed_form(ctx):
    X = np.array([[0.25, 0.5, 0.75]])
    y = np.array([1.4])
    s2, sn2 = 1.2, 0.03
    v = s2 + sn2
    lml, g = ctx.lml(X, y, [0.3, 0.4, 0.5], s2, sn2)
    assert lml == pytest.approx(-y[0] ** 2 / (2 * v) - 0.5 * math.log(v) - 0.5 * math.log(2 * math.pi), rel=1e-14)
    assert np.all(g[:3] == 0.0)
    assert g[3] == pytest.approx(0.5 * s2 * (y[0] ** 2 / v ** 2 - 1 / v), rel=1e-13)
    assert g[4] == pytest.approx(0.5 * sn2 * (y[0] ** 2 / v ** 2 - 1 / v), rel=1e-13)


def test_lml_host_equals_device_and_is_deterministic(ctx):
    from tests._util import to_dev
    X, y = _obs(333, 7, 11)
    ls = W.lengthscale_rule(7)
    a = ctx.lml(X, y, ls, 1.0, 1e-3)
    b = ctx.lml(to_dev(X), to_dev(y), ls, 1.0, 1e-3)
    c = ctx.lml(to_dev(X), to_dev(y), ls, 1.0, 1e-3)
    assert a[0] == b[0] == c[0]
    assert np.array_equal(a[1], b[1]) and np.array_equal(b[1], c[1])


def test_lml_full_size_matches_oracle(ctx, orc):
    """The bench's hyperparameter workload: n = 4096 observations in d = 20."""
    from tests._util import to_dev
    n, d = 4096, 20
    X, y = _obs(n, d, 4242, noise=0.02)
    ls = W.lengthscale_rule(d)
    lml, g = ctx.lml(to_dev(X), to_dev(y), ls, 1.0, 1e-3)
    _check(orc, X, y, ls, 1.0, 1e-3, lml, g)


def test_lml_rejects_bad_arguments(ctx):
    from paper_2403_08131_b300 import gpbo
    X, y = _obs(10, 2, 1)
    with pytest.raises(gpbo.GpboError):
        ctx.lml(X, y, [0.3, 0.3], 1.0, 0.0)   # noise_var must be positive
    with pytest.raises(gpbo.GpboError):
        ctx.lml(X, y, [0.3, -0.3], 1.0, 1e-3)
    with pytest.raises(gpbo.GpboError):
        ctx.fit_mle(X, y, np.zeros((1, 4)), [1.0] * 4, [0.0] * 4)  # lo > hi
    with pytest.raises(gpbo.GpboError):
        ctx.fit_mle(X, y, np.zeros((0, 4)), -1.0, 1.0)


BOUNDS_LO = None


def _mle_problem():
    X, y = _obs(150, 3, 77, noise=0.1)
    lo = np.array([-4.0, -4.0, -4.0, -3.0, -12.0])
    hi = np.array([2.0, 2.0, 2.0, 3.0, 0.0])
    return X, y, lo, hi


def test_fit_mle_matches_scipy_lbfgsb_on_oracle(ctx, orc):
    import scipy.optimize
    X, y, lo, hi = _mle_problem()
    t0 = np.log([0.5, 0.5, 0.5, 1.0, 1e-2])
    th, lml, evals = ctx.fit_mle(X, y, t0[None, :], lo, hi, max_iter=200, gtol=1e-7)
    assert evals > 1

    def negf(t):
        e = np.exp(t)
        v, g = orc.lml_grad(X, y, e[:3], e[3], e[4])
        return -v, -g

    r = scipy.optimize.minimize(negf, t0, jac=True, method="L-BFGS-B", bounds=list(zip(lo, hi)),
                                options={"ftol": 1e-15, "gtol": 1e-9, "maxiter": 500})
    assert lml == pytest.approx(-r.fun, rel=1e-8, abs=1e-8)
    assert np.allclose(th, r.x, atol=2e-3), (th, r.x)
    assert np.all(th >= lo) and np.all(th <= hi)
    e = np.exp(th)
    _, g = ctx.lml(X, y, e[:3], e[3], e[4])
    free = (th > lo + 1e-9) & (th < hi - 1e-9)
    assert np.abs(g[free]).max() < 1e-4


def test_fit_mle_multistart_takes_the_best_start(ctx):
    X, y, lo, hi = _mle_problem()
    starts = np.array([[0.0, 0.0, 0.0, 0.0, -2.0],
                       [-3.0, 1.5, -1.0, 2.0, -10.0],
                       [1.5, -3.5, 1.0, -2.0, -6.0]])
    th, lml, ev = ctx.fit_mle(X, y, starts, lo, hi, max_iter=100)
    singles = [ctx.fit_mle(X, y, s[None, :], lo, hi, max_iter=100) for s in starts]
    best = max(range(3), key=lambda i: singles[i][1])
    assert lml == singles[best][1]
    assert np.array_equal(th, singles[best][0])
    assert ev == sum(s[2] for s in singles)


def test_fit_mle_stops_at_active_bounds(ctx):
    """With the box cut below the unconstrained optimum in the lengthscales, the fit ends on
    those bounds with the LML still rising outwards (projected gradient zero)."""
    X, y, lo, hi = _mle_problem()
    hi2 = hi.copy()
    hi2[:3] = -3.5  # far shorter lengthscales than the data support
    th, lml, _ = ctx.fit_mle(X, y, np.array([[-3.8, -3.8, -3.8, 0.0, -4.0]]), lo, hi2, max_iter=100)
    assert np.all(th[:3] == hi2[:3])
    e = np.exp(th)
    _, g = ctx.lml(X, y, e[:3], e[3], e[4])
    assert np.all(g[:3] > 0)
    assert np.abs(g[3:]).max() < 1e-3 * max(1.0, np.abs(g[:3]).max())


def test_lml_trace_phase(ctx):
    X, y = _obs(500, 6, 5)
    ctx.trace(True)
    ctx.lml(X, y, W.lengthscale_rule(6), 1.0, 1e-3)
    tr = ctx.trace_read()
    ctx.trace(False)
    flops = sum(2.0 * (p + 1) * (500 - p) for p in range(500))
    assert tr["lml"]["intervals"] == 1
    assert tr["lml"]["flops"] == flops
    assert tr["lml"]["ms"] > 0
