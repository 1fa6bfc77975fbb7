"""Pins of the FP64 oracle against things other than itself.

Each test checks one oracle function against a published value, a closed form,
an invariant, a library routine (numpy / scipy / scikit-learn) or brute force.
No test here needs a GPU or loads the CUDA library.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg
import scipy.special
import scipy.stats

from paper_2403_08131_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- RNG
def test_splitmix64_published_vectors(orc):
    # Stream 0 makes the oracle's key equal to the plain seed, so its counter-th
    # output is the generator's counter-th published output.
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "splitmix64.txt")) if not ln.startswith("#")]
    for row in rows:
        seed = int(row[0], 0)
        for c, want in enumerate(row[1:]):
            assert orc.splitmix64(seed, 0, c) == int(want, 0)
            assert int(W.splitmix64(seed, 0, c)) == int(want, 0)


def test_uniform_grid_and_streams(orc):
    u = orc.uniform_points(7, 2, 5000, 3)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all(u * (1 << 24) == np.floor(u * (1 << 24)))          # 24-bit grid
    assert np.array_equal(u, W.uniform_points(7, 2, 5000, 3))
    assert np.array_equal(u.astype(np.float32).astype(np.float64), u)  # exact in fp32
    # Kolmogorov-Smirnov against U(0,1)
    assert scipy.stats.kstest(u.ravel(), "uniform").pvalue > 1e-3
    # different streams differ
    assert not np.array_equal(u, orc.uniform_points(7, 3, 5000, 3))


def test_normal_is_standard_normal(orc):
    z = np.array([orc.normal(11, 4, c) for c in range(20000)])
    assert np.allclose(z[:50], W.normal(11, 4, np.arange(50)), rtol=0, atol=1e-15)
    assert scipy.stats.kstest(z, "norm").pvalue > 1e-3


# ---------------------------------------------------------------- objectives
def test_objective_closed_forms(orc):
    # the unit-box centre maps to z = 0: Ackley(0) = 0, Rastrigin(0) = 0
    assert abs(orc.block_value(W.FN_ACKLEY, np.full(4, 0.5))) < 1e-12
    assert abs(orc.block_value(W.FN_RASTRIGIN, np.full(4, 0.5))) < 1e-12
    # x = 0.75 maps to z = 1: Rosenbrock minimum
    assert orc.block_value(W.FN_ROSENBROCK, np.full(5, 0.75)) == 0.0
    # Ackley at z = (1,...,1): -20 exp(-0.2) - exp(1) + 20 + e = 20 - 20 exp(-0.2)
    x = np.full(3, (1.0 + 32.768) / 65.536)
    assert abs(orc.block_value(W.FN_ACKLEY, x) - (20.0 - 20.0 * math.exp(-0.2))) < 1e-9
    # Rastrigin at integer z: sum z^2 (cosine terms cancel the 10 per dim)
    zz = np.array([1.0, -2.0, 3.0])
    x = (zz + 5.12) / 10.24
    assert abs(orc.block_value(W.FN_RASTRIGIN, x) - np.sum(zz ** 2)) < 1e-9
    # Rosenbrock(0, 0) in z = 1; chained over 3 dims at z = (0,0,0) = 2
    assert abs(orc.block_value(W.FN_ROSENBROCK, np.full(2, 0.5)) - 1.0) < 1e-12
    assert abs(orc.block_value(W.FN_ROSENBROCK, np.full(3, 0.5)) - 2.0) < 1e-12


def test_objective_matches_input_generator(orc):
    obj = W.five_block_objective(1, noise_sd=0.0)
    X = W.uniform_points(3, 1, 50, 20)
    want = obj.routines(X)
    for p in range(50):
        ft, fr = orc.objective(obj.block_dim, obj.block_fn, X[p])
        assert np.allclose(fr, want[p], rtol=1e-13, atol=1e-12)
        assert abs(ft - want[p].sum()) < 1e-11


# ---------------------------------------------------------------- Matern / K
def _matern_bessel(r, nu=2.5):
    r = np.asarray(r, dtype=np.float64)
    t = math.sqrt(2 * nu) * r
    return 2 ** (1 - nu) / scipy.special.gamma(nu) * t ** nu * scipy.special.kv(nu, t)


def test_matern52_against_bessel_form(orc):
    assert orc.matern52(0.0) == 1.0
    assert abs(orc.matern52(1.0) - (1 + math.sqrt(5) + 5 / 3) * math.exp(-math.sqrt(5))) < 1e-15
    for r in [1e-3, 0.1, 0.5, 1.0, 2.0, 3.7, 10.0]:
        assert abs(orc.matern52(r) - _matern_bessel(r)) < 1e-12


def test_kmat_against_sklearn(orc):
    from sklearn.gaussian_process.kernels import Matern
    rng = np.random.default_rng(0)
    X = rng.random((30, 5))
    ls = np.array([0.3, 0.5, 0.7, 1.1, 0.2])
    K = orc.kmat(X, ls, 1.7, 1e-3)
    Ks = 1.7 * Matern(length_scale=ls, nu=2.5)(X) + 1e-3 * np.eye(30)
    assert np.allclose(K, Ks, rtol=1e-12, atol=1e-14)
    assert np.array_equal(K, K.T)
    assert np.all(np.diag(K) == 1.7 + 1e-3)


def test_kmat_spd_small(orc):
    rng = np.random.default_rng(1)
    for n in range(1, 7):
        X = rng.random((n, 3))
        K = orc.kmat(X, 0.4, 1.0, 1e-6)
        assert np.all(np.linalg.eigvalsh(K) > 0)
        orc.cholesky(K)   # succeeds


# ---------------------------------------------------------------- Cholesky / solves
def test_cholesky_2x2_closed_form(orc):
    a, b, c = 4.0, 2.0, 5.0
    Lm = orc.cholesky(np.array([[a, b], [b, c]]))
    assert np.allclose(Lm, [[math.sqrt(a), 0], [b / math.sqrt(a), math.sqrt(c - b * b / a)]], rtol=0, atol=1e-15)


def test_cholesky_against_numpy_and_residual(orc):
    rng = np.random.default_rng(2)
    for n in [1, 3, 17, 64]:
        X = rng.random((n, 4))
        K = orc.kmat(X, 0.3, 1.0, 1e-6)
        Lm = orc.cholesky(K)
        assert np.allclose(Lm, np.linalg.cholesky(K), rtol=1e-9, atol=1e-12)
        assert np.allclose(np.triu(Lm, 1), 0)
        eps = np.finfo(float).eps
        assert np.abs(Lm @ Lm.T - K).max() <= 4 * n * eps * np.abs(K).max()


def test_cholesky_rejects_non_spd(orc):
    with pytest.raises(Exception) as e:
        orc.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))
    assert getattr(e.value, "code", None) == 2


def test_triangular_solves_and_inverse(orc):
    rng = np.random.default_rng(3)
    X = rng.random((40, 3))
    Lm = orc.cholesky(orc.kmat(X, 0.5, 1.0, 1e-4))
    b = rng.standard_normal(40)
    assert np.allclose(orc.forward(Lm, b), scipy.linalg.solve_triangular(Lm, b, lower=True), rtol=1e-10)
    assert np.allclose(orc.backward_t(Lm, b), scipy.linalg.solve_triangular(Lm.T, b, lower=False), rtol=1e-10)
    Li = orc.tri_inverse(Lm)
    assert np.allclose(Li, np.linalg.inv(Lm), rtol=1e-8, atol=1e-10)
    assert np.allclose(np.triu(Li, 1), 0)


def test_fit_alpha_against_dense_solve(orc):
    w = W.config1()
    K, Lm, alpha = orc.gp_fit(w.X, w.y, w.lengthscale, 1.0, w.noise_var)
    ref = np.linalg.solve(K, w.y)
    assert np.abs(alpha - ref).max() <= 1e-6 * np.abs(ref).max()
    # the refined residual is at rounding level
    assert np.abs(w.y - K @ alpha).max() <= 1e-8 * np.abs(w.y).max()


# ---------------------------------------------------------------- posterior
def _sklearn_gp(X, y, ls, s2, sn2):
    from sklearn.gaussian_process import GaussianProcessRegressor
    from sklearn.gaussian_process.kernels import ConstantKernel, Matern
    k = ConstantKernel(s2, "fixed") * Matern(length_scale=ls, length_scale_bounds="fixed", nu=2.5)
    return GaussianProcessRegressor(kernel=k, alpha=sn2, optimizer=None, normalize_y=False).fit(X, y)


def test_posterior_against_sklearn(orc):
    rng = np.random.default_rng(4)
    X = rng.random((60, 4))
    y = np.sin(6 * X[:, 0]) + X[:, 1] ** 2 - X[:, 2] * X[:, 3]
    ls = np.array([0.3, 0.4, 0.5, 0.6])
    _, Lm, alpha = orc.gp_fit(X, y, ls, 1.3, 1e-4)
    Xc = rng.random((500, 4))
    mu, sg = orc.posterior(X, ls, 1.3, Lm, alpha, Xc)
    m2, s2 = _sklearn_gp(X, y, ls, 1.3, 1e-4).predict(Xc, return_std=True)
    assert np.allclose(mu, m2, rtol=1e-8, atol=1e-9)
    assert np.allclose(sg, s2, rtol=1e-6, atol=1e-7)


def test_posterior_residual_and_training_variance(orc):
    # P1: mu(x_i) = y_i - sn2 alpha_i.  P2: sigma^2(x_i) = sn2 (1 - sn2 (K^-1)_ii).
    rng = np.random.default_rng(5)
    X = rng.random((25, 3))
    y = rng.standard_normal(25)
    sn2 = 1e-2
    K, Lm, alpha = orc.gp_fit(X, y, 0.5, 1.0, sn2)
    mu, sg = orc.posterior(X, 0.5, 1.0, Lm, alpha, X)
    assert np.allclose(mu, y - sn2 * alpha, rtol=0, atol=1e-10)
    Kinv = np.linalg.inv(K)
    assert np.allclose(sg ** 2, sn2 * (1 - sn2 * np.diag(Kinv)), rtol=1e-6, atol=1e-12)
    assert np.all(sg ** 2 <= sn2 * (1 + 1e-9))


def test_posterior_interpolates_when_noise_free(orc):
    rng = np.random.default_rng(6)
    X = rng.random((20, 2))
    y = rng.standard_normal(20)
    _, Lm, alpha = orc.gp_fit(X, y, 0.3, 1.0, 1e-12)
    mu, sg = orc.posterior(X, 0.3, 1.0, Lm, alpha, X)
    assert np.allclose(mu, y, atol=1e-8)
    assert np.all(sg < 1e-4)


def test_posterior_single_observation_closed_form(orc):
    # P3: n = 1 -> mu = k y / (s2 + sn2), sigma^2 = s2 - k^2 / (s2 + sn2)
    X = np.array([[0.2, 0.7]])
    y = np.array([1.5])
    s2, sn2, ls = 2.0, 0.1, np.array([0.3, 0.6])
    _, Lm, alpha = orc.gp_fit(X, y, ls, s2, sn2)
    Xc = np.array([[0.25, 0.6], [0.9, 0.1], [0.2, 0.7]])
    mu, sg = orc.posterior(X, ls, s2, Lm, alpha, Xc)
    r = np.sqrt((((Xc - X) / ls) ** 2).sum(1))
    k = np.array([s2 * _matern_bessel(v) if v > 0 else s2 for v in r])
    assert np.allclose(mu, k * 1.5 / (s2 + sn2), rtol=1e-12)
    assert np.allclose(sg ** 2, s2 - k ** 2 / (s2 + sn2), rtol=1e-12)


def test_posterior_far_field(orc):
    # P4: tiny lengthscale -> every candidate is far: mu = 0, sigma^2 = s2
    rng = np.random.default_rng(7)
    X = rng.random((10, 3))
    _, Lm, alpha = orc.gp_fit(X, rng.standard_normal(10), 1e-4, 1.5, 1e-6)
    mu, sg = orc.posterior(X, 1e-4, 1.5, Lm, alpha, rng.random((20, 3)))
    assert np.all(mu == 0.0)
    assert np.allclose(sg ** 2, 1.5)


# ---------------------------------------------------------------- EI / argmax
def test_ei_closed_forms(orc):
    assert abs(orc.ei(0.3, 0.7, 0.3) - 0.7 / math.sqrt(2 * math.pi)) < 1e-15
    assert orc.ei(0.1, 0.0, 0.5) == pytest.approx(0.4, abs=1e-15)
    assert orc.ei(0.9, 0.0, 0.5) == 0.0
    assert orc.ei(0.1, 0.2, 0.5, xi=0.1) == pytest.approx(orc.ei(0.2, 0.2, 0.5), abs=1e-15)


@pytest.mark.parametrize("mu,sigma,tau", [(0.0, 1.0, 0.5), (1.2, 0.3, 0.4), (-2.0, 0.05, -1.9), (0.3, 2.0, -1.0)])
def test_ei_against_quadrature(orc, mu, sigma, tau):
    f = lambda y: max(tau - y, 0.0) * scipy.stats.norm.pdf(y, mu, sigma)
    q, _ = scipy.integrate.quad(f, mu - 12 * sigma, tau, epsabs=1e-14, epsrel=1e-12, limit=200) \
        if tau > mu - 12 * sigma else (0.0, 0.0)
    assert abs(orc.ei(mu, sigma, tau) - q) < 1e-10


def test_ei_monotone(orc):
    sig = np.linspace(0.01, 3, 50)
    e = [orc.ei(0.2, s, 0.0) for s in sig]
    assert np.all(np.diff(e) > 0)
    mus = np.linspace(-2, 2, 50)
    e = [orc.ei(m, 0.5, 0.0) for m in mus]
    assert np.all(np.diff(e) < 0)


def test_argmax_first_of_ties(orc):
    rng = np.random.default_rng(8)
    v = rng.random(4096)
    assert orc.argmax(v) == int(np.argmax(v))
    v[[10, 500, 4000]] = 2.0
    assert orc.argmax(v) == 10 == int(np.argmax(v))


def test_standardize(orc):
    y = np.array([3.0, 1.0, 4.0, 1.0, 5.0, 9.0])
    ys, m, s = orc.standardize(y)
    assert m == pytest.approx(np.mean(y)) and s == pytest.approx(np.std(y))
    assert abs(ys.mean()) < 1e-15 and abs(ys.std() - 1) < 1e-15
    ys, m, s = orc.standardize(np.full(4, 2.0))
    assert s == 1.0 and np.all(ys == 0)


def test_search_step_against_library_pipeline(orc):
    """Whole BO step vs numpy standardisation + scikit-learn GP + scipy EI."""
    w = W.config1()
    Xc = w.candidates(2048).astype(np.float64)
    out = orc.search_step(w.X, w.y, w.lengthscale, 1.0, w.noise_var, Xc=Xc, want_arrays=True)
    ys = (w.y - w.y.mean()) / w.y.std()
    mu, sd = _sklearn_gp(w.X, ys, w.lengthscale, 1.0, w.noise_var).predict(Xc, return_std=True)
    tau = ys.min()
    z = (tau - mu) / sd
    ei = (tau - mu) * scipy.stats.norm.cdf(z) + sd * scipy.stats.norm.pdf(z)
    assert np.allclose(out["mu"], mu, rtol=1e-6, atol=1e-7)
    assert np.allclose(out["ei"], ei, rtol=1e-5, atol=1e-8)
    srt = np.sort(ei)
    assert (srt[-1] - srt[-2]) / srt[-1] > 1e-4           # a clear winner
    assert out["argmax"] == int(np.argmax(ei))
    assert np.array_equal(out["x_next"], Xc[out["argmax"]])


def test_search_step_generates_seeded_candidates(orc):
    w = W.config1()
    a = orc.search_step(w.X, w.y, w.lengthscale, 1.0, w.noise_var, M=1024, seed=w.seed)
    b = orc.search_step(w.X, w.y, w.lengthscale, 1.0, w.noise_var, Xc=w.candidates(1024).astype(np.float64))
    assert a["argmax"] == b["argmax"] and a["ei_max"] == b["ei_max"]


# ---------------------------------------------------------------- screens
def test_pairwise_screen_separable_is_zero(orc):
    # Rastrigin is a sum of one-dimensional terms: every mixed difference vanishes.
    score, sens = orc.screen_pairwise([5], [W.FN_RASTRIGIN], 0.0, 3, 16, 0.1)
    assert np.abs(score).max() < 1e-10
    assert np.all(sens > 0)


def test_pairwise_screen_rosenbrock_closed_form(orc):
    # 2-D Rosenbrock f = 100 (z1 - z0^2)^2 + (1 - z0)^2 on z = -2 + 4x, step a = 4h in z.
    # Analytic differences (no finite differencing):
    #   mixed   D  = -200 a (2 a z0 + a^2)
    #   along 0 F0 = 100 ((z1 - (z0+a)^2)^2 - (z1 - z0^2)^2) + (1 - z0 - a)^2 - (1 - z0)^2
    #   along 1 F1 = 100 a (2 (z1 - z0^2) + a)
    h, n_base, seed = 0.1, 32, 5
    score, sens = orc.screen_pairwise([2], [W.FN_ROSENBROCK], 0.0, seed, n_base, h)
    b = 0.9 * W.uniform_points(seed, W.STREAM_BASE, n_base, 2)
    z0, z1 = -2 + 4 * b[:, 0], -2 + 4 * b[:, 1]
    a = 4 * h
    D = -200 * a * (2 * a * z0 + a * a)
    F0 = 100 * ((z1 - (z0 + a) ** 2) ** 2 - (z1 - z0 ** 2) ** 2) + (1 - z0 - a) ** 2 - (1 - z0) ** 2
    F1 = 100 * a * (2 * (z1 - z0 ** 2) + a)
    want = np.mean(np.abs(D)) / (np.mean(np.abs(F0) + np.abs(F1)) + 1e-12)
    assert score[0, 1] == pytest.approx(want, rel=1e-9)
    assert score[1, 0] == score[0, 1] and score[0, 0] == 0 and score[1, 1] == 0
    f0 = 100 * (z1 - z0 ** 2) ** 2 + (1 - z0) ** 2
    assert sens == pytest.approx([np.mean(np.abs(F0) / f0), np.mean(np.abs(F1) / f0)], rel=1e-9)


def test_pairwise_screen_recovers_planted_graph(orc):
    sw = W.screen_config2(noise_sd=0.0)
    o = sw.objective
    score, sens = orc.screen_pairwise(o.block_dim, o.block_fn, 0.0, sw.seed, sw.n_base, sw.h)
    g, ng, fixed = orc.partition_pairwise(score, sw.cutoff, sw.max_dims, sens)
    # Ackley blocks (0, 2, 4) are single groups; Rastrigin blocks (1, 3) split into singletons.
    want = np.arange(20)
    for b in (0, 2, 4):
        want[4 * b:4 * b + 4] = 4 * b
    assert np.array_equal(g, want)
    assert ng == 3 + 8
    assert not fixed.any()
    # cross-block scores are at rounding level
    blk = np.arange(20) // 4
    cross = score[blk[:, None] != blk[None, :]]
    assert cross.max() < 1e-9


def test_pairwise_screen_noise_margin(orc):
    sw = W.screen_config2(noise_sd=0.01)
    o = sw.objective
    score, sens = orc.screen_pairwise(o.block_dim, o.block_fn, 0.01, sw.seed, sw.n_base, sw.h)
    g, ng, _ = orc.partition_pairwise(score, sw.cutoff, sw.max_dims, sens)
    blk = np.arange(20) // 4
    ack = np.isin(blk, [0, 2, 4])
    inside = score[(blk[:, None] == blk[None, :]) & ack[:, None] & ~np.eye(20, dtype=bool)]
    outside = score[(blk[:, None] != blk[None, :]) | ~ack[:, None]]
    outside = outside[outside > 0]
    assert inside.min() / outside.max() > 2.0
    assert ng == 11


def test_routine_screen_cross_block_zero_and_recovery(orc):
    sw = W.screen_config2(noise_sd=0.0)
    o = sw.objective
    S = orc.screen_routine(o.block_dim, o.block_fn, 0.0, sw.seed, sw.n_base, sw.h)
    owner = orc.block_owner(o.block_dim)
    for gi in range(5):
        for i in range(20):
            if owner[i] != gi:
                assert S[gi, i] == 0.0
            else:
                assert S[gi, i] > 0.0
    g, ng, fixed = orc.partition_routine(S, owner, sw.cutoff_routine, sw.max_dims)
    assert ng == 5 and np.array_equal(g, 4 * owner)


def test_partition_union_find_labels_and_cap(orc):
    d = 14
    score = np.zeros((d, d))
    edges = [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 6), (6, 7), (7, 8), (8, 9), (9, 10), (10, 11), (12, 13)]
    for i, j in edges:
        score[i, j] = score[j, i] = 0.9
    infl = np.linspace(1.0, 0.1, d)
    infl[3] = 0.01          # the two weakest members of the 12-group
    infl[7] = 0.02
    g, ng, fixed = orc.partition_pairwise(score, 0.25, 10, infl)
    assert list(g) == [0] * 12 + [12, 12]
    assert ng == 2
    assert list(np.nonzero(fixed)[0]) == [3, 7]
    # edge exactly at the cut-off does not link (strict >)
    score2 = np.zeros((3, 3))
    score2[0, 1] = score2[1, 0] = 0.25
    g, ng, _ = orc.partition_pairwise(score2, 0.25, 10, np.ones(3))
    assert list(g) == [0, 1, 2] and ng == 3


def test_partition_routine_paper_case_study_1(orc):
    """Decision-level golden from the paper's RT-TDDFT Case Study 1 tables."""
    gd = json.load(open(os.path.join(GOLDEN, "rttddft_cs1_routine_sensitivity.json")))
    params, routines = gd["params"], gd["routines"]
    S = np.zeros((len(routines), len(params)))
    for r, name in enumerate(routines):
        for p, v in gd["variability_percent"][name].items():
            S[r, params.index(p)] = v / 100.0
    g, ng, fixed = orc.partition_routine(S, np.array(gd["owner"]), gd["cutoff"], gd["max_dims"])
    groups = {}
    for i, lab in enumerate(g):
        groups.setdefault(int(lab), []).append(params[i])
    assert sorted(map(sorted, groups.values())) == sorted(map(sorted, gd["expected_groups"]))
    assert sorted(params[i] for i in np.nonzero(fixed)[0]) == sorted(gd["expected_fixed"])
