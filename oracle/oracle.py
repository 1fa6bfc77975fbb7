"""ctypes wrapper around the C oracle (test infrastructure only).

Every function mirrors one C entry point in gpbo_oracle.c and works in float64
numpy arrays.  Nothing here imports the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build_oracle import build

_lib = None

_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_L = C.POINTER(C.c_int64)


def lib():
    global _lib
    if _lib is None:
        path = build()
        _lib = C.CDLL(path)
        L = _lib
        L.orc_splitmix64.restype = C.c_uint64
        L.orc_splitmix64.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
        L.orc_uniform24.restype = C.c_double
        L.orc_uniform24.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
        L.orc_normal.restype = C.c_double
        L.orc_normal.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
        L.orc_uniform_points.argtypes = [C.c_uint64, C.c_uint64, C.c_int64, C.c_int64, C.c_int, _D]
        L.orc_block_value.restype = C.c_double
        L.orc_block_value.argtypes = [C.c_int, _D, C.c_int]
        L.orc_objective.argtypes = [C.c_int, _I, _I, _D, _D, _D]
        L.orc_matern52.restype = C.c_double
        L.orc_matern52.argtypes = [C.c_double]
        L.orc_kmat.argtypes = [_D, C.c_int, C.c_int, _D, C.c_double, C.c_double, _D]
        L.orc_cholesky.restype = C.c_int
        L.orc_cholesky.argtypes = [_D, C.c_int, _D]
        L.orc_forward.argtypes = [_D, C.c_int, _D, _D]
        L.orc_backward_t.argtypes = [_D, C.c_int, _D, _D]
        L.orc_tri_inverse.argtypes = [_D, C.c_int, _D]
        L.orc_gp_fit.restype = C.c_int
        L.orc_gp_fit.argtypes = [_D, _D, C.c_int, C.c_int, _D, C.c_double, C.c_double, _D, _D, _D]
        L.orc_posterior.argtypes = [_D, C.c_int, C.c_int, _D, C.c_double, _D, _D, _D, C.c_int64, _D, _D]
        L.orc_ei.restype = C.c_double
        L.orc_ei.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double]
        L.orc_ei_batch.argtypes = [_D, _D, C.c_int64, C.c_double, C.c_double, _D]
        L.orc_argmax.restype = C.c_int64
        L.orc_argmax.argtypes = [_D, C.c_int64]
        L.orc_standardize.argtypes = [_D, C.c_int, _D, _D, _D]
        L.orc_search_step.restype = C.c_int
        L.orc_search_step.argtypes = [_D, _D, C.c_int, C.c_int, _D, C.c_double, C.c_double, _D, C.c_int64,
                                      C.c_uint64, C.c_double, _D, _D, _L, _D, _D, _D]
        L.orc_screen_pairwise.restype = C.c_int
        L.orc_screen_pairwise.argtypes = [C.c_int, _I, _I, C.c_double, C.c_uint64, C.c_int, C.c_int,
                                          C.c_double, _D, _D]
        L.orc_screen_routine.restype = C.c_int
        L.orc_screen_routine.argtypes = [C.c_int, _I, _I, C.c_double, C.c_uint64, C.c_int, C.c_int,
                                         C.c_double, _D]
        L.orc_partition_pairwise.restype = C.c_int
        L.orc_partition_pairwise.argtypes = [_D, C.c_int, C.c_double, C.c_int, _D, _I, _I, _I]
        L.orc_partition_routine.restype = C.c_int
        L.orc_partition_routine.argtypes = [_D, C.c_int, C.c_int, _I, C.c_double, C.c_int, _I, _I, _I]
        if hasattr(L, "orc_mlp_forward"):
            _bind_mlp(L)
        if hasattr(L, "orc_lml_grad"):
            L.orc_lml_grad.restype = C.c_int
            L.orc_lml_grad.argtypes = [_D, _D, C.c_int, C.c_int, _D, C.c_double, C.c_double, _D, _D]
    return _lib


def _bind_mlp(L):
    L.orc_gelu.restype = C.c_double
    L.orc_gelu.argtypes = [C.c_double]
    L.orc_mlp_forward.argtypes = [_D, C.c_int, C.c_int, C.c_int] + [_D] * 10
    L.orc_mlp_ensemble.argtypes = [_D, C.c_int, _D, C.c_int, C.c_int, C.c_int, _D, C.c_double, C.c_double, _D, _D,
                                   _D]
    L.orc_mlp_backward.restype = C.c_double
    L.orc_mlp_backward.argtypes = [_D, C.c_int, C.c_int, C.c_int] + [_D] * 14


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_D)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_I)


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle status {code}")
        self.code = code


def _check(st):
    if st != 0:
        raise OracleError(st)


# ------------------------------------------------------------------ wrappers
def splitmix64(seed, stream, counter):
    return int(lib().orc_splitmix64(seed, stream, counter))


def uniform24(seed, stream, counter):
    return float(lib().orc_uniform24(seed, stream, counter))


def normal(seed, stream, counter):
    return float(lib().orc_normal(seed, stream, counter))


def uniform_points(seed, stream, count, d, first=0):
    out = np.empty((count, d))
    lib().orc_uniform_points(seed, stream, first, count, d, out.ctypes.data_as(_D))
    return out


def block_value(fn, x01):
    x, px = _d(x01)
    return float(lib().orc_block_value(fn, px, x.shape[-1]))


def objective(block_dim, block_fn, x):
    bd, pbd = _i(block_dim)
    bf, pbf = _i(block_fn)
    xx, px = _d(x)
    fr = np.empty(len(bd))
    ft = np.empty(1)
    lib().orc_objective(len(bd), pbd, pbf, px, fr.ctypes.data_as(_D), ft.ctypes.data_as(_D))
    return float(ft[0]), fr


def matern52(r):
    return float(lib().orc_matern52(float(r)))


def kmat(X, ls, s2, sn2):
    X, pX = _d(X)
    n, d = X.shape
    ls, pls = _d(np.broadcast_to(np.asarray(ls, dtype=np.float64), (d,)))
    K = np.empty((n, n))
    lib().orc_kmat(pX, n, d, pls, s2, sn2, K.ctypes.data_as(_D))
    return K


def cholesky(K):
    K, pK = _d(K)
    n = K.shape[0]
    Lm = np.empty((n, n))
    _check(lib().orc_cholesky(pK, n, Lm.ctypes.data_as(_D)))
    return Lm


def forward(Lm, b):
    Lm, pL = _d(Lm)
    b, pb = _d(b)
    x = np.empty_like(b)
    lib().orc_forward(pL, Lm.shape[0], pb, x.ctypes.data_as(_D))
    return x


def backward_t(Lm, b):
    Lm, pL = _d(Lm)
    b, pb = _d(b)
    x = np.empty_like(b)
    lib().orc_backward_t(pL, Lm.shape[0], pb, x.ctypes.data_as(_D))
    return x


def tri_inverse(Lm):
    Lm, pL = _d(Lm)
    n = Lm.shape[0]
    out = np.empty((n, n))
    lib().orc_tri_inverse(pL, n, out.ctypes.data_as(_D))
    return out


def gp_fit(X, y, ls, s2, sn2):
    X, pX = _d(X)
    y, py = _d(y)
    n, d = X.shape
    ls, pls = _d(np.broadcast_to(np.asarray(ls, dtype=np.float64), (d,)))
    K = np.empty((n, n))
    Lm = np.empty((n, n))
    alpha = np.empty(n)
    _check(lib().orc_gp_fit(pX, py, n, d, pls, s2, sn2, K.ctypes.data_as(_D), Lm.ctypes.data_as(_D),
                            alpha.ctypes.data_as(_D)))
    return K, Lm, alpha


def posterior(X, ls, s2, Lm, alpha, Xc):
    X, pX = _d(X)
    n, d = X.shape
    ls, pls = _d(np.broadcast_to(np.asarray(ls, dtype=np.float64), (d,)))
    Lm, pL = _d(Lm)
    alpha, pa = _d(alpha)
    Xc, pXc = _d(Xc)
    M = Xc.shape[0]
    mu = np.empty(M)
    sg = np.empty(M)
    lib().orc_posterior(pX, n, d, pls, s2, pL, pa, pXc, M, mu.ctypes.data_as(_D), sg.ctypes.data_as(_D))
    return mu, sg


def ei(mu, sigma, tau, xi=0.0):
    return float(lib().orc_ei(mu, sigma, tau, xi))


def ei_batch(mu, sigma, tau, xi=0.0):
    mu, pm = _d(mu)
    sg, ps = _d(sigma)
    out = np.empty_like(mu)
    lib().orc_ei_batch(pm, ps, mu.shape[0], tau, xi, out.ctypes.data_as(_D))
    return out


def argmax(v):
    v, pv = _d(v)
    return int(lib().orc_argmax(pv, v.shape[0]))


def standardize(y):
    y, py = _d(y)
    ys = np.empty_like(y)
    m = np.empty(1)
    s = np.empty(1)
    lib().orc_standardize(py, y.shape[0], ys.ctypes.data_as(_D), m.ctypes.data_as(_D), s.ctypes.data_as(_D))
    return ys, float(m[0]), float(s[0])


def search_step(X, y, ls, s2, sn2, M=None, seed=0, Xc=None, xi=0.0, want_arrays=False):
    X, pX = _d(X)
    y, py = _d(y)
    n, d = X.shape
    ls, pls = _d(np.broadcast_to(np.asarray(ls, dtype=np.float64), (d,)))
    if Xc is not None:
        Xc, pXc = _d(Xc)
        M = Xc.shape[0]
    else:
        pXc = C.cast(None, _D)
    x_next = np.empty(d)
    ei_max = np.empty(1)
    am = np.empty(1, dtype=np.int64)
    arrs = [np.empty(M) for _ in range(3)] if want_arrays else None
    ptrs = [a.ctypes.data_as(_D) for a in arrs] if want_arrays else [C.cast(None, _D)] * 3
    _check(lib().orc_search_step(pX, py, n, d, pls, s2, sn2, pXc, M, seed, xi, x_next.ctypes.data_as(_D),
                                 ei_max.ctypes.data_as(_D), am.ctypes.data_as(_L), *ptrs))
    out = {"x_next": x_next, "ei_max": float(ei_max[0]), "argmax": int(am[0])}
    if want_arrays:
        out.update(mu=arrs[0], sigma=arrs[1], ei=arrs[2])
    return out


def screen_pairwise(block_dim, block_fn, noise_sd, seed, n_base, h):
    bd, pbd = _i(block_dim)
    bf, pbf = _i(block_fn)
    d = int(bd.sum())
    score = np.empty((d, d))
    sens = np.empty(d)
    _check(lib().orc_screen_pairwise(len(bd), pbd, pbf, noise_sd, seed, d, n_base, h,
                                     score.ctypes.data_as(_D), sens.ctypes.data_as(_D)))
    return score, sens


def screen_routine(block_dim, block_fn, noise_sd, seed, n_base, h):
    bd, pbd = _i(block_dim)
    bf, pbf = _i(block_fn)
    d = int(bd.sum())
    S = np.empty((len(bd), d))
    _check(lib().orc_screen_routine(len(bd), pbd, pbf, noise_sd, seed, d, n_base, h, S.ctypes.data_as(_D)))
    return S


def partition_pairwise(score, cutoff, max_dims, influence):
    score, ps = _d(score)
    d = score.shape[0]
    infl, pi = _d(influence)
    g = np.empty(d, dtype=np.int32)
    ng = np.empty(1, dtype=np.int32)
    fx = np.empty(d, dtype=np.int32)
    _check(lib().orc_partition_pairwise(ps, d, cutoff, max_dims, pi, g.ctypes.data_as(_I),
                                        ng.ctypes.data_as(_I), fx.ctypes.data_as(_I)))
    return g, int(ng[0]), fx


def partition_routine(S, owner, cutoff, max_dims):
    S, pS = _d(S)
    R, d = S.shape
    ow, pow_ = _i(owner)
    g = np.empty(d, dtype=np.int32)
    ng = np.empty(1, dtype=np.int32)
    fx = np.empty(d, dtype=np.int32)
    _check(lib().orc_partition_routine(pS, R, d, pow_, cutoff, max_dims, g.ctypes.data_as(_I),
                                       ng.ctypes.data_as(_I), fx.ctypes.data_as(_I)))
    return g, int(ng[0]), fx


def block_owner(block_dim):
    return np.repeat(np.arange(len(block_dim)), block_dim).astype(np.int32)


# ------------------------------------------------------------------ MLP (pre-screen network)
def mlp_sizes(d, H):
    """(name, shape) of each parameter block in the flat layout W1, b1, W2, b2, W3, b3."""
    return [("W1", (d, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, 2)), ("b3", (2,))]


def mlp_count(d, H):
    return d * H + H + H * H + H + 2 * H + 2


def mlp_split(theta, d, H):
    out, o = [], 0
    for _, shp in mlp_sizes(d, H):
        k = int(np.prod(shp))
        out.append(np.ascontiguousarray(theta[o:o + k], dtype=np.float64))
        o += k
    return out


def gelu(z):
    return float(lib().orc_gelu(float(z)))


def mlp_forward(theta, X, d, H):
    X, pX = _d(X)
    B = X.shape[0]
    parts = mlp_split(np.asarray(theta, dtype=np.float64), d, H)
    o = np.empty((B, 2))
    nul = C.cast(None, _D)
    lib().orc_mlp_forward(pX, B, d, H, *[q.ctypes.data_as(_D) for q in parts], nul, nul, nul, o.ctypes.data_as(_D))
    return o


def mlp_grad(theta, X, T, d, H):
    """(loss, flat gradient) of L = 1/(2B) sum (o - t)^2."""
    X, pX = _d(X)
    T, pT = _d(T)
    B = X.shape[0]
    parts = mlp_split(np.asarray(theta, dtype=np.float64), d, H)
    grads = [np.empty_like(q) for q in parts]
    loss = np.empty(1)
    lib().orc_mlp_backward(pX, B, d, H, *[q.ctypes.data_as(_D) for q in parts], pT,
                           *[g.ctypes.data_as(_D) for g in grads], loss.ctypes.data_as(_D))
    return float(loss[0]), np.concatenate([g.ravel() for g in grads])


def mlp_ensemble(thetas, X, d, H, norm4=(0.0, 1.0, 0.0, 1.0), tau=0.0, xi=0.0):
    """(mu_bar, sigma_bar, ei) of the ensemble `thetas` (E x P) on the rows of X."""
    th, pth = _d(np.asarray(thetas, dtype=np.float64).reshape(-1))
    E = th.shape[0] // mlp_count(d, H)
    X, pX = _d(X)
    B = X.shape[0]
    nm, pn = _d(np.asarray(norm4, dtype=np.float64))
    mu, sg, ei_ = np.empty(B), np.empty(B), np.empty(B)
    lib().orc_mlp_ensemble(pth, E, pX, B, d, H, pn, float(tau), float(xi), mu.ctypes.data_as(_D),
                           sg.ctypes.data_as(_D), ei_.ctypes.data_as(_D))
    return mu, sg, ei_


# ------------------------------------------------------------------ GP marginal likelihood
def lml_grad(X, y, ls, s2, sn2):
    """(log marginal likelihood, gradient over (log l_1..log l_d, log s2, log sn2))."""
    X, pX = _d(X)
    y, py = _d(y)
    n, d = X.shape
    ls, pls = _d(np.broadcast_to(np.asarray(ls, dtype=np.float64), (d,)))
    lml = np.empty(1)
    g = np.empty(d + 2)
    _check(lib().orc_lml_grad(pX, py, n, d, pls, float(s2), float(sn2), lml.ctypes.data_as(_D), g.ctypes.data_as(_D)))
    return float(lml[0]), g


def lml_grad_dense(X, y, ls, s2, sn2, scales=False):
    """The same LML and gradient as lml_grad with library primitives as the steps (scipy's
    Cholesky and triangular solves, numpy's matrix products), for sizes where the C loops
    are too slow.  Returns (lml, grad, kappa1) where kappa1 = |K|_1 |K^-1|_1 >= cond_2(K).
    With scales=True also the sums of absolute terms that bound the effect of a relative
    perturbation of alpha and K^-1: (|y| |alpha| + sum |log L_ii| + n, and per component
    1/2 sum (|alpha_p alpha_q| + |K^-1_pq|) |dK_pq/dtheta_j|)."""
    import scipy.linalg
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n, d = X.shape
    ls = np.broadcast_to(np.asarray(ls, dtype=np.float64), (d,))
    Z = X / ls
    r2 = np.zeros((n, n))
    for k in range(d):
        t = Z[:, k][:, None] - Z[None, :, k]
        r2 += t * t
    r = np.sqrt(r2)
    e = np.exp(-np.sqrt(5.0) * r)
    m = (1.0 + np.sqrt(5.0) * r + (5.0 / 3.0) * r2) * e
    K = s2 * m + sn2 * np.eye(n)
    L = scipy.linalg.cholesky(K, lower=True)
    alpha = scipy.linalg.cho_solve((L, True), y)
    alpha = alpha + scipy.linalg.cho_solve((L, True), y - K @ alpha)
    lml = -0.5 * y @ alpha - np.log(np.diag(L)).sum() - 0.5 * n * np.log(2 * np.pi)
    Li = scipy.linalg.solve_triangular(L, np.eye(n), lower=True)
    Ki = Li.T @ Li
    W = np.outer(alpha, alpha) - Ki
    c = s2 * (5.0 / 3.0) * (1.0 + np.sqrt(5.0) * r) * e
    g = np.empty(d + 2)
    for k in range(d):
        t = Z[:, k][:, None] - Z[None, :, k]
        g[k] = 0.5 * np.sum(W * c * t * t)
    g[d] = 0.5 * np.sum(W * s2 * m)
    g[d + 1] = 0.5 * sn2 * np.trace(W)
    kappa1 = np.abs(K).sum(0).max() * np.abs(Ki).sum(0).max()
    if not scales:
        return float(lml), g, float(kappa1)
    Wa = np.abs(np.outer(alpha, alpha)) + np.abs(Ki)
    gs = np.empty(d + 2)
    for k in range(d):
        t = Z[:, k][:, None] - Z[None, :, k]
        gs[k] = 0.5 * np.sum(Wa * np.abs(c) * t * t)
    gs[d] = 0.5 * np.sum(Wa * s2 * m)
    gs[d + 1] = 0.5 * sn2 * np.trace(Wa)
    ls_ = np.linalg.norm(y) * np.linalg.norm(alpha) + np.abs(np.log(np.diag(L))).sum() + n
    return float(lml), g, float(kappa1), float(ls_), gs


# ------------------------------------------------------------------ a BO search
def bo_search(fn, x_init, budget, M, seed, ls, s2, sn2, xi=0.0):
    """One BO search with fixed hyperparameters (§III-A): evaluate the initial design, then at
    evaluation t take the EI argmax of search_step over the M candidates drawn from seed + t
    and evaluate it.  Returns (X, y, index of the smallest y)."""
    X = [np.asarray(u, dtype=np.float64) for u in np.atleast_2d(x_init)]
    y = [float(fn(u)) for u in X]
    for t in range(len(X), budget):
        r = search_step(np.array(X), np.array(y), ls, s2, sn2, M=M, seed=seed + t, xi=xi)
        X.append(r["x_next"])
        y.append(float(fn(r["x_next"])))
    y = np.array(y)
    return np.array(X), y, int(np.argmin(y))


# ------------------------------------------------------------------ the paper's sensitivity series
def series_points(u0, i, V, growth, lo, hi):
    """The V variations of parameter i from baseline u0 (§IV-B): the value in its own units
    grown by (1 + growth) once per variation, clamped to [lo, hi], back in [0, 1]."""
    out = np.tile(np.asarray(u0, dtype=np.float64), (V, 1))
    x = lo + (hi - lo) * float(u0[i])
    for v in range(V):
        x = x * (1.0 + growth)
        out[v, i] = (min(max(x, lo), hi) - lo) / (hi - lo)
    return out


def screen_routine_series(routines_fn, d, R, V, growth, seed, lo, hi, owner, cutoff, max_dims):
    """Routine sensitivity on the paper's schedule: baseline b = point 0 of stream 3; for each
    parameter i its V variations; S_gi = mean_v |(f_g(b) - f_g(variation)) / f_g(b)| (with
    1e-12 added to |f_g(b)|); a shared parameter (owner -1) goes to the routine it influences
    most; then the routine partition (links above the cut-off, merge, cap).
    routines_fn(u) -> R outputs for one configuration u in [0,1]^d."""
    lo = np.broadcast_to(np.asarray(lo, dtype=np.float64), (d,))
    hi = np.broadcast_to(np.asarray(hi, dtype=np.float64), (d,))
    u0 = uniform_points(seed, 3, 1, d)[0]  # counters 0 .. d-1 of stream 3
    f0 = np.asarray(routines_fn(u0), dtype=np.float64)
    S = np.zeros((R, d))
    for i in range(d):
        for u in series_points(u0, i, V, growth, lo[i], hi[i]):
            S[:, i] += np.abs((f0 - np.asarray(routines_fn(u), dtype=np.float64)) / (np.abs(f0) + 1e-12))
    S /= V
    own = np.array([int(np.argmax(S[:, i])) if o < 0 else int(o) for i, o in enumerate(owner)], dtype=np.int32)
    g, ng, fx = partition_routine(S, own, cutoff, max_dims)
    return S, g, ng, fx, own
