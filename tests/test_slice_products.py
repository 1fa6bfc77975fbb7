"""The arithmetic of the tensor-core trailing update, emulated exactly on the CPU, against
exact rational products (the error-free splitting of Ozaki, Ogita, Oishi and Rump 2012, as the
kernel applies it).

Each row of a Cholesky panel P (64 columns) is 2^(e-7) times 7 integer slices of at most 8
bits -- the balanced base-256 digits of X = round(x 2^(55-e)) (ties away from zero), taken from
the least significant end as the kernels take them from the bits of x; slice pairs with s + t <= 9 are multiplied exactly (integer sums below 2^23, as the FP32
accumulators hold them), the 8 levels are folded in int64 (hi: levels 2..5, lo: 6..9), combined
as hi 2^16 + floor(lo / 2^16), and turned into a double by truncation.  The test checks the
exactness conditions the kernel relies on and that the result is within 2^-52 * 64 *
max|P_r| max|P_c| of the exact product (the size of an FP64 dot product's own error bound)."""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2403_08131_b300 import workloads as W

SLICES, LEVEL_MAX = 7, 9


def _fixed(x, e, prec=55):
    """round(x 2^(prec - e)) as an exact integer, ties away from zero."""
    if x == 0.0:
        return 0
    m, ex = math.frexp(x)                      # |x| = mi 2^(ex - 53), mi a 53-bit integer
    mi = int(math.ldexp(abs(m), 53))
    sh = ex - 53 + prec - e
    X = mi << sh if sh >= 0 else ((mi + (1 << (-sh - 1))) >> -sh if sh > -64 else 0)
    return X if x > 0 else -X


def _digits(X):
    """X = sum_s d_s 256^(SLICES - 1 - s), balanced digits from the least significant end."""
    d = [0] * SLICES
    for s in range(SLICES - 1, 0, -1):
        q = (X + 128) >> 8                     # floor division, as the kernels' arithmetic shift
        d[s] = X - (q << 8)
        X = q
    d[0] = X
    return d


def _split(P):
    mx = np.abs(P).max(1)
    e = np.array([math.frexp(m)[1] if m > 0 else 0 for m in mx])  # m < 2^e
    out = [np.zeros(P.shape, dtype=np.int64) for _ in range(SLICES)]
    for i in range(P.shape[0]):
        for j in range(P.shape[1]):
            X = _fixed(float(P[i, j]), int(e[i]))
            assert abs(X) <= 2 ** 55
            for s, dv in enumerate(_digits(X)):
                assert (-128 <= dv <= 128) if s == 0 else (-128 <= dv <= 127)
                out[s][i, j] = dv
    return e, out


def _emulate(Pr, Pc, drop_level=None, lo_shift=16, exp_bias=0):
    er, sr = _split(Pr)
    ec, sc = _split(Pc)
    acc = {l: 0 for l in range(2, LEVEL_MAX + 1)}
    for s in range(1, SLICES + 1):
        for t in range(1, SLICES + 1):
            if s + t <= LEVEL_MAX and s + t != drop_level:
                acc[s + t] = acc[s + t] + sr[s - 1] @ sc[t - 1].T
    for l, v in acc.items():
        assert np.abs(v).max() < 2 ** 23, l          # exact in the FP32 accumulator
    hi = acc[2]
    for l in (3, 4, 5):
        hi = hi * 256 + acc[l]
    lo = acc[6]
    for l in (7, 8, 9):
        lo = lo * 256 + acc[l]
    assert np.abs(hi).max() < 2 ** 47 and np.abs(lo).max() < 2 ** 47
    C = hi * 65536 + (lo >> lo_shift)
    out = np.empty(C.shape)
    for i in range(C.shape[0]):
        for j in range(C.shape[1]):
            x = int(C[i, j])
            k = int(er[i] + ec[j] - 54 + exp_bias)
            # truncation toward zero to 53 significant bits, as the kernel builds the double
            if x == 0:
                out[i, j] = 0.0
                continue
            nb = abs(x).bit_length()
            keep = abs(x) >> max(nb - 53, 0) << max(nb - 53, 0)
            out[i, j] = math.ldexp(float(keep if x > 0 else -keep), k)
    return out


@pytest.mark.parametrize("kb", [0, 7, 20])
def test_slice_products_on_matern_cholesky_panels(orc, kb):
    w = W.config4(n=1536)
    K = orc.kmat(w.X, w.lengthscale, 1.0, w.noise_var)
    L = np.linalg.cholesky(K)
    P = L[(kb + 2) * 64:(kb + 4) * 64, kb * 64:(kb + 1) * 64]
    Q = L[(kb + 2) * 64:(kb + 3) * 64, kb * 64:(kb + 1) * 64]
    em = _emulate(P, Q)
    rows, cols = range(0, 128, 9), range(0, 64, 5)
    for i in rows:
        for j in cols:
            ex = sum(Fraction(a) * Fraction(b) for a, b in zip(P[i], Q[j]))
            bound = 2.0 ** -52 * 64 * np.abs(P[i]).max() * np.abs(Q[j]).max()
            assert abs(Fraction(em[i, j]) - ex) <= Fraction(bound), (i, j)


def test_slice_products_planted_mistakes_fail():
    """A dropped level, a wrong shift of lo, or an exponent off by one lands outside the bound."""
    rng = np.random.default_rng(3)
    P = rng.normal(size=(16, 64))
    Q = rng.normal(size=(8, 64))
    ex = np.array([[float(sum(Fraction(a) * Fraction(b) for a, b in zip(P[i], Q[j]))) for j in range(8)]
                   for i in range(16)])
    bound = 2.0 ** -52 * 64 * np.abs(P).max(1)[:, None] * np.abs(Q).max(1)[None, :]
    assert np.all(np.abs(_emulate(P, Q) - ex) <= bound)
    for kw in ({"drop_level": 5}, {"drop_level": 7}, {"lo_shift": 15}, {"exp_bias": 1}):
        assert np.any(np.abs(_emulate(P, Q, **kw) - ex) > bound), kw
