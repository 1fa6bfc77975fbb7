"""The integer-pipe FP64 functions of the kernel matrix and the likelihood epilogue
(paper_2403_08131_b300/csrc/int_math.cuh), emulated exactly with Python integers.

exp(-t): x = t / ln2 in 128-bit fixed point, 2^h = e^(h ln2) by its Taylor series in Q62,
rounded to 53 bits.  1/sqrt(p): an FP32 seed and two Newton-Raphson steps in Q63.  The tests
re-derive the header's constants from their definitions (ln2 = sum 1 / (k 2^k); the series
coefficients (ln2)^k / k!; 2^126 / ln2), check the stated error bounds (0.52 and 0.51 ulp)
against 60-digit references, and check that planted mistakes fall outside them.  The kernel
matrix's fixed-point squared distances (k_kmat_fixed: coordinates quantised to 2^(e - 58),
exact 128-bit sums, one two-part rounding) are checked against exact rational distances.
These pins need no GPU."""
import math
import re
import struct
from decimal import Decimal, getcontext
from fractions import Fraction
from pathlib import Path

import numpy as np
import pytest

HEADER = Path(__file__).resolve().parents[1] / "paper_2403_08131_b300" / "csrc" / "int_math.cuh"
M64 = (1 << 64) - 1
getcontext().prec = 60


def _ln2():
    return sum(Fraction(1, k * 2 ** k) for k in range(1, 300))


def _header_constants():
    src = HEADER.read_text()
    chi = int(re.search(r"CHI = (0x[0-9a-f]+)ull", src).group(1), 16)
    clo = int(re.search(r"CLO = (0x[0-9a-f]+)ull", src).group(1), 16)
    body = re.search(r"EXP_C\[19\] = \{(.*?)\};", src, re.S).group(1)
    coef = [int(h, 16) for h in re.findall(r"0x([0-9a-f]+)ull", body)]
    return chi, clo, coef


def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _dbl(b):
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def _exp_neg(t, chi, clo, coef, shift=0):
    """Bit-for-bit model of exp_neg_int for t > 0 (shift plants a wrong fraction shift)."""
    if t >= 708.0:
        return 0.0
    b = _bits(t)
    E = b >> 52
    m = (b & ((1 << 52) - 1)) | (1 << 52)
    sc = 63 if t < 1.0 else 52
    sh = E - 1075 + sc
    T = (m << sh) if sh >= 0 else (((m + (1 << (-sh - 1))) >> -sh) if sh > -64 else 0)
    c = (T * clo) >> 64
    slo = (T * chi + c) & M64
    shi = ((T * chi) >> 64) + (1 if slo < c else 0)
    r = sc - 2 + shift
    n = shi >> r
    fq = ((shi << (64 - r)) | (slo >> r)) & M64
    h = (1 << 63) - (fq >> 1)
    p = coef[18]
    for k in range(17, -1, -1):
        p = coef[k] + ((h * p) >> 63)
    ex = 1022 - n
    if p >= 1 << 63:
        mm, ex = 0, ex + 1
    else:
        mm = (p >> 10) + ((p >> 9) & 1)
        if mm >> 53:
            mm >>= 1
            ex += 1
        mm &= (1 << 52) - 1
    return 0.0 if ex < 1 else _dbl((ex << 52) | mm)


def _rsqrt(p, seed_rel=0.0, steps=2):
    """Bit-for-bit model of rsqrt_int with an FP32 seed of relative error seed_rel."""
    b = _bits(p)
    E = b >> 52
    f = b & ((1 << 52) - 1)
    u = E - 1023
    odd = u & 1
    k = (u - odd) // 2
    Mq = (f | (1 << 52)) << (10 + odd)
    Mf = struct.unpack("<f", struct.pack("<I", ((127 + odd) << 23) | (f >> 29)))[0]
    yf = np.float32(np.float32(1.0) / np.sqrt(np.float32(Mf)) * np.float32(1.0 + seed_rel))
    yb = struct.unpack("<I", struct.pack("<f", float(yf)))[0]
    yq = ((yb & 0x7FFFFF) | 0x800000) << (40 - (127 - (yb >> 23)))
    for _ in range(steps):
        t = (Mq * ((yq * yq) >> 64)) >> 64
        e = (0x3000000000000000 - t) & M64
        yq = ((yq * e) >> 61) & M64
    if yq >= 1 << 63:
        return _dbl((1023 - k) << 52)
    m = (yq >> 10) + ((yq >> 9) & 1)
    ex = 1022 - k
    if m >> 53:
        m >>= 1
        ex += 1
    return _dbl((ex << 52) | (m & ((1 << 52) - 1)))


def _ulp_err(got, exact):
    ulp = 2.0 ** (math.frexp(float(exact))[1] - 53)
    return abs(Decimal(got) - exact) / Decimal(ulp)


def test_exp_constants_follow_from_their_definitions():
    ln2 = _ln2()
    chi, clo, coef = _header_constants()
    assert (chi << 64) | clo == round(Fraction(2 ** 126) / ln2)
    want, term = [], Fraction(1)
    for k in range(19):
        if k:
            term = term * ln2 / k
        want.append(round(term * 2 ** 62))
    assert coef == want


def test_exp_neg_within_its_bound():
    chi, clo, coef = _header_constants()
    rng = np.random.default_rng(5)
    ts = np.concatenate([rng.uniform(0, 700, 400), rng.uniform(0, 20, 400), np.ldexp(rng.uniform(0.5, 1, 200),
                         -rng.integers(1, 60, 200)), [1.0, 2.0, 0.5, 1e-300, math.nextafter(1.0, 0.0)]])
    worst = max(_ulp_err(_exp_neg(float(t), chi, clo, coef), (-Decimal(float(t))).exp()) for t in ts)
    assert worst <= Decimal("0.52"), worst


def test_rsqrt_within_its_bound_for_seed_errors():
    rng = np.random.default_rng(6)
    ps = np.ldexp(rng.uniform(1, 2, 300), rng.integers(-900, 900, 300))
    worst = Decimal(0)
    for seed_rel in (0.0, 3e-7, -3e-7):
        for p in ps:
            exact = 1 / Decimal(float(p)).sqrt()
            worst = max(worst, _ulp_err(_rsqrt(float(p), seed_rel), exact))
    assert worst <= Decimal("0.51"), worst


def test_planted_mistakes_fall_outside_the_bounds():
    chi, clo, coef = _header_constants()
    t = 3.7
    exact = (-Decimal(t)).exp()
    bad = list(coef)
    bad[3] += 1 << 20
    assert _ulp_err(_exp_neg(t, chi, clo, bad), exact) > 1
    assert _ulp_err(_exp_neg(t, chi ^ (1 << 40), clo, coef), exact) > 1
    assert _ulp_err(_exp_neg(t, chi, clo, coef, shift=1), exact) > 1
    assert _ulp_err(_rsqrt(7.25, 3e-7, steps=1), 1 / Decimal(7.25).sqrt()) > 1


def _fixed(x, e, prec=58):
    """round(x 2^(prec - e)) with ties away from zero, as the kernels take it from the bits of x."""
    if x == 0.0:
        return 0
    m, ex = math.frexp(x)
    mi = int(math.ldexp(abs(m), 53))
    sh = ex - 53 + prec - e
    X = mi << sh if sh >= 0 else ((mi + (1 << (-sh - 1))) >> -sh if sh > -64 else 0)
    return X if x > 0 else -X


def _r2_fixed(a, b, e, scale_bias=0):
    """Bit-for-bit model of k_kmat_fixed's squared distance between rows a and b."""
    S = sum((_fixed(x, e) - _fixed(y, e)) ** 2 for x, y in zip(a, b))
    hi, lo = S >> 64, S & M64
    return (float(hi) * 18446744073709551616.0 + float(lo)) * 2.0 ** (2 * (e - 58) + scale_bias)


def test_fixed_point_distances_within_their_bound():
    """Exact integer squares and sums, one two-part rounding: within 2 ulp of the exact distance
    of the quantised coordinates, which move by at most 2^(e - 59) each."""
    rng = np.random.default_rng(7)
    Xs = rng.uniform(-0.5, 0.5, (40, 20)) / rng.uniform(0.2, 2.0, 20)
    Xs[3] = Xs[4] + 1e-9 * rng.standard_normal(20)            # a near pair
    mx = np.abs(Xs).max()
    e = math.frexp(mx)[1]                                       # |x| < 2^e
    for i in range(40):
        for j in range(i):
            got = _r2_fixed(Xs[i], Xs[j], e)
            exact = sum((Fraction(x) - Fraction(y)) ** 2 for x, y in zip(Xs[i], Xs[j]))
            quant = sum(2 * abs(Fraction(x) - Fraction(y)) * Fraction(2) ** (e - 58) + Fraction(2) ** (2 * (e - 58))
                        for x, y in zip(Xs[i], Xs[j]))
            bound = Fraction(2) * Fraction(2) ** -52 * exact + quant
            assert abs(Fraction(got) - exact) <= bound, (i, j)
    # a wrong power of two in the scaling lands far outside
    assert abs(_r2_fixed(Xs[1], Xs[0], e, scale_bias=1) - float(sum((Fraction(x) - Fraction(y)) ** 2
               for x, y in zip(Xs[1], Xs[0])))) > 0.1 * float(sum((x - y) ** 2 for x, y in zip(Xs[1], Xs[0])))


def _sq_to_double(t, shift=11):
    """Bit-for-bit model of sq_to_double (mle.cu): t^2 for an exact integer t, its leading 64
    bits rounded to 53 with ties away from zero (shift plants a wrong mantissa shift)."""
    if t == 0:
        return 0.0
    a = abs(t)
    lz = 64 - a.bit_length()
    top = a << lz
    h = (top * top) >> 64
    ex = 1023 + 127 - 2 * lz
    if not h >> 63:
        h = ((h << 1) | (((top * top) & M64) >> 63)) & M64
        ex -= 1
    m = (h >> shift) + ((h >> (shift - 1)) & 1)
    if m >> 53:
        m >>= 1
        ex += 1
    return _dbl((ex << 52) | (m & ((1 << 52) - 1)))


def test_integer_square_within_half_an_ulp():
    """The likelihood gradient's (x_p - x_q)^2 from fixed-point differences |t| <= 2^59: within
    0.5 ulp of the exact square (rounding to nearest, the tie away from zero), on random
    magnitudes, powers of two and their neighbours, and values whose square sits at a tie."""
    rng = np.random.default_rng(8)
    ts = [int(v) for v in rng.integers(1, 1 << 59, 3000, dtype=np.int64)]
    ts += [int(rng.integers(1, 1 << int(b))) for b in rng.integers(1, 59, 2000)]
    ts += [(1 << k) + o for k in range(0, 59) for o in (-1, 0, 1) if (1 << k) + o > 0]
    ts += [(1 << 27) + 1, (1 << 40) + 3, -(1 << 33) - 7]     # squares wider than 53 bits
    worst = Fraction(0)
    for t in ts:
        got = Fraction(_sq_to_double(t))
        exact = Fraction(t * t)
        ulp = Fraction(2) ** ((t * t).bit_length() - 53)
        worst = max(worst, abs(got - exact) / ulp)
        assert abs(got - exact) <= ulp / 2, t
    assert _sq_to_double(-12345) == _sq_to_double(12345) == 12345.0 ** 2
    assert _sq_to_double(1) == 1.0 and _sq_to_double(1 << 59) == 2.0 ** 118
    # a mantissa taken one bit too low is off by a factor near 2
    t = (1 << 40) + 12345
    assert abs(_sq_to_double(t, shift=10) / (t * t) - 1) > 0.4
