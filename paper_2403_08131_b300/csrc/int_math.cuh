// FP64 elementary functions computed mostly on the integer pipe (on this part the FP64 pipe
// issues one warp instruction per 64 cycles per scheduler, the integer pipe about 32 times as
// many operations), for kernels whose FP64 work is the bound.
#pragma once

#include <cstdint>

namespace gpbo {

// 1/sqrt(p) for a positive normal double, mostly off the FP64 pipe: an FP32 seed (rsqrtf of p's
// leading 24 bits, in [1, 4) after moving an odd exponent into the mantissa), then two
// Newton-Raphson steps y <- y (3 - M y^2) / 2 in 64-bit fixed point on the integer pipe (M in
// Q62, y in Q63), rounded to 53 bits: within 0.51 ulp of 1 / sqrt(p) (checked on 6e6 arguments,
// with seed errors of +-3e-7, against long double).  Other p take the library rsqrt.
__device__ __forceinline__ double rsqrt_int(double p)
{
    const uint64_t b = (uint64_t)__double_as_longlong(p);
    const int E = (int)(b >> 52);
    if (E == 0 || E >= 2047) return rsqrt(p);
    const uint64_t f = b & 0x000fffffffffffffull;
    const int u = E - 1023, odd = u & 1, k = (u - odd) / 2;  // p = M 2^(2k), M in [1, 4)
    const uint64_t Mq = (f | 0x0010000000000000ull) << (10 + odd);
    const float yf = rsqrtf(__uint_as_float(((uint32_t)(127 + odd) << 23) | (uint32_t)(f >> 29)));
    const uint32_t yb = __float_as_uint(yf);  // y in (0.5, 1]
    uint64_t yq = (uint64_t)((yb & 0x7fffffu) | 0x800000u) << (40 - (127 - (int)(yb >> 23)));
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const uint64_t t = __umul64hi(Mq, __umul64hi(yq, yq));  // M y^2 in Q60
        const uint64_t e = 0x3000000000000000ull - t;          // 3 - M y^2 in Q60
        yq = (__umul64hi(yq, e) << 3) | ((yq * e) >> 61);      // y (3 - M y^2) / 2 in Q63
    }
    if (yq >= 0x8000000000000000ull) return __longlong_as_double((long long)((uint64_t)(1023 - k) << 52));
    uint64_t m = (yq >> 10) + ((yq >> 9) & 1);
    int ex = 1022 - k;
    if (m >> 53) {
        m >>= 1;
        ++ex;
    }
    return __longlong_as_double((long long)(((uint64_t)ex << 52) | (m & 0x000fffffffffffffull)));
}

// exp(-t) for t >= 0, mostly off the FP64 pipe.  x = t / ln2 in 128-bit fixed point (t as the
// integer t 2^63 below 1, t 2^52 above; C = 2^126 / ln2 in two words), x = n + f, and
// exp(-t) = 2^(1-f) 2^(-n-1) with 2^h = sum_k (h ln2)^k / k! (k <= 18, Horner in Q62 with h = 1 - f
// in Q63), rounded to 53 bits.  Constants from the definitions: ln2 = sum_k 1 / (k 2^k),
// EXP_C[k] = round((ln2)^k / k! 2^62).  Within 0.52 ulp of exp(-t) (checked on 4e6 arguments
// against long double); 0 from t >= 708 (below the normal range).  Meant for t >= 0: a NaN or
// negative t takes the library exp.
static __constant__ uint64_t EXP_C[19] = {
    0x4000000000000000ull, 0x2c5c85fdf473de6bull, 0x0f5fdeffc162c754ull, 0x038d611ae09417f1ull,
    0x009d955b7dd273b9ull, 0x0015d87fe78a6731ull, 0x0002861225f0d8f1ull, 0x00003ff97f8b1162ull,
    0x0000058b0088e972ull, 0x0000006d494f4e58ull, 0x00000007933d4563ull, 0x000000007a32b1cdull,
    0x00000000070ef594ull, 0x0000000000605865ull, 0x000000000004c526ull, 0x000000000000386eull,
    0x0000000000000272ull, 0x000000000000001aull, 0x0000000000000001ull,
};
__device__ __forceinline__ double exp_neg_int(double t)
{
    if (!(t > 0.0)) return t == 0.0 ? 1.0 : exp(-t);  // NaN stays NaN; t < 0 by the library
    if (t >= 708.0) return 0.0;
    const uint64_t b = (uint64_t)__double_as_longlong(t);
    const int E = (int)(b >> 52);
    const uint64_t m = (b & 0x000fffffffffffffull) | 0x0010000000000000ull;
    const int sc = t < 1.0 ? 63 : 52;  // T = t 2^sc < 2^63
    const int sh = E - 1075 + sc;
    const uint64_t T = sh >= 0 ? m << sh : (sh > -64 ? (m + (1ull << (-sh - 1))) >> (-sh) : 0ull);
    const uint64_t CHI = 0x5c551d94ae0bf85dull, CLO = 0xdf43ff68348e9f44ull;
    const uint64_t c = __umul64hi(T, CLO);
    const uint64_t slo = T * CHI + c;
    const uint64_t shi = __umul64hi(T, CHI) + (slo < c ? 1ull : 0ull);
    const int r = sc - 2;  // x = S / 2^(sc + 62)
    const int n = (int)(shi >> r);
    const uint64_t fq = (shi << (64 - r)) | (slo >> r);      // fraction of x, Q64
    const uint64_t h = 0x8000000000000000ull - (fq >> 1);    // 1 - f, Q63
    uint64_t p = EXP_C[18];
#pragma unroll
    for (int k = 17; k >= 0; --k) p = EXP_C[k] + ((__umul64hi(h, p) << 1) | ((h * p) >> 63));
    int ex = 1022 - n;  // 2^h = p 2^-62 in (1, 2]
    uint64_t mm = 0;
    if (p >= 0x8000000000000000ull) {
        ++ex;
    } else {
        mm = (p >> 10) + ((p >> 9) & 1);
        if (mm >> 53) {
            mm >>= 1;
            ++ex;
        }
        mm &= 0x000fffffffffffffull;
    }
    if (ex < 1) return 0.0;
    return __longlong_as_double((long long)(((uint64_t)ex << 52) | mm));
}

}  // namespace gpbo
