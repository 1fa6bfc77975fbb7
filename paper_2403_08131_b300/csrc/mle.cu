// GP hyperparameters by type-II maximum likelihood: the log marginal likelihood of y under
// the Matern-5/2 ARD prior, its gradient over theta = (log l_1..log l_d, log s2, log sn2), and
// a multi-start bound-constrained L-BFGS on the host that drives it (§III-A: the surrogate is
// trained on the evaluated configurations; §IV-D: GP training is the O(N^3) part).
//
//   LML = -1/2 y^T alpha - sum_i log L_ii - n/2 log(2 pi)
//   dLML/dtheta_j = 1/2 sum_pq (alpha_p alpha_q - [K^-1]_pq) dK_pq/dtheta_j
// with K^-1 = L^-T L^-1 (Rasmussen & Williams 2006, eqs. 2.30 and 5.9).  The fit (K, L, alpha,
// L^-1) is the FP64 fit of gp_fit; one fused kernel forms each 64 x 64 tile of K^-1 and, without
// writing it out, folds it into the d + 2 gradient sums.

#include "int_math.cuh"
#include "tc_common.cuh"
#include "gpbo_internal.cuh"
#include "gpbo.h"

#include <cmath>
#include <new>
#include <vector>

namespace gpbo {

namespace {

constexpr int LT = 64;   // K^-1 tile
constexpr int LBK = 16;  // rows of L^-1 per step

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Largest |x_k / l_k| of each dimension as magnitude bits (dmax zeroed before).  n_pad is a
// multiple of 64, so a warp's 32 elements lie in one dimension.
__global__ void k_lml_dim_max(const double *__restrict__ Xs, int n_pad, int64_t count,
                              unsigned long long *__restrict__ dmax)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned long long m = t < count ? (unsigned long long)tcx::mag_bits(Xs[t]) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m && t < count) atomicMax(&dmax[t / n_pad], m);
}

// Fixed-point coordinates for the pair terms of models whose kernel matrix takes its squared
// distances in integers (n_pad >= 1536, k_kmat_fixed).  Qx = round(Xs 2^(58 - e)) with the
// fit's e (from the largest |x / l| over all dimensions), so each pair's r^2 is the one K was
// built from.  Qg = round(Xs 2^(58 - e_k)) with each dimension's own e_k, for the gradient's
// (x_pk - x_qk)^2: a dimension with a long lengthscale keeps its own 58 bits (its FP64
// coordinates carry 53).
__global__ void k_lml_fixed_coords(const double *__restrict__ Xs, const unsigned long long *__restrict__ xmax,
                                   const unsigned long long *__restrict__ dmax, int n_pad, int64_t count,
                                   long long *__restrict__ Qx, long long *__restrict__ Qg)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= count) return;
    const bool finite = *xmax < 0x7ff0000000000000ull;  // else the fit has failed already
    Qx[t] = finite ? tcx::fixed_of(Xs[t], tcx::exp_of_mag(*xmax), 58) : 0;
    Qg[t] = finite ? tcx::fixed_of(Xs[t], tcx::exp_of_mag(dmax[t / n_pad]), 58) : 0;
}

// t^2 as a double for an exact integer t, on the integer pipe: |t| normalised by its leading
// zeros, the leading 64 bits of its 128-bit square, 53 of them rounded to nearest with ties
// away from zero (the bits below the leading 64 are not looked at: a tie rounds up, so the
// result is within 0.5 ulp of t^2 either way).  |t| < 2^61, so the exponent (at most 121) is
// always normal.
__device__ __forceinline__ double sq_to_double(long long t)
{
    if (t == 0) return 0.0;
    const unsigned long long a = t < 0 ? 0ull - (unsigned long long)t : (unsigned long long)t;
    const int lz = __clzll((long long)a);
    const unsigned long long top = a << lz;  // [2^63, 2^64); a^2 = top^2 2^(-2 lz)
    unsigned long long h = __umul64hi(top, top);
    int ex = 1023 + 127 - 2 * lz;
    if (!(h >> 63)) {
        h = (h << 1) | ((top * top) >> 63);
        --ex;
    }
    unsigned long long m = (h >> 11) + ((h >> 10) & 1ull);
    if (m >> 53) {
        m >>= 1;
        ++ex;
    }
    return __longlong_as_double((long long)(((unsigned long long)ex << 52) | (m & 0x000FFFFFFFFFFFFFull)));
}

// The pair terms of one thread's 4 x 4 piece of a K^-1 tile (rows p0 + ty + 16 u, columns
// q0 + tx + 16 v), reduced over the CTA into part[j * ntiles + p] (see k_lml_pairs).  FIXED:
// the squared distances are exact 128-bit sums over the fixed-point coordinates Qx, rounded
// once (as in k_kmat_fixed, bit for bit), in two halves of 8 pairs to bound the registers.
template <bool FIXED>
__device__ __forceinline__ void lml_pair_epilogue(double (&acc)[4][4], const double *__restrict__ Xs,
                                                  const long long *__restrict__ Qx,
                                                  const unsigned long long *__restrict__ xmax,
                                                  const long long *__restrict__ Qg,
                                                  const unsigned long long *__restrict__ dmax,
                                                  const double *__restrict__ alpha, int n, int d, int n_pad,
                                                  double s2, double sn2, int ntiles, double *__restrict__ part, int p,
                                                  int p0, int q0, double (*red)[GPBO_MAX_D + 2])
{
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4, lane = tid & 31, warp = tid >> 5;
    double r2[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) r2[u][v] = 0.0;
    if constexpr (FIXED) {
        const int sh = 2 * (tcx::exp_of_mag(*xmax) - 58);
        const bool fast = sh > -1000 && sh < 1000;
        const double scale = fast ? ldexp(1.0, sh) : 0.0;
#pragma unroll
        for (int uh = 0; uh < 4; uh += 2) {
            unsigned long long lo[2][4], hi[2][4];
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) lo[u][v] = hi[u][v] = 0ull;
            for (int k = 0; k < d; ++k) {
                const long long *row = Qx + (int64_t)k * n_pad;
                long long qp[2], qq[4];
#pragma unroll
                for (int u = 0; u < 2; ++u) qp[u] = __ldg(row + p0 + ty + 16 * (uh + u));
#pragma unroll
                for (int v = 0; v < 4; ++v) qq[v] = __ldg(row + q0 + tx + 16 * v);
#pragma unroll
                for (int u = 0; u < 2; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const long long t = qp[u] - qq[v];
                        const unsigned long long a = (unsigned long long)(t < 0 ? -t : t);
                        const unsigned long long pl = a * a;
                        lo[u][v] += pl;
                        hi[u][v] += __umul64hi(a, a) + (lo[u][v] < pl ? 1ull : 0ull);
                    }
            }
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const double S = (double)hi[u][v] * 18446744073709551616.0 + (double)lo[u][v];
                    r2[uh + u][v] = fast ? S * scale : ldexp(S, sh);
                }
        }
    }
    for (int k = 0; !FIXED && k < d; ++k) {
        const double *row = Xs + (int64_t)k * n_pad;
        double xp[4], xq[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) { xp[u] = __ldg(row + p0 + ty + 16 * u); xq[u] = __ldg(row + q0 + tx + 16 * u); }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const double t = xp[u] - xq[v];
                r2[u][v] = fma(t, t, r2[u][v]);
            }
    }
    const double sq5 = 2.2360679774997896964;  // sqrt(5)
    double gs = 0.0, gn = 0.0;
    double ap[4], aq[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) { ap[u] = alpha[p0 + ty + 16 * u]; aq[u] = alpha[q0 + tx + 16 * u]; }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int pp = p0 + ty + 16 * u, qq = q0 + tx + 16 * v;
            const double G = ap[u] * aq[v] - acc[u][v];
            double w = 0.0;
            if (pp < n && qq < n) {
                if (pp == qq) {
                    gs += 0.5 * G * s2;
                    gn += 0.5 * G * sn2;
                } else if (pp > qq) {
                    // square root and exponential on the integer pipe (int_math.cuh): this
                    // epilogue is bound by the FP64 pipe
                    const double r = r2[u][v] > 0.0 ? r2[u][v] * rsqrt_int(r2[u][v]) : 0.0;
                    const double e = exp_neg_int(sq5 * r);
                    gs += G * s2 * (1.0 + sq5 * r + (5.0 / 3.0) * r2[u][v]) * e;
                    w = G * s2 * (5.0 / 3.0) * (1.0 + sq5 * r) * e;
                }
            }
            acc[u][v] = w;
        }
    for (int k = 0; k < d; ++k) {
        double g = 0.0;
        if constexpr (FIXED) {
            // (x_pk - x_qk)^2 2^(116 - 2 e_k) exactly from the per-dimension fixed-point
            // coordinates, rounded once on the integer pipe; 2^(2 e_k - 116) is applied to the
            // CTA's sum below
            const long long *row = Qg + (int64_t)k * n_pad;
            long long qp[4], qq[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) { qp[u] = __ldg(row + p0 + ty + 16 * u); qq[u] = __ldg(row + q0 + tx + 16 * u); }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) g = fma(acc[u][v], sq_to_double(qp[u] - qq[v]), g);
        } else {
            const double *row = Xs + (int64_t)k * n_pad;
            double xp[4], xq[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) { xp[u] = __ldg(row + p0 + ty + 16 * u); xq[u] = __ldg(row + q0 + tx + 16 * u); }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const double t = xp[u] - xq[v];
                    g = fma(acc[u][v], t * t, g);
                }
        }
        g = warp_sum(g);
        if (lane == 0) red[warp][k] = g;
    }
    gs = warp_sum(gs);
    gn = warp_sum(gn);
    if (lane == 0) {
        red[warp][d] = gs;
        red[warp][d + 1] = gn;
    }
    __syncthreads();
    if (tid < d + 2) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < 8; ++w) s += red[w][tid];
        if (FIXED && tid < d) s = ldexp(s, 2 * (tcx::exp_of_mag(dmax[tid]) - 58));
        part[(int64_t)tid * ntiles + p] = s;
    }
}

// One CTA per lower tile (I, J), J <= I, numbered p = I (I + 1) / 2 + J so that the tiles with
// the most rows of L^-1 to reduce start first.  S = [K^-1]_{I,J} = sum_{k >= 64 I} L^-1[k, I]^T
// L^-1[k, J] (L^-1 is lower triangular, so rows above block I are zero in both operands); each
// thread holds a 4 x 4 piece (rows ty + 16 u, columns tx + 16 v).  Rows k of both operands are
// contiguous 64-double segments, staged through two shared buffers (one barrier per step).
// Epilogue, for p > q both < n (weight 1 = 2 x 1/2 by symmetry) with t = (x_p - x_q) / l,
// r = |t|, e = exp(-sqrt5 r), G = alpha_p alpha_q - S_pq:
//   g_k   += G s2 (5/3)(1 + sqrt5 r) e t_k^2            (k < d)
//   g_d   += G s2 (1 + sqrt5 r + 5/3 r^2) e
// and for p = q < n (weight 1/2): g_d += G s2 / 2, g_{d+1} += G sn2 / 2.
// part[j * ntiles + p] receives the CTA's sum for component j (fixed order: deterministic).
template <bool FIXED>
__global__ void __launch_bounds__(256) k_lml_pairs(const double *__restrict__ Linv, const double *__restrict__ Xs,
                                                   const long long *__restrict__ Qx,
                                                   const unsigned long long *__restrict__ xmax,
                                                   const long long *__restrict__ Qg,
                                                   const unsigned long long *__restrict__ dmax,
                                                   const double *__restrict__ alpha, int n, int d, int n_pad, int kend,
                                                   double s2, double sn2, int ntiles, double *__restrict__ part)
{
    __shared__ __align__(16) double As[2][LBK][LT];
    __shared__ __align__(16) double Bs[2][LBK][LT];
    __shared__ double red[8][GPBO_MAX_D + 2];
    const int p = blockIdx.x;
    int I = (int)((sqrt(8.0 * (double)p + 1.0) - 1.0) * 0.5);
    while ((I + 1) * (I + 2) / 2 <= p) ++I;
    while (I * (I + 1) / 2 > p) --I;
    const int J = p - I * (I + 1) / 2;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int p0 = I * LT, q0 = J * LT;
    const int lr = tid >> 4, lc = (tid & 15) * 4;

    double acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;

    double2 ra0, ra1, rb0, rb1;
    {
        const double *a = Linv + (int64_t)(p0 + lr) * n_pad + p0 + lc;
        const double *b = Linv + (int64_t)(p0 + lr) * n_pad + q0 + lc;
        ra0 = *reinterpret_cast<const double2 *>(a);
        ra1 = *reinterpret_cast<const double2 *>(a + 2);
        rb0 = *reinterpret_cast<const double2 *>(b);
        rb1 = *reinterpret_cast<const double2 *>(b + 2);
    }
    int buf = 0;
    for (int k0 = p0; k0 < kend; k0 += LBK) {
        *reinterpret_cast<double2 *>(&As[buf][lr][lc]) = ra0;
        *reinterpret_cast<double2 *>(&As[buf][lr][lc + 2]) = ra1;
        *reinterpret_cast<double2 *>(&Bs[buf][lr][lc]) = rb0;
        *reinterpret_cast<double2 *>(&Bs[buf][lr][lc + 2]) = rb1;
        __syncthreads();
        if (k0 + LBK < kend) {
            const double *a = Linv + (int64_t)(k0 + LBK + lr) * n_pad + p0 + lc;
            const double *b = Linv + (int64_t)(k0 + LBK + lr) * n_pad + q0 + lc;
            ra0 = *reinterpret_cast<const double2 *>(a);
            ra1 = *reinterpret_cast<const double2 *>(a + 2);
            rb0 = *reinterpret_cast<const double2 *>(b);
            rb1 = *reinterpret_cast<const double2 *>(b + 2);
        }
#pragma unroll
        for (int t = 0; t < LBK; ++t) {
            double x[4], y[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) { x[u] = As[buf][t][ty + 16 * u]; y[u] = Bs[buf][t][tx + 16 * u]; }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(x[u], y[v], acc[u][v]);
        }
        buf ^= 1;
    }

    lml_pair_epilogue<FIXED>(acc, Xs, Qx, xmax, Qg, dmax, alpha, n, d, n_pad, s2, sn2, ntiles, part, p, p0, q0, red);
}

// The same pair terms with K^-1 read from memory (the lower 64 x 64 tiles that kinv_tc forms
// on the tensor cores), tile p = I (I + 1) / 2 + J as in k_lml_pairs.
template <bool FIXED>
__global__ void __launch_bounds__(256) k_lml_pairs_kinv(const double *__restrict__ Kinv, const double *__restrict__ Xs,
                                                        const long long *__restrict__ Qx,
                                                        const unsigned long long *__restrict__ xmax,
                                                        const long long *__restrict__ Qg,
                                                        const unsigned long long *__restrict__ dmax,
                                                        const double *__restrict__ alpha, int n, int d, int n_pad,
                                                        double s2, double sn2, int ntiles, double *__restrict__ part)
{
    __shared__ double red[8][GPBO_MAX_D + 2];
    const int p = blockIdx.x;
    int I = (int)((sqrt(8.0 * (double)p + 1.0) - 1.0) * 0.5);
    while ((I + 1) * (I + 2) / 2 <= p) ++I;
    while (I * (I + 1) / 2 > p) --I;
    const int J = p - I * (I + 1) / 2;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int p0 = I * LT, q0 = J * LT;
    double acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = Kinv[(int64_t)(p0 + ty + 16 * u) * n_pad + q0 + tx + 16 * v];
    lml_pair_epilogue<FIXED>(acc, Xs, Qx, xmax, Qg, dmax, alpha, n, d, n_pad, s2, sn2, ntiles, part, p, p0, q0, red);
}

__device__ double block_sum256(double v, double *sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// out[0] = LML, out[1 + j] = dLML/dtheta_j (one CTA of 256 threads, fixed summation order).
__global__ void __launch_bounds__(256) k_lml_finish(const double *__restrict__ part, int ntiles, int nq,
                                                    const double *__restrict__ y, const double *__restrict__ alpha,
                                                    const double *__restrict__ L, int n, int n_pad,
                                                    double half_n_log2pi, double *__restrict__ out)
{
    __shared__ double sh[256];
    for (int j = 0; j < nq; ++j) {
        double s = 0.0;
        for (int t = threadIdx.x; t < ntiles; t += 256) s += part[(int64_t)j * ntiles + t];
        s = block_sum256(s, sh);
        if (threadIdx.x == 0) out[1 + j] = s;
    }
    double q = 0.0, ld = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) {
        q = fma(y[i], alpha[i], q);
        ld += log(L[(int64_t)i * n_pad + i]);
    }
    q = block_sum256(q, sh);
    ld = block_sum256(ld, sh);
    if (threadIdx.x == 0) out[0] = -0.5 * q - ld - half_n_log2pi;
}

}  // namespace

// Per-call state: an FP64 model of the problem's shape, refitted for each theta.
struct MleState {
    gpbo_ctx *ctx = nullptr;
    gp_model *m = nullptr;
    const double *X = nullptr, *y = nullptr;  // device
    double *part = nullptr;                    // (d + 2) x ntiles
    double *out = nullptr;                     // d + 3 (device)
    double *host = nullptr;                    // d + 3 (pinned)
    void *kslices = nullptr;                   // tensor-core K^-1 (n_pad a multiple of 128): slices,
    int *kexps = nullptr;                      //   their exponents
    double *kinv = nullptr;                    //   and K^-1's lower tiles
    long long *qx = nullptr;                   // fixed-point coordinates, 2 x d x n_pad (models with
    unsigned long long *dmax = nullptr;        //   xmax): common and per-dimension exponents; d maxima
    int ntiles = 0;
    int64_t evals = 0;
};

static void mle_release(MleState &s)
{
    if (s.part) cudaFree(s.part);
    if (s.out) cudaFree(s.out);
    if (s.host) cudaFreeHost(s.host);
    if (s.kslices) cudaFree(s.kslices);
    if (s.kexps) cudaFree(s.kexps);
    if (s.kinv) cudaFree(s.kinv);
    if (s.qx) cudaFree(s.qx);
    if (s.dmax) cudaFree(s.dmax);
    if (s.m) model_free(s.m);
    s.kslices = nullptr;
    s.kexps = nullptr;
    s.kinv = nullptr;
    s.qx = nullptr;
    s.dmax = nullptr;
    s.part = s.out = s.host = nullptr;
    s.m = nullptr;
}

static int mle_init(MleState &s, gpbo_ctx *ctx, const double *X, const double *y, int n, int d)
{
    s.ctx = ctx;
    s.X = X;
    s.y = y;
    GPBO_TRY(model_create(ctx, n, d, GPBO_PREC_F64, &s.m));
    const int nblk = s.m->n_pad / LT;
    s.ntiles = nblk * (nblk + 1) / 2;
    GPBO_CUDA_TRY(cudaMalloc(&s.part, sizeof(double) * (size_t)(d + 2) * s.ntiles));
    GPBO_CUDA_TRY(cudaMalloc(&s.out, sizeof(double) * (d + 3)));
    GPBO_CUDA_TRY(cudaMallocHost(&s.host, sizeof(double) * (d + 3)));
    const int n_pad = s.m->n_pad;
    if (s.m->xmax) {
        GPBO_CUDA_TRY(cudaMalloc(&s.qx, sizeof(long long) * 2 * (size_t)d * n_pad));
        GPBO_CUDA_TRY(cudaMalloc(&s.dmax, sizeof(unsigned long long) * d));
    }
    if (n_pad % 128 == 0 && n_pad >= 256) {
        GPBO_CUDA_TRY(cudaMalloc(&s.kslices, kinv_tc_slice_bytes(n_pad)));
        GPBO_CUDA_TRY(cudaMalloc(&s.kexps, sizeof(int) * n_pad));
        GPBO_CUDA_TRY(cudaMalloc(&s.kinv, sizeof(double) * (size_t)n_pad * n_pad));
    }
    return GPBO_OK;
}

// LML and gradient at theta (d + 2 log parameters); writes lml and grad (host).
static int mle_eval(MleState &s, const double *theta, double *lml, double *grad)
{
    gp_model *m = s.m;
    gpbo_ctx *ctx = s.ctx;
    const int n = m->n, d = m->d, n_pad = m->n_pad;
    for (int k = 0; k < d; ++k) m->ls[k] = std::exp(theta[k]);
    m->s2 = std::exp(theta[d]);
    m->sn2 = std::exp(theta[d + 1]);
    for (int k = 0; k < d + 2; ++k)
        if (!std::isfinite(theta[k])) return GPBO_EINVAL;
    if (!(m->s2 > 0) || !std::isfinite(m->s2) || !std::isfinite(m->sn2)) return GPBO_EINVAL;
    for (int k = 0; k < d; ++k)
        if (!(m->ls[k] > 0) || !std::isfinite(m->ls[k])) return GPBO_EINVAL;
    ++s.evals;
    const double nn = (double)n;
    GPBO_TRY(trace_begin(ctx, PH_FIT, nn * nn * nn / 3.0));
    GPBO_TRY(fit_model(ctx, m, s.X, s.y));
    GPBO_TRY(trace_end(ctx));
    const int kend = (int)round_up(n, LBK);
    // algorithmic flops: [K^-1]_pq for q <= p needs the n - p products of rows k >= p
    double flops = 0.0;
    for (int p = 0; p < n; ++p) flops += 2.0 * (double)(p + 1) * (double)(n - p);
    GPBO_TRY(trace_begin(ctx, PH_LML, flops));
    long long *qg = s.qx ? s.qx + (int64_t)d * n_pad : nullptr;
    if (s.qx) {
        const int64_t cnt = (int64_t)d * n_pad;
        const unsigned blocks = (unsigned)((cnt + 255) / 256);
        GPBO_CUDA_TRY(cudaMemsetAsync(s.dmax, 0, sizeof(unsigned long long) * d, ctx->stream));
        k_lml_dim_max<<<blocks, 256, 0, ctx->stream>>>(m->Xs64, n_pad, cnt, s.dmax);
        k_lml_fixed_coords<<<blocks, 256, 0, ctx->stream>>>(m->Xs64, m->xmax, s.dmax, n_pad, cnt, s.qx, qg);
    }
    if (s.kinv) {
        // K^-1 on the tensor cores (FP64 accuracy), then the pair terms from memory
        GPBO_TRY(kinv_tc(ctx, ctx->stream, m->Linv64, n_pad, s.kslices, s.kexps, s.kinv));
        auto k = s.qx ? k_lml_pairs_kinv<true> : k_lml_pairs_kinv<false>;
        k<<<s.ntiles, 256, 0, ctx->stream>>>(s.kinv, m->Xs64, s.qx, m->xmax, qg, s.dmax, m->alpha64, n, d, n_pad, m->s2, m->sn2,
                                             s.ntiles, s.part);
    } else {
        auto k = s.qx ? k_lml_pairs<true> : k_lml_pairs<false>;
        k<<<s.ntiles, 256, 0, ctx->stream>>>(m->Linv64, m->Xs64, s.qx, m->xmax, qg, s.dmax, m->alpha64, n, d, n_pad, kend, m->s2,
                                             m->sn2, s.ntiles, s.part);
    }
    GPBO_LAUNCH_CHECK(ctx);
    GPBO_TRY(trace_end(ctx));
    k_lml_finish<<<1, 256, 0, ctx->stream>>>(s.part, s.ntiles, d + 2, s.y, m->alpha64, m->L, n, n_pad,
                                             0.5 * nn * std::log(2.0 * 3.14159265358979323846), s.out);
    GPBO_LAUNCH_CHECK(ctx);
    GPBO_CUDA_TRY(cudaMemcpyAsync(s.host, s.out, sizeof(double) * (d + 3), cudaMemcpyDeviceToHost, ctx->stream));
    unsigned bits = 0;
    GPBO_TRY(take_device_status(ctx, &bits));  // synchronises the stream
    if (bits & DEV_NOTSPD) return GPBO_ENOTSPD;
    if (bits & DEV_TIMEOUT) return GPBO_ETIMEOUT;
    *lml = s.host[0];
    for (int j = 0; j < d + 2; ++j) grad[j] = s.host[1 + j];
    return GPBO_OK;
}

// ------------------------------------------------------------------ bound-constrained L-BFGS
// Minimises f = -LML over the box [lo, hi] (Nocedal & Wright 2006, Alg. 7.4 two-loop
// recursion) with a projected step: components at a bound whose gradient points out of the
// box are held fixed for the iteration; the trial point x + a p is projected onto the box and
// accepted on the Armijo condition f(x') <= f(x) + 1e-4 g^T (x' - x), halving a otherwise.  A
// factorisation that fails (K not positive definite at the trial point) counts as a rejected
// step.  Stops when the projected gradient's largest component is below gtol, when f changes
// by less than 1e-12 (1 + |f|) over an accepted step, or after max_iter iterations.
struct LbfgsResult {
    std::vector<double> x;
    double f = INFINITY;
    int iters = 0;
    int status = GPBO_OK;
};

static double proj_grad_norm(const std::vector<double> &x, const std::vector<double> &g, const double *lo,
                             const double *hi)
{
    double mx = 0.0;
    for (size_t i = 0; i < x.size(); ++i) {
        const double t = std::fmin(std::fmax(x[i] - g[i], lo[i]), hi[i]) - x[i];
        mx = std::fmax(mx, std::fabs(t));
    }
    return mx;
}

static LbfgsResult lbfgs_box(MleState &s, const double *x0, const double *lo, const double *hi, int max_iter,
                             double gtol)
{
    const int q = s.m->d + 2, mem = 10;
    LbfgsResult R;
    std::vector<double> x(q), g(q), xn(q), gn(q), p(q), a(mem), rho(mem);
    std::vector<std::vector<double>> S(mem, std::vector<double>(q)), Y(mem, std::vector<double>(q));
    int stored = 0, head = 0;
    for (int i = 0; i < q; ++i) x[i] = std::fmin(std::fmax(x0[i], lo[i]), hi[i]);
    auto eval = [&](const std::vector<double> &at, double &f, std::vector<double> &grad) -> int {
        double lml = 0.0;
        const int st = mle_eval(s, at.data(), &lml, grad.data());
        if (st == GPBO_ENOTSPD) {
            f = INFINITY;
            return GPBO_OK;
        }
        if (st != GPBO_OK) return st;
        f = -lml;
        for (int i = 0; i < q; ++i) grad[i] = -grad[i];
        return GPBO_OK;
    };
    double f = 0.0;
    R.status = eval(x, f, g);
    if (R.status != GPBO_OK) return R;
    if (!std::isfinite(f)) {
        R.status = GPBO_ENOTSPD;
        return R;
    }
    for (int it = 0; it < max_iter; ++it) {
        R.iters = it + 1;
        if (proj_grad_norm(x, g, lo, hi) <= gtol) break;
        std::vector<char> fixed(q, 0);
        for (int i = 0; i < q; ++i)
            fixed[i] = (x[i] <= lo[i] && g[i] > 0) || (x[i] >= hi[i] && g[i] < 0);
        // two-loop recursion on the free components
        for (int i = 0; i < q; ++i) p[i] = fixed[i] ? 0.0 : -g[i];
        for (int k = 0; k < stored; ++k) {
            const int j = (head - 1 - k + mem) % mem;
            double sp = 0.0;
            for (int i = 0; i < q; ++i) sp += S[j][i] * p[i];
            a[j] = rho[j] * sp;
            for (int i = 0; i < q; ++i) p[i] -= a[j] * Y[j][i];
        }
        if (stored > 0) {
            const int j = (head - 1 + mem) % mem;
            double sy = 0.0, yy = 0.0;
            for (int i = 0; i < q; ++i) { sy += S[j][i] * Y[j][i]; yy += Y[j][i] * Y[j][i]; }
            for (int i = 0; i < q; ++i) p[i] *= sy / yy;
        }
        for (int k = stored - 1; k >= 0; --k) {
            const int j = (head - 1 - k + mem) % mem;
            double yp = 0.0;
            for (int i = 0; i < q; ++i) yp += Y[j][i] * p[i];
            const double b = rho[j] * yp;
            for (int i = 0; i < q; ++i) p[i] += S[j][i] * (a[j] - b);
        }
        double gp = 0.0;
        for (int i = 0; i < q; ++i) {
            if (fixed[i]) p[i] = 0.0;
            gp += g[i] * p[i];
        }
        if (!(gp < 0.0)) {  // not a descent direction: restart from steepest descent
            stored = 0;
            gp = 0.0;
            for (int i = 0; i < q; ++i) {
                p[i] = fixed[i] ? 0.0 : -g[i];
                gp += g[i] * p[i];
            }
            if (!(gp < 0.0)) break;
        }
        double step = 1.0;
        if (stored == 0) {
            double pm = 0.0;
            for (int i = 0; i < q; ++i) pm = std::fmax(pm, std::fabs(p[i]));
            step = std::fmin(1.0, 1.0 / pm);
        }
        bool accepted = false;
        double fn = 0.0;
        for (int ls = 0; ls < 40; ++ls) {
            double dec = 0.0;
            for (int i = 0; i < q; ++i) {
                xn[i] = std::fmin(std::fmax(x[i] + step * p[i], lo[i]), hi[i]);
                dec += g[i] * (xn[i] - x[i]);
            }
            R.status = eval(xn, fn, gn);
            if (R.status != GPBO_OK) return R;
            if (std::isfinite(fn) && fn <= f + 1e-4 * dec) {
                accepted = true;
                break;
            }
            step *= 0.5;
        }
        if (!accepted) break;
        double sy = 0.0, ss = 0.0, yy = 0.0;
        for (int i = 0; i < q; ++i) {
            S[head][i] = xn[i] - x[i];
            Y[head][i] = gn[i] - g[i];
            sy += S[head][i] * Y[head][i];
            ss += S[head][i] * S[head][i];
            yy += Y[head][i] * Y[head][i];
        }
        if (sy > 1e-10 * std::sqrt(ss * yy)) {
            rho[head] = 1.0 / sy;
            head = (head + 1) % mem;
            stored = std::min(stored + 1, mem);
        }
        const double df = f - fn;
        x.swap(xn);
        g.swap(gn);
        f = fn;
        if (df <= 1e-12 * (1.0 + std::fabs(f))) break;
    }
    R.x = x;
    R.f = f;
    return R;
}

}  // namespace gpbo

using namespace gpbo;

static int stage_inputs(gpbo_ctx *ctx, const double *X, const double *y, int n, int d, unsigned flags, double **buf,
                        const double **Xd, const double **yd)
{
    *buf = nullptr;
    if (!(flags & GPBO_HOST_PTRS)) {
        *Xd = X;
        *yd = y;
        return GPBO_OK;
    }
    for (int64_t i = 0; i < (int64_t)n * d; ++i)
        if (!std::isfinite(X[i])) return GPBO_ENAN;
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(y[i])) return GPBO_ENAN;
    GPBO_CUDA_TRY(cudaMalloc(buf, sizeof(double) * ((size_t)n * d + n)));
    GPBO_CUDA_TRY(cudaMemcpyAsync(*buf, X, sizeof(double) * n * d, cudaMemcpyHostToDevice, ctx->stream));
    GPBO_CUDA_TRY(cudaMemcpyAsync(*buf + (size_t)n * d, y, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
    *Xd = *buf;
    *yd = *buf + (size_t)n * d;
    return GPBO_OK;
}

extern "C" {

int gp_lml(gpbo_ctx *ctx, const double *X, const double *y, int n, int d, const gp_hyper *hyp, unsigned flags,
           double *lml, double *grad)
{
    if (!ctx || !X || !y || !lml || n < 1 || n > GPBO_MAX_N || d < 1 || d > GPBO_MAX_D) return GPBO_EINVAL;
    GPBO_TRY(check_hyper(hyp, d));
    if (!(hyp->noise_var > 0)) return GPBO_EINVAL;
    GPBO_CUDA_TRY(cudaSetDevice(ctx->device));
    double *buf = nullptr;
    const double *Xd = nullptr, *yd = nullptr;
    GPBO_TRY(stage_inputs(ctx, X, y, n, d, flags, &buf, &Xd, &yd));
    MleState s;
    int st = mle_init(s, ctx, Xd, yd, n, d);
    std::vector<double> theta(d + 2), g(d + 2);
    for (int k = 0; k < d; ++k) theta[k] = std::log(hyp->lengthscale[k]);
    theta[d] = std::log(hyp->signal_var);
    theta[d + 1] = std::log(hyp->noise_var);
    double v = 0.0;
    if (st == GPBO_OK) st = mle_eval(s, theta.data(), &v, g.data());
    cudaStreamSynchronize(ctx->stream);
    mle_release(s);
    if (buf) cudaFree(buf);
    if (st != GPBO_OK) return st;
    *lml = v;
    if (grad)
        for (int j = 0; j < d + 2; ++j) grad[j] = g[j];
    return GPBO_OK;
}

int gp_fit_mle(gpbo_ctx *ctx, const double *X, const double *y, int n, int d, int n_starts, const double *theta0,
               const double *lo, const double *hi, int max_iter, double gtol, unsigned flags, double *theta_best,
               double *lml_best, int64_t *evals)
{
    if (!ctx || !X || !y || !theta0 || !lo || !hi || !theta_best || !lml_best || n < 1 || n > GPBO_MAX_N || d < 1 ||
        d > GPBO_MAX_D || n_starts < 1 || max_iter < 0 || !(gtol >= 0))
        return GPBO_EINVAL;
    const int q = d + 2;
    for (int i = 0; i < q; ++i)
        if (!std::isfinite(lo[i]) || !std::isfinite(hi[i]) || !(lo[i] <= hi[i])) return GPBO_EINVAL;
    for (int64_t i = 0; i < (int64_t)n_starts * q; ++i)
        if (!std::isfinite(theta0[i])) return GPBO_EINVAL;
    GPBO_CUDA_TRY(cudaSetDevice(ctx->device));
    double *buf = nullptr;
    const double *Xd = nullptr, *yd = nullptr;
    GPBO_TRY(stage_inputs(ctx, X, y, n, d, flags, &buf, &Xd, &yd));
    MleState s;
    int st = mle_init(s, ctx, Xd, yd, n, d);
    LbfgsResult best;
    bool any = false;
    for (int r = 0; r < n_starts && st == GPBO_OK; ++r) {
        LbfgsResult R = lbfgs_box(s, theta0 + (int64_t)r * q, lo, hi, max_iter, gtol);
        if (R.status == GPBO_ENOTSPD) continue;  // this start's initial point cannot be factored
        if (R.status != GPBO_OK) {
            st = R.status;
            break;
        }
        if (!any || R.f < best.f) {
            best = R;
            any = true;
        }
    }
    const int64_t ne = s.evals;
    cudaStreamSynchronize(ctx->stream);
    mle_release(s);
    if (buf) cudaFree(buf);
    if (st != GPBO_OK) return st;
    if (!any) return GPBO_ENOTSPD;
    for (int i = 0; i < q; ++i) theta_best[i] = best.x[i];
    *lml_best = -best.f;
    if (evals) *evals = ne;
    return GPBO_OK;
}

}  // extern "C"
