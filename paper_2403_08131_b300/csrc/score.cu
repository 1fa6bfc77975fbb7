// Candidate scoring: posterior mean, posterior standard deviation, expected improvement
// and its argmax over M candidates (§III-A: the acquisition function picks the next
// configuration to evaluate).
//
//   gen_candidates   x_ck = uniform24(seed, 2, c*d + k)                    (A2)
//   k_xkern          K*_ci = s2 m(r(x_c, x_i)) and mu_c = sum_i K*_ci alpha_i  (A7)
//   k_var_simt       v_c = L^-1 K*_c, sigma_c^2 = s2 - |v_c|^2, EI, argmax   (A8, A9)
//                    (FP64 / FP32 CUDA-core path; the 16-bit operand path runs the
//                    same step on tcgen05 tensor cores in score_tc.cu)
//   k_argmax_final   reduces the per-CTA (EI, index) winners; ties -> lowest index
//
// K* never exists for the whole pool: the pool is processed in chunks sized to the
// context's workspace bound, K* for a chunk is written once (row-major, candidate-major,
// observations contiguous, so that the variance GEMM streams it along its K dimension)
// and consumed by the variance kernel before the next chunk.
#include "gpbo_internal.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <mutex>

namespace gpbo {

__global__ void k_gen_candidates(uint64_t seed, int64_t first, int64_t M, int d, float *__restrict__ out)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t total = M * d;
    for (; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = t / d;
        int k = (int)(t - c * d);
        out[t] = uniform24f(seed, 2, (uint64_t)((first + c) * d + k));
    }
}

int gen_candidates(gpbo_ctx *ctx, uint64_t seed, int64_t first, int64_t M, int d, float *out)
{
    int64_t total = M * d;
    unsigned grid = (unsigned)std::min<int64_t>(cdiv64(total, 256), (int64_t)ctx->sm_count * 16);
    k_gen_candidates<<<std::max(1u, grid), 256, 0, ctx->stream>>>(seed, first, M, d, out);
    GPBO_LAUNCH_CHECK(ctx);
    return GPBO_OK;
}

template <typename A> __device__ __forceinline__ A matern_acc(A r2);
template <> __device__ __forceinline__ double matern_acc<double>(double r2) { return matern52_r2(r2); }
template <> __device__ __forceinline__ float matern_acc<float>(float r2) { return matern52_r2f(r2); }

// Cross-kernel and mean for candidates [c0, c0 + C) of the pool.
//   Acc  : arithmetic type (double for F64 scoring, float otherwise)
//   Out  : K* element type (double / float / bf16 / half)
//   Xc   : M x d FP32 candidates, or NULL to draw them from `seed`
//   Xs   : d x n_pad observations divided by the lengthscales, zero padding
//   Kst  : C x n_pad chunk buffer; mu: pool-indexed output
// CTA = 256 threads: 32 candidates (4 per warp) x 128 observations per tile (4 per lane).
template <typename Acc, typename Out>
__global__ void __launch_bounds__(256) k_xkern(const float *__restrict__ Xc, uint64_t seed, int64_t c0, int64_t C,
                                               int d, const Acc *__restrict__ Xs, const Acc *__restrict__ alpha,
                                               int n, int n_pad, Acc s2, Lengthscales_inv ls, Out *__restrict__ Kst,
                                               Acc *__restrict__ mu)
{
    extern __shared__ unsigned char smraw[];
    Acc *xc = reinterpret_cast<Acc *>(smraw);          // [32][d]
    Acc *xo = xc + 32 * d;                              // [d][128]
    Acc *al = xo + (int64_t)d * 128;                    // [128]
    const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
    const int64_t cbase = blockIdx.x * 32ll;
    for (int e = tid; e < 32 * d; e += 256) {
        int r = e / d, k = e % d;
        int64_t c = c0 + cbase + r;
        float x = Xc ? (cbase + r < C ? Xc[c * d + k] : 0.0f) : uniform24f(seed, 2, (uint64_t)(c * d + k));
        xc[e] = (Acc)x * (Acc)ls.inv[k];
    }
    Acc mp[4] = {Acc(0), Acc(0), Acc(0), Acc(0)};
    for (int i0 = 0; i0 < n_pad; i0 += 128) {
        __syncthreads();
        for (int e = tid; e < d * 128; e += 256) {
            int k = e / 128, q = e % 128;
            xo[e] = i0 + q < n_pad ? Xs[(int64_t)k * n_pad + i0 + q] : Acc(0);
        }
        if (tid < 128) al[tid] = i0 + tid < n_pad ? alpha[i0 + tid] : Acc(0);
        __syncthreads();
        Acc r2[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) r2[a][b] = Acc(0);
        for (int k = 0; k < d; ++k) {
            Acc cv[4], ov[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) cv[a] = xc[(warp * 4 + a) * d + k];
#pragma unroll
            for (int b = 0; b < 4; ++b) ov[b] = xo[k * 128 + lane + 32 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    Acc t = cv[a] - ov[b];
                    r2[a][b] = fma(t, t, r2[a][b]);
                }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int64_t cl = cbase + warp * 4 + a;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int i = i0 + lane + 32 * b;
                Acc kv = i < n ? s2 * matern_acc<Acc>(r2[a][b]) : Acc(0);
                mp[a] = fma(kv, al[lane + 32 * b], mp[a]);
                if (cl < C && i < n_pad) Kst[cl * n_pad + i] = (Out)kv;
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        Acc v = mp[a];
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        const int64_t cl = cbase + warp * 4 + a;
        if (lane == 0 && cl < C) mu[c0 + cl] = v;
    }
}

// FP32 cross-kernel and mean (F32, BF16 and F16 models): same results as k_xkern<float, Out>
// up to the last bits of r = sqrt(r^2) and exp, with fewer instructions per K* element.
// CTA = 256 threads = 8 warps x 8 candidates; each lane owns 4 consecutive observations of a
// 128-observation chunk, read as one float4 per dimension straight from L1/L2; K* leaves as
// one 8- or 16-byte store per candidate and chunk.
template <typename Out> struct Pack4;
template <> struct Pack4<float> {
    using T = float4;
    __device__ static T make(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
};
template <> struct Pack4<__half> {
    using T = uint2;
    __device__ static T make(float a, float b, float c, float d)
    {
        __half2 x = __floats2half2_rn(a, b), y = __floats2half2_rn(c, d);
        return make_uint2(*reinterpret_cast<uint32_t *>(&x), *reinterpret_cast<uint32_t *>(&y));
    }
};
template <> struct Pack4<__nv_bfloat16> {
    using T = uint2;
    __device__ static T make(float a, float b, float c, float d)
    {
        __nv_bfloat162 x = __floats2bfloat162_rn(a, b), y = __floats2bfloat162_rn(c, d);
        return make_uint2(*reinterpret_cast<uint32_t *>(&x), *reinterpret_cast<uint32_t *>(&y));
    }
};

// s2 (1 + sqrt5 r + 5 r^2 / 3) exp(-sqrt5 r) with r = r2 rsqrt(r2) (r = 0 at coincidence).
__device__ __forceinline__ float matern_fast(float r2, float s2)
{
    const float r = r2 > 0.0f ? r2 * rsqrtf(r2) : 0.0f;
    const float e = __expf(-2.2360680f * r);
    return s2 * fmaf(1.6666666f, r2, fmaf(2.2360680f, r, 1.0f)) * e;
}

template <typename Out>
__global__ void __launch_bounds__(256) k_xkern32(const float *__restrict__ Xc, uint64_t seed, int64_t c0, int64_t C,
                                                 int d, const float *__restrict__ Xs, const float *__restrict__ alpha,
                                                 int n, int n_pad, float s2, Lengthscales_inv ls, Out *__restrict__ Kst,
                                                 float *__restrict__ mu)
{
    constexpr int CW = 8;                 // candidates per warp
    extern __shared__ float cs[];         // [64][d]
    const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
    const int64_t cbase = blockIdx.x * 64ll;
    for (int e = tid; e < 64 * d; e += 256) {
        const int r = e / d, k = e - (e / d) * d;
        const int64_t c = c0 + cbase + r;
        const float x = Xc ? (cbase + r < C ? Xc[c * d + k] : 0.0f) : uniform24f(seed, 2, (uint64_t)(c * d + k));
        cs[e] = x * (float)ls.inv[k];
    }
    __syncthreads();
    const float *cw = cs + warp * CW * d;
    float mp[CW];
#pragma unroll
    for (int a = 0; a < CW; ++a) mp[a] = 0.0f;
    for (int i0 = 0; i0 < n_pad; i0 += 128) {
        const int i = i0 + 4 * lane;
        if (i >= n_pad) break;
        float r2[CW][4];
#pragma unroll
        for (int a = 0; a < CW; ++a) r2[a][0] = r2[a][1] = r2[a][2] = r2[a][3] = 0.0f;
        for (int k = 0; k < d; ++k) {
            const float4 o = *reinterpret_cast<const float4 *>(Xs + (size_t)k * n_pad + i);
#pragma unroll
            for (int a = 0; a < CW; ++a) {
                const float cv = cw[a * d + k];
                const float t0 = cv - o.x, t1 = cv - o.y, t2 = cv - o.z, t3 = cv - o.w;
                r2[a][0] = fmaf(t0, t0, r2[a][0]);
                r2[a][1] = fmaf(t1, t1, r2[a][1]);
                r2[a][2] = fmaf(t2, t2, r2[a][2]);
                r2[a][3] = fmaf(t3, t3, r2[a][3]);
            }
        }
        const float4 al = *reinterpret_cast<const float4 *>(alpha + i);
        const bool v0 = i < n, v1 = i + 1 < n, v2 = i + 2 < n, v3 = i + 3 < n;
#pragma unroll
        for (int a = 0; a < CW; ++a) {
            const float k0 = v0 ? matern_fast(r2[a][0], s2) : 0.0f;
            const float k1 = v1 ? matern_fast(r2[a][1], s2) : 0.0f;
            const float k2 = v2 ? matern_fast(r2[a][2], s2) : 0.0f;
            const float k3 = v3 ? matern_fast(r2[a][3], s2) : 0.0f;
            mp[a] = fmaf(k0, al.x, fmaf(k1, al.y, fmaf(k2, al.z, fmaf(k3, al.w, mp[a]))));
            const int64_t cl = cbase + warp * CW + a;
            if (cl < C)
                *reinterpret_cast<typename Pack4<Out>::T *>(Kst + cl * n_pad + i) = Pack4<Out>::make(k0, k1, k2, k3);
        }
    }
#pragma unroll
    for (int a = 0; a < CW; ++a) {
        float v = mp[a];
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        const int64_t cl = cbase + warp * CW + a;
        if (lane == 0 && cl < C) mu[c0 + cl] = v;
    }
}

// Variance, EI and per-CTA argmax on CUDA cores.  CTA = 64 candidates; it walks the
// lower triangle of L^-1 in 64-row blocks (outputs) and 16-wide K steps.
template <typename T>
__global__ void __launch_bounds__(256) k_var_simt(const T *__restrict__ Kst, int64_t C, int64_t c0, int n_pad,
                                                  const T *__restrict__ Linv, const T *__restrict__ mu, T s2,
                                                  double y_best, const double *__restrict__ tau_dev, T xi,
                                                  T *__restrict__ sigma_out, T *__restrict__ ei_out,
                                                  T *__restrict__ part_ei, int64_t *__restrict__ part_idx,
                                                  int part_base)
{
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    __shared__ T red_v[BM];
    __shared__ int64_t red_i[BM];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int64_t cb = blockIdx.x * (int64_t)BM;
    T sig2[4] = {T(0), T(0), T(0), T(0)};
    for (int i0 = 0; i0 < n_pad; i0 += BN) {
        T acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
        const int kend = i0 + BN;
        for (int k0 = 0; k0 < kend; k0 += BK) {
            {
                const int r = tid / 4, c = (tid % 4) * 4;
                const int64_t cr = cb + r;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    As[c + q][r] = cr < C ? Kst[cr * n_pad + k0 + c + q] : T(0);
                    Bs[c + q][r] = Linv[(int64_t)(i0 + r) * n_pad + k0 + c + q];
                }
            }
            __syncthreads();
#pragma unroll
            for (int t = 0; t < BK; ++t) {
                T x[4], y[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) { x[u] = As[t][ty + 16 * u]; y[u] = Bs[t][tx + 16 * u]; }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = fma(x[u], y[v], acc[u][v]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) sig2[u] = fma(acc[u][v], acc[u][v], sig2[u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
        for (int o = 1; o < 16; o <<= 1) sig2[u] += __shfl_xor_sync(0xffffffffu, sig2[u], o);
    const T tau = tau_dev ? (T)*tau_dev : (T)y_best;
    if (tx == 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = ty + 16 * u;
            const int64_t cl = cb + r, c = c0 + cl;
            T e = T(-1);
            if (cl < C) {
                T var = s2 - sig2[u];
                T sg = var > T(0) ? sqrt(var) : T(0);
                T m = mu[c];
                if constexpr (sizeof(T) == 8) e = ei_min(m, sg, tau, xi);
                else e = ei_minf(m, sg, tau, xi);
                if (sigma_out) sigma_out[c] = sg;
                if (ei_out) ei_out[c] = e;
            }
            red_v[r] = e;
            red_i[r] = cl < C ? c : INT64_MAX;
        }
    }
    __syncthreads();
    for (int s = BM / 2; s; s >>= 1) {
        if (tid < s) {
            if (better(red_v[tid + s], red_i[tid + s], red_v[tid], red_i[tid])) {
                red_v[tid] = red_v[tid + s];
                red_i[tid] = red_i[tid + s];
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        part_ei[part_base + blockIdx.x] = red_v[0];
        part_idx[part_base + blockIdx.x] = red_i[0];
    }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_argmax_final(const T *__restrict__ part_ei, const int64_t *__restrict__ part_idx,
                                                       int np, double *__restrict__ out_ei, int64_t *__restrict__ out_idx)
{
    __shared__ T sv[1024];
    __shared__ int64_t si[1024];
    T bv = T(-2);
    int64_t bi = INT64_MAX;
    for (int p = threadIdx.x; p < np; p += blockDim.x)
        if (better(part_ei[p], part_idx[p], bv, bi)) { bv = part_ei[p]; bi = part_idx[p]; }
    sv[threadIdx.x] = bv;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s; s >>= 1) {
        if (threadIdx.x < s && better(sv[threadIdx.x + s], si[threadIdx.x + s], sv[threadIdx.x], si[threadIdx.x])) {
            sv[threadIdx.x] = sv[threadIdx.x + s];
            si[threadIdx.x] = si[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *out_ei = (double)sv[0];
        *out_idx = si[0];
    }
}

// ------------------------------------------------------------------ orchestration
template <typename Acc, typename Out>
static int launch_xkern(gpbo_ctx *ctx, const gp_model *m, const float *Xc, uint64_t seed, int64_t c0, int64_t C,
                        const Acc *Xs, const Acc *alpha, Out *Kst, Acc *mu)
{
    Lengthscales_inv ls;
    for (int k = 0; k < m->d; ++k) ls.inv[k] = 1.0 / m->ls[k];
    if constexpr (sizeof(Acc) == 4) {
        // FP32 models: the register-tiled kernel (n_pad is a multiple of 64, so every float4 is in bounds)
        const size_t smem = sizeof(float) * 64 * (size_t)m->d;
        k_xkern32<Out><<<(unsigned)cdiv64(C, 64), 256, smem, ctx->stream>>>(Xc, seed, c0, C, m->d, Xs, alpha, m->n,
                                                                             m->n_pad, (float)m->s2, ls, Kst, mu);
        GPBO_LAUNCH_CHECK(ctx);
        return GPBO_OK;
    }
    const size_t smem = sizeof(Acc) * ((size_t)32 * m->d + (size_t)m->d * 128 + 128);
    static int attr_bytes = 0;  // one per template instance
    if ((int)smem > attr_bytes) {
        GPBO_CUDA_TRY(cudaFuncSetAttribute(k_xkern<Acc, Out>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_bytes = (int)smem;
    }
    k_xkern<Acc, Out><<<(unsigned)cdiv64(C, 32), 256, smem, ctx->stream>>>(Xc, seed, c0, C, m->d, Xs, alpha, m->n,
                                                                          m->n_pad, (Acc)m->s2, ls, Kst, mu);
    GPBO_LAUNCH_CHECK(ctx);
    return GPBO_OK;
}

template <typename T>
static int score_simt(gpbo_ctx *ctx, const gp_model *m, const float *Xc, int64_t M, uint64_t seed, double y_best,
                      const double *tau_dev, double xi, T *mu_out, T *sigma_out, T *ei_out, int64_t *argmax,
                      double *ei_max)
{
    const int n_pad = m->n_pad;
    const T *Xs = nullptr, *alpha = nullptr, *Linv = nullptr;
    if constexpr (sizeof(T) == 8) { Xs = m->Xs64; alpha = m->alpha64; Linv = m->Linv64; }
    else { Xs = m->Xs32; alpha = m->alpha32; Linv = m->Linv32; }
    // chunk so that K* fits in the workspace bound (minus the small vectors)
    const int64_t per_cand = (int64_t)n_pad * sizeof(T);
    const int64_t budget = std::max<int64_t>(ctx->ws_limit / 2, 64 * per_cand);
    int64_t C = std::min<int64_t>(M, std::max<int64_t>(64, budget / per_cand / 64 * 64));
    const int64_t nchunks = cdiv64(M, C);
    const int64_t parts_per_chunk = cdiv64(C, 64);
    const int64_t np = parts_per_chunk * nchunks;
    const size_t bytes = sizeof(int64_t) * np + 16 + sizeof(T) * np + 48 + 256 + (size_t)C * per_cand +
                         (mu_out ? 0 : sizeof(T) * (size_t)M) + 256;
    void *w = nullptr;
    GPBO_TRY(ws_reserve(ctx, bytes, &w));
    char *p = (char *)w;
    int64_t *pidx = (int64_t *)p;            p += sizeof(int64_t) * np;
    double *res = (double *)p;               p += 16;
    T *pei = (T *)p;                         p += sizeof(T) * np + 48;
    T *Kst = (T *)(((uintptr_t)p + 255) & ~(uintptr_t)255);
    p = (char *)(Kst + C * n_pad);
    T *mu = mu_out ? mu_out : (T *)p;
    int part = 0;
    for (int64_t c0 = 0; c0 < M; c0 += C) {
        const int64_t Cc = std::min(C, M - c0);
        const double nn = (double)m->n;
        GPBO_TRY(trace_begin(ctx, PH_XKERN, (double)Cc * (3.0 * nn * m->d + 2.0 * nn)));
        GPBO_TRY((launch_xkern<T, T>(ctx, m, Xc, seed, c0, Cc, Xs, alpha, Kst, mu)));
        GPBO_TRY(trace_end(ctx));
        const unsigned g = (unsigned)cdiv64(Cc, 64);
        GPBO_TRY(trace_begin(ctx, PH_VAR, (double)Cc * nn * (nn + 1.0)));
        k_var_simt<T><<<g, 256, 0, ctx->stream>>>(Kst, Cc, c0, n_pad, Linv, mu, (T)m->s2, y_best, tau_dev, (T)xi,
                                                  sigma_out, ei_out, pei, pidx, part);
        GPBO_LAUNCH_CHECK(ctx);
        GPBO_TRY(trace_end(ctx));
        part += (int)g;
    }
    k_argmax_final<T><<<1, 1024, 0, ctx->stream>>>(pei, pidx, part, res, (int64_t *)(res + 1));
    GPBO_LAUNCH_CHECK(ctx);
    GPBO_CUDA_TRY(cudaMemcpyAsync(ctx->pinned, res, 16, cudaMemcpyDeviceToHost, ctx->stream));
    GPBO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    *ei_max = ((double *)ctx->pinned)[0];
    *argmax = ((int64_t *)ctx->pinned)[1];
    return GPBO_OK;
}

template <typename Out>
static int score_tc(gpbo_ctx *ctx, const gp_model *m, const float *Xc, int64_t M, uint64_t seed, double y_best,
                    const double *tau_dev, double xi, float *mu_out, float *sigma_out, float *ei_out,
                    int64_t *argmax, double *ei_max)
{
    const int n_pad = m->n_pad;
    const int64_t per_cand = (int64_t)n_pad * sizeof(Out);
    const int64_t budget = std::max<int64_t>(ctx->ws_limit / 2, 128 * per_cand);
    int64_t C = std::min<int64_t>(round_up64(M, 128), std::max<int64_t>(128, budget / per_cand / 128 * 128));
    const int64_t nchunks = cdiv64(M, C);
    const int64_t np = (int64_t)ctx->sm_count * 2 * nchunks + 16;
    const size_t bytes = sizeof(int64_t) * np + 16 + sizeof(float) * np + 48 + 1024 + (size_t)C * per_cand +
                         (mu_out ? 0 : sizeof(float) * (size_t)M) + 256;
    void *w = nullptr;
    GPBO_TRY(ws_reserve(ctx, bytes, &w));
    char *p = (char *)w;
    int64_t *pidx = (int64_t *)p;            p += sizeof(int64_t) * np;
    double *res = (double *)p;               p += 16;
    float *pei = (float *)p;                 p += sizeof(float) * np + 48;
    Out *Kst = (Out *)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
    p = (char *)(Kst + C * n_pad);
    float *mu = mu_out ? mu_out : (float *)p;
    int part = 0;
    for (int64_t c0 = 0; c0 < M; c0 += C) {
        const int64_t Cc = std::min(C, M - c0);
        const double nn = (double)m->n;
        GPBO_TRY(trace_begin(ctx, PH_XKERN, (double)Cc * (3.0 * nn * m->d + 2.0 * nn)));
        if (xkern_tc_usable(m))
            GPBO_TRY(xkern_tc(ctx, m, Xc, seed, c0, Cc, Kst, mu));
        else
            GPBO_TRY((launch_xkern<float, Out>(ctx, m, Xc, seed, c0, Cc, m->Xs32, m->alpha32, Kst, mu)));
        GPBO_TRY(trace_end(ctx));
        int used = 0;
        GPBO_TRY(trace_begin(ctx, PH_VAR, (double)Cc * nn * (nn + 1.0)));
        GPBO_TRY(tc_variance_ei(ctx, m, Kst, Cc, c0, mu, y_best, tau_dev, xi, sigma_out, ei_out, pei + part,
                                pidx + part, &used));
        GPBO_TRY(trace_end(ctx));
        part += used;
    }
    k_argmax_final<float><<<1, 1024, 0, ctx->stream>>>(pei, pidx, part, res, (int64_t *)(res + 1));
    GPBO_LAUNCH_CHECK(ctx);
    GPBO_CUDA_TRY(cudaMemcpyAsync(ctx->pinned, res, 16, cudaMemcpyDeviceToHost, ctx->stream));
    GPBO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    unsigned bits = 0;
    GPBO_TRY(take_device_status(ctx, &bits));
    if (bits & DEV_TIMEOUT) return GPBO_ETIMEOUT;
    *ei_max = ((double *)ctx->pinned)[0];
    *argmax = ((int64_t *)ctx->pinned)[1];
    return GPBO_OK;
}

int score_model(gpbo_ctx *ctx, const gp_model *m, const float *Xc, int64_t M, uint64_t seed, double y_best,
                const double *tau_dev, double xi, void *mu, void *sigma, void *ei, int64_t *argmax, double *ei_max)
{
    switch (m->prec) {
    case GPBO_PREC_F64:
        return score_simt<double>(ctx, m, Xc, M, seed, y_best, tau_dev, xi, (double *)mu, (double *)sigma,
                                  (double *)ei, argmax, ei_max);
    case GPBO_PREC_F32:
        return score_simt<float>(ctx, m, Xc, M, seed, y_best, tau_dev, xi, (float *)mu, (float *)sigma,
                                 (float *)ei, argmax, ei_max);
    case GPBO_PREC_BF16:
        return score_tc<__nv_bfloat16>(ctx, m, Xc, M, seed, y_best, tau_dev, xi, (float *)mu, (float *)sigma,
                                       (float *)ei, argmax, ei_max);
    case GPBO_PREC_F16:
        return score_tc<__half>(ctx, m, Xc, M, seed, y_best, tau_dev, xi, (float *)mu, (float *)sigma,
                                (float *)ei, argmax, ei_max);
    }
    return GPBO_EINVAL;
}

// ------------------------------------------------------------------ allocation-free scoring
// gp_posterior_ei_noalloc: the CUDA-core scoring path with its scratch (K* chunk, per-CTA
// argmax partials, running best) in one fixed file-scope device array instead of the
// context's workspace, so that a call allocates nothing.

static __device__ __align__(256) unsigned char g_noalloc_scratch[GPBO_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
unsigned char *g_noalloc_dev[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on `device` (which must be current).  In host code the
// array's name is only a stand-in for the symbol, never a usable address.
int noalloc_scratch(int device, unsigned char **out)
{
    if (device < 0 || device >= NOALLOC_MAX_DEVICES) return GPBO_ENOTSUP;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_dev[device]) {
        void *p = nullptr;
        GPBO_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_dev[device] = (unsigned char *)p;
    }
    *out = g_noalloc_dev[device];
    return GPBO_OK;
}
}  // namespace

__global__ void k_noalloc_reset(double *best_ei, int64_t *best_idx)
{
    *best_ei = -2.0;
    *best_idx = INT64_MAX;
}

// Reduce one chunk's per-CTA partials and merge them into the running best.
template <typename T>
__global__ void __launch_bounds__(1024) k_noalloc_merge(const T *__restrict__ part_ei, const int64_t *__restrict__ part_idx,
                                                        int np, double *best_ei, int64_t *best_idx)
{
    __shared__ double sv[1024];
    __shared__ int64_t si[1024];
    double bv = -2.0;
    int64_t bi = INT64_MAX;
    for (int p = threadIdx.x; p < np; p += blockDim.x)
        if (better((double)part_ei[p], part_idx[p], bv, bi)) { bv = (double)part_ei[p]; bi = part_idx[p]; }
    sv[threadIdx.x] = bv;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s; s >>= 1) {
        if (threadIdx.x < s && better(sv[threadIdx.x + s], si[threadIdx.x + s], sv[threadIdx.x], si[threadIdx.x])) {
            sv[threadIdx.x] = sv[threadIdx.x + s];
            si[threadIdx.x] = si[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && better(sv[0], si[0], *best_ei, *best_idx)) {
        *best_ei = sv[0];
        *best_idx = si[0];
    }
}

template <typename T>
static int score_noalloc(gpbo_ctx *ctx, const gp_model *m, const float *Xc, int64_t M, uint64_t seed, double y_best,
                         double xi, T *mu_out, T *sigma_out, T *ei_out, int64_t *argmax, double *ei_max)
{
    const int n_pad = m->n_pad;
    const size_t per_cand = (size_t)n_pad * sizeof(T);
    // layout: [0,256) running best | partials (ei T, idx int64) | mu chunk (if needed) | K* chunk
    const size_t head = 256;
    auto need = [&](int64_t C) {
        const size_t np = (size_t)cdiv64(C, 64);
        size_t b = head + np * (sizeof(T) + sizeof(int64_t)) + 256;
        b += (mu_out ? 0 : (size_t)C * sizeof(T)) + 256;
        return b + (size_t)C * per_cand;
    };
    int64_t C = (int64_t)(GPBO_NOALLOC_SCRATCH_BYTES / (per_cand + sizeof(T) + 1)) / 64 * 64;
    while (C >= 64 && need(C) > GPBO_NOALLOC_SCRATCH_BYTES) C -= 64;
    if (C < 64) return GPBO_ESCRATCH;
    C = std::min<int64_t>(C, round_up64(M, 64));
    unsigned char *base = nullptr;
    GPBO_TRY(noalloc_scratch(ctx->device, &base));
    double *best_ei = (double *)base;
    int64_t *best_idx = (int64_t *)(base + 8);
    const int64_t np = cdiv64(C, 64);
    int64_t *pidx = (int64_t *)(base + head);
    T *pei = (T *)(base + head + np * sizeof(int64_t));
    unsigned char *p = (unsigned char *)(((uintptr_t)(pei + np) + 255) & ~(uintptr_t)255);
    T *mu_chunk = nullptr;
    if (!mu_out) {
        mu_chunk = (T *)p;
        p = (unsigned char *)(((uintptr_t)(mu_chunk + C) + 255) & ~(uintptr_t)255);
    }
    T *Kst = (T *)p;
    const T *Xs = nullptr, *alpha = nullptr, *Linv = nullptr;
    if constexpr (sizeof(T) == 8) { Xs = m->Xs64; alpha = m->alpha64; Linv = m->Linv64; }
    else { Xs = m->Xs32; alpha = m->alpha32; Linv = m->Linv32; }
    k_noalloc_reset<<<1, 1, 0, ctx->stream>>>(best_ei, best_idx);
    GPBO_LAUNCH_CHECK(ctx);
    for (int64_t c0 = 0; c0 < M; c0 += C) {
        const int64_t Cc = std::min(C, M - c0);
        // the kernels index mu by pool position; the chunk buffer stands in for [c0, c0 + Cc)
        T *mu = mu_out ? mu_out : mu_chunk - c0;
        GPBO_TRY((launch_xkern<T, T>(ctx, m, Xc, seed, c0, Cc, Xs, alpha, Kst, mu)));
        const unsigned g = (unsigned)cdiv64(Cc, 64);
        k_var_simt<T><<<g, 256, 0, ctx->stream>>>(Kst, Cc, c0, n_pad, Linv, mu, (T)m->s2, y_best, nullptr, (T)xi,
                                                  sigma_out, ei_out, pei, pidx, 0);
        GPBO_LAUNCH_CHECK(ctx);
        k_noalloc_merge<T><<<1, 1024, 0, ctx->stream>>>(pei, pidx, (int)g, best_ei, best_idx);
        GPBO_LAUNCH_CHECK(ctx);
    }
    GPBO_CUDA_TRY(cudaMemcpyAsync(ctx->pinned, base, 16, cudaMemcpyDeviceToHost, ctx->stream));
    GPBO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    *ei_max = ((double *)ctx->pinned)[0];
    *argmax = ((int64_t *)ctx->pinned)[1];
    return GPBO_OK;
}

}  // namespace gpbo

extern "C" int gp_posterior_ei_noalloc(gpbo_ctx *ctx, const gp_model *m, const float *Xc, int64_t M, uint64_t seed,
                                       double y_best, double xi, void *mu, void *sigma, void *ei, int64_t *argmax,
                                       double *ei_max)
{
    using namespace gpbo;
    if (!ctx || !m || !argmax || !ei_max || M < 1 || M > 0x7fffffffll) return GPBO_EINVAL;
    if (!std::isfinite(y_best) || !std::isfinite(xi)) return GPBO_EINVAL;
    if (m->prec != GPBO_PREC_F32 && m->prec != GPBO_PREC_F64) return GPBO_ENOTSUP;
    GPBO_CUDA_TRY(cudaSetDevice(ctx->device));
    int64_t am = -1;
    double em = 0.0;
    int st = m->prec == GPBO_PREC_F64
                 ? score_noalloc<double>(ctx, m, Xc, M, seed, y_best, xi, (double *)mu, (double *)sigma, (double *)ei,
                                         &am, &em)
                 : score_noalloc<float>(ctx, m, Xc, M, seed, y_best, xi, (float *)mu, (float *)sigma, (float *)ei,
                                        &am, &em);
    if (st != GPBO_OK) return st;
    *argmax = am;
    *ei_max = em;
    return GPBO_OK;
}

