// Device bodies of the scoring kernels (candidates, cross-kernel, CUDA-core variance + EI,
// argmax), shared by the single-problem kernels (score.cu) and the batched kernels
// (batched.cu).  Each body takes its block coordinates as arguments.
#pragma once
#include <type_traits>

#include "gpbo_internal.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace gpbo {

__device__ __forceinline__ void k_gen_candidates_body(uint64_t seed, int64_t first, int64_t M, int d, float *__restrict__ out, const int bx, const int by, const int gx)
{
    int64_t t = bx * (int64_t)blockDim.x + threadIdx.x;
    int64_t total = M * d;
    for (; t < total; t += (int64_t)gx * blockDim.x) {
        int64_t c = t / d;
        int k = (int)(t - c * d);
        out[t] = uniform24f(seed, 2, (uint64_t)((first + c) * d + k));
    }
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
__device__ __forceinline__ void k_xkern_body(const float *__restrict__ Xc, uint64_t seed, int64_t c0, int64_t C,
                                               int d, const Acc *__restrict__ Xs, const Acc *__restrict__ alpha,
                                               int n, int n_pad, Acc s2, Lengthscales_inv ls, Out *__restrict__ Kst,
                                               Acc *__restrict__ mu, const int bx, const int by, const int gx)
{
    extern __shared__ unsigned char smraw[];
    Acc *xc = reinterpret_cast<Acc *>(smraw);          // [32][d]
    Acc *xo = xc + 32 * d;                              // [d][128]
    Acc *al = xo + (int64_t)d * 128;                    // [128]
    const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
    const int64_t cbase = bx * 32ll;
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

// Cross-kernel and mean for FP32 scoring: CTA = 256 threads = 64 candidates (8 per warp) x
// blocks of 128 observations (4 per lane).  Dynamic shared memory: sizeof(float) (192 d + 128).
// Its kernels are bounded to 64 registers (four CTAs per SM, no spills): 128 left two CTAs
// per SM, too few warps to cover the shared-memory and MUFU latencies (the batched step
// 17.97 -> 17.57 ms, 17.73 ms at three CTAs).
template <typename Out>
__device__ __forceinline__ void k_xkern32_body(const float *__restrict__ Xc, uint64_t seed, int64_t c0, int64_t C,
                                                 int d, const float *__restrict__ Xs, const float *__restrict__ alpha,
                                                 int n, int n_pad, float s2, Lengthscales_inv ls, Out *__restrict__ Kst,
                                                 float *__restrict__ mu, const int bx, const int by, const int gx)
{
    constexpr int CW = 8;                 // candidates per warp
    extern __shared__ float cs[];         // [64][d] candidates, [d][128] observations, [128] alpha
    float *xo = cs + 64 * d;
    float *al = xo + 128 * d;
    const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
    const int64_t cbase = bx * 64ll;
    for (int e = tid; e < 64 * d; e += 256) {
        const int r = e / d, k = e - (e / d) * d;
        const int64_t c = c0 + cbase + r;
        const float x = Xc ? (cbase + r < C ? Xc[c * d + k] : 0.0f) : uniform24f(seed, 2, (uint64_t)(c * d + k));
        cs[e] = x * (float)ls.inv[k];
    }
    const float *cw = cs + warp * CW * d;
    float mp[CW];
#pragma unroll
    for (int a = 0; a < CW; ++a) mp[a] = 0.0f;
    for (int i0 = 0; i0 < n_pad; i0 += 128) {
        // the block's observations and alpha, staged once for the CTA (the previous block's
        // reads are done first): the d-step loop below then never waits on a global load
        __syncthreads();
        for (int e = tid; e < d * 128; e += 256) {
            const int k = e >> 7, q = e & 127;
            xo[e] = i0 + q < n_pad ? Xs[(size_t)k * n_pad + i0 + q] : 0.0f;
        }
        if (tid < 128) al[tid] = i0 + tid < n_pad ? alpha[i0 + tid] : 0.0f;
        __syncthreads();
        const int i = i0 + 4 * lane;
        if (i >= n_pad) continue;  // n_pad is a multiple of 64: whole float4s or none
        float r2[CW][4];
#pragma unroll
        for (int a = 0; a < CW; ++a) r2[a][0] = r2[a][1] = r2[a][2] = r2[a][3] = 0.0f;
        for (int k = 0; k < d; ++k) {
            const float4 o = *reinterpret_cast<const float4 *>(xo + k * 128 + 4 * lane);
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
        const float4 alv = *reinterpret_cast<const float4 *>(al + 4 * lane);
        const bool v0 = i < n, v1 = i + 1 < n, v2 = i + 2 < n, v3 = i + 3 < n;
#pragma unroll
        for (int a = 0; a < CW; ++a) {
            const float k0 = v0 ? matern_fast(r2[a][0], s2) : 0.0f;
            const float k1 = v1 ? matern_fast(r2[a][1], s2) : 0.0f;
            const float k2 = v2 ? matern_fast(r2[a][2], s2) : 0.0f;
            const float k3 = v3 ? matern_fast(r2[a][3], s2) : 0.0f;
            mp[a] = fmaf(k0, alv.x, fmaf(k1, alv.y, fmaf(k2, alv.z, fmaf(k3, alv.w, mp[a]))));
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

// Variance, EI and per-CTA argmax on CUDA cores.  CTA = BM candidates (32, 64 or 128; each
// thread owns BM/16 of them); it walks the lower triangle of L^-1 in 64-row blocks (outputs)
// and 16-wide K steps.  Every candidate's sums run in the same order for every BM, so the
// results do not depend on the tile.
template <typename T, int BM = 64>
__device__ __forceinline__ void k_var_simt_body(const T *__restrict__ Kst, int64_t C, int64_t c0, int n_pad,
                                                  const T *__restrict__ Linv, const T *__restrict__ mu, T s2,
                                                  double y_best, const double *__restrict__ tau_dev, T xi,
                                                  T *__restrict__ sigma_out, T *__restrict__ ei_out,
                                                  T *__restrict__ part_ei, int64_t *__restrict__ part_idx,
                                                  int part_base, const int bx, const int by, const int gx)
{
    static_assert(BM == 32 || BM == 64 || BM == 128, "tile");
    constexpr int BN = 64, BK = 16, TM = BM / 16, EA = BM * BK / 256;
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    __shared__ T red_v[BM];
    __shared__ int64_t red_i[BM];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int64_t cb = bx * (int64_t)BM;
    T sig2[TM];
#pragma unroll
    for (int u = 0; u < TM; ++u) sig2[u] = T(0);
    for (int i0 = 0; i0 < n_pad; i0 += BN) {
        T acc[TM][4];
#pragma unroll
        for (int u = 0; u < TM; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
        const int kend = i0 + BN;
        for (int k0 = 0; k0 < kend; k0 += BK) {
            {
                const int r = tid / (BK / EA), c = (tid % (BK / EA)) * EA;
                const int64_t cr = cb + r;
#pragma unroll
                for (int q = 0; q < EA; ++q) As[c + q][r] = cr < C ? Kst[cr * n_pad + k0 + c + q] : T(0);
                const int rb = tid / 4, cbk = (tid % 4) * 4;
#pragma unroll
                for (int q = 0; q < 4; ++q) Bs[cbk + q][rb] = Linv[(int64_t)(i0 + rb) * n_pad + k0 + cbk + q];
            }
            __syncthreads();
#pragma unroll
            for (int t = 0; t < BK; ++t) {
                T x[TM], y[4];
#pragma unroll
                for (int u = 0; u < TM; ++u) x[u] = As[t][ty + 16 * u];
#pragma unroll
                for (int v = 0; v < 4; ++v) y[v] = Bs[t][tx + 16 * v];
#pragma unroll
                for (int u = 0; u < TM; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = fma(x[u], y[v], acc[u][v]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int u = 0; u < TM; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) sig2[u] = fma(acc[u][v], acc[u][v], sig2[u]);
    }
#pragma unroll
    for (int u = 0; u < TM; ++u)
        for (int o = 1; o < 16; o <<= 1) sig2[u] += __shfl_xor_sync(0xffffffffu, sig2[u], o);
    const T tau = tau_dev ? (T)*tau_dev : (T)y_best;
    if (tx == 0) {
#pragma unroll
        for (int u = 0; u < TM; ++u) {
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
        part_ei[part_base + bx] = red_v[0];
        part_idx[part_base + bx] = red_i[0];
    }
}

// FP32 variance, EI and per-CTA argmax on CUDA cores, BM = 64, 128 or 256 candidates per CTA.
// The output is worked through in chunks of 128 rows of L^-1 (chunk q needs K columns below
// 128 (q + 1) only: the triangle's zero blocks are skipped).  Thread (ty, tx) of 16 x 16 owns
// candidates ty*TM .. ty*TM+TM-1 (TM = BM/16) and rows tx*4 .. tx*4+3 and 64+tx*4 .. 64+tx*4+3
// of each chunk: an 8 x TM register tile, so each K step reads 8 + TM floats from shared
// memory (128-bit reads, conflict-free) for 8 TM FMAs, within the shared-memory port at the
// FMA rate.  K* is read in 64-byte row segments (four lanes per candidate) and L^-1 likewise;
// both go through transposed shared tiles in K steps of 8, the next step's global loads held
// in registers while the current one is multiplied (short steps keep the register count at
// 128, so that two CTAs share an SM and hide each other's latencies).  Successive chunks run over K in opposite
// directions, so a chunk starts on the K* columns the previous one read last (still in L2).
// Every candidate's sums run in the same order for every BM, so the tile changes no result.
template <int BM, bool TRI_SKIP = false>
__device__ __forceinline__ void k_var_f32_body(const float *__restrict__ Kst, int64_t C, int64_t c0, int n_pad,
                                               const float *__restrict__ Linv, const float *__restrict__ mu, float s2,
                                               double y_best, const double *__restrict__ tau_dev, float xi,
                                               float *__restrict__ sigma_out, float *__restrict__ ei_out,
                                               float *__restrict__ part_ei, int64_t *__restrict__ part_idx,
                                               int part_base, const int bx)
{
    static_assert(BM == 64 || BM == 128 || BM == 256, "tile");
    constexpr int BN = 128, BK = 8, TM = BM / 16, PAD = 4;
    constexpr int LPR = BK / 4;              // lanes per row segment (float4 each)
    constexpr int RPP = 256 / LPR;           // rows covered by one pass of the CTA's threads
    constexpr int AQ = (BM + RPP - 1) / RPP; // K* float4s per thread per K step (some idle if BM < RPP)
    constexpr int BQ = BN / RPP;             // L^-1 float4s per thread per K step
    __shared__ __align__(16) float As[2][BK][BM + PAD];
    __shared__ __align__(16) float Bs[2][BK][BN + PAD];
    __shared__ float red_v[BM];
    __shared__ int64_t red_i[BM];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int64_t cb = bx * (int64_t)BM;
    const int lr = tid / LPR, lk = (tid % LPR) * 4;  // loader: row within a pass, first k
    float4 pa[AQ], pb[BQ];
    auto fetch = [&](int k0, int i0) {
#pragma unroll
        for (int q = 0; q < AQ; ++q) {
            const int64_t c = cb + lr + q * RPP;
            pa[q] = c < C && (BM >= RPP || lr + q * RPP < BM) ? *reinterpret_cast<const float4 *>(Kst + c * n_pad + k0 + lk)
                                               : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < BQ; ++q) {
            const int i = i0 + lr + q * RPP;
            pb[q] = i < n_pad ? *reinterpret_cast<const float4 *>(Linv + (int64_t)i * n_pad + k0 + lk)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    auto stash = [&](int buf) {
#pragma unroll
        for (int q = 0; q < AQ; ++q) {
            const int r = lr + q * RPP;
            if (BM < RPP && r >= BM) break;
            As[buf][lk + 0][r] = pa[q].x;
            As[buf][lk + 1][r] = pa[q].y;
            As[buf][lk + 2][r] = pa[q].z;
            As[buf][lk + 3][r] = pa[q].w;
        }
#pragma unroll
        for (int q = 0; q < BQ; ++q) {
            const int r = lr + q * RPP;
            Bs[buf][lk + 0][r] = pb[q].x;
            Bs[buf][lk + 1][r] = pb[q].y;
            Bs[buf][lk + 2][r] = pb[q].z;
            Bs[buf][lk + 3][r] = pb[q].w;
        }
    };
    float sig2[TM];
#pragma unroll
    for (int u = 0; u < TM; ++u) sig2[u] = 0.f;
    int buf = 0;
    for (int i0 = 0, q = 0; i0 < n_pad; i0 += BN, ++q) {
        // acc[u2][v] = the products of candidates 2 u2 and 2 u2 + 1 with row v, on paired FP32
        // lanes: each lane runs the scalar FMA sequence, so the sums are those of one lane each
        float2 acc[TM / 2][8];
#pragma unroll
        for (int u = 0; u < TM / 2; ++u)
#pragma unroll
            for (int v = 0; v < 8; ++v) acc[u][v] = make_float2(0.f, 0.f);
        const int ksteps = (min(i0 + BN, n_pad) + BK - 1) / BK;
        const bool down = (q & 1) != 0;
        fetch(down ? (ksteps - 1) * BK : 0, i0);
        stash(buf);
        __syncthreads();
        // Rows v = 0..3 of the thread's tile lie in the chunk's first 64 rows, v = 4..7 in the
        // second.  L^-1 is lower triangular with exact zeros above its diagonal, so the K steps
        // from column i0 + 64 on contribute exactly nothing to the first 64 rows, and a chunk
        // that ends 64 rows early (n_pad - i0 = 64) has only padding in its second half.  With
        // TRI_SKIP those products are skipped, which leaves every sum as it was: the batched
        // form's many small problems execute 13% fewer FMAs; at n = 4096 the single path would
        // save 1.5%, less than the extra code costs it (its 128-candidate tile then spills).
        const int kz = (i0 + 64) / BK;              // first K step of the chunk's second half
        const bool half_chunk = n_pad - i0 <= 64;
        // one K step over rows v in [V0, V1) of the thread tile
        auto kstep = [&](auto V0c, auto V1c) {
            constexpr int V0 = decltype(V0c)::value, V1 = decltype(V1c)::value;
#pragma unroll
            for (int t0 = 0; t0 < BK; ++t0) {
                const int t = down ? BK - 1 - t0 : t0;  // K fully descending on those chunks
                float a[TM], b[8];
#pragma unroll
                for (int g = 0; g < TM / 4; ++g) {
                    const float4 f = *reinterpret_cast<const float4 *>(&As[buf][t][ty * TM + 4 * g]);
                    a[4 * g] = f.x;
                    a[4 * g + 1] = f.y;
                    a[4 * g + 2] = f.z;
                    a[4 * g + 3] = f.w;
                }
                if (V0 == 0) {
                    const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][t][tx * 4]);
                    b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
                }
                if (V1 == 8) {
                    const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][t][64 + tx * 4]);
                    b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
                }
#pragma unroll
                for (int v = V0; v < V1; ++v) {
                    const float2 bb = make_float2(b[v], b[v]);
#pragma unroll
                    for (int u = 0; u < TM / 2; ++u) acc[u][v] = fma2(make_float2(a[2 * u], a[2 * u + 1]), bb, acc[u][v]);
                }
            }
        };
        for (int s = 0; s < ksteps; ++s) {
            const bool more = s + 1 < ksteps;
            if (more) fetch((down ? ksteps - 2 - s : s + 1) * BK, i0);
            const int ks = down ? ksteps - 1 - s : s;   // the K step computed now
            if constexpr (TRI_SKIP) {
                if (half_chunk) kstep(std::integral_constant<int, 0>(), std::integral_constant<int, 4>());
                else if (ks >= kz) kstep(std::integral_constant<int, 4>(), std::integral_constant<int, 8>());
                else kstep(std::integral_constant<int, 0>(), std::integral_constant<int, 8>());
            } else {
                (void)ks;
                kstep(std::integral_constant<int, 0>(), std::integral_constant<int, 8>());
            }
            if (more) stash(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
#pragma unroll
        for (int u = 0; u < TM / 2; ++u) {
            float2 s = make_float2(sig2[2 * u], sig2[2 * u + 1]);
#pragma unroll
            for (int v = 0; v < 8; ++v) s = fma2(acc[u][v], acc[u][v], s);
            sig2[2 * u] = s.x;
            sig2[2 * u + 1] = s.y;
        }
    }
#pragma unroll
    for (int u = 0; u < TM; ++u)
        for (int o = 1; o < 16; o <<= 1) sig2[u] += __shfl_xor_sync(0xffffffffu, sig2[u], o);
    const float tau = tau_dev ? (float)*tau_dev : (float)y_best;
    if (tx == 0) {
#pragma unroll
        for (int u = 0; u < TM; ++u) {
            const int r = ty * TM + u;
            const int64_t cl = cb + r, c = c0 + cl;
            float e = -1.0f;
            if (cl < C) {
                const float var = s2 - sig2[u];
                const float sg = var > 0.0f ? sqrtf(var) : 0.0f;
                e = ei_minf(mu[c], sg, tau, xi);
                if (sigma_out) sigma_out[c] = sg;
                if (ei_out) ei_out[c] = e;
            }
            red_v[r] = e;
            red_i[r] = cl < C ? c : INT64_MAX;
        }
    }
    __syncthreads();
    for (int s = BM / 2; s; s >>= 1) {
        for (int i = tid; i < s; i += blockDim.x)
            if (better(red_v[i + s], red_i[i + s], red_v[i], red_i[i])) {
                red_v[i] = red_v[i + s];
                red_i[i] = red_i[i + s];
            }
        __syncthreads();
    }
    if (tid == 0) {
        part_ei[part_base + bx] = red_v[0];
        part_idx[part_base + bx] = red_i[0];
    }
}

template <typename T>
__device__ __forceinline__ void k_argmax_final_body(const T *__restrict__ part_ei, const int64_t *__restrict__ part_idx,
                                                       int np, double *__restrict__ out_ei, int64_t *__restrict__ out_idx, const int bx, const int by, const int gx)
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


}  // namespace gpbo
