// Learned pre-screen: an ensemble of E small networks d -> H -> H -> 2 (exact GELU) trained
// on (x, GP posterior) pairs to predict (mu, log sigma) in standardised units; it scores a
// very large candidate pool cheaply, keeps the top k by the ensemble's expected improvement,
// and the exact GP-EI re-scores those k (the exact score is both the fallback and the measure
// of the screen's error).
//
// Ensemble combine (mean of the members, total variance):
//   mu_bar = mean_e mu_e,  sigma_bar^2 = mean_e sigma_e^2 + var_e mu_e.
// Training: L = 1/(2B) sum (o - t)^2 per network, Adam (lr, 0.9, 0.999, 1e-8), minibatches
// drawn with replacement from the counter stream, all E networks in the same launches; the
// step is captured once per call into a CUDA graph and replayed.
//
// Parameter layout per network (FP32, contiguous): W1 [d x H], b1 [H], W2 [H x H], b2 [H],
// W3 [H x 2], b3 [2] -- weights stored input-major, the same layout as the FP64 oracle.
#include "gpbo_internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

struct gpbo_mlp {
    gpbo_ctx *ctx = nullptr;
    int E = 0, d = 0, H = 0;
    int64_t P = 0;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    int64_t step = 0;
    double norm[4] = {0.0, 1.0, 0.0, 1.0};  // mu mean, mu sd, log-sigma mean, log-sigma sd
    // training buffers (sized for `cap` rows)
    int cap = 0;
    float *bx = nullptr, *bt = nullptr, *z1 = nullptr, *h1 = nullptr, *z2 = nullptr, *h2 = nullptr, *o = nullptr;
    float *d2 = nullptr, *d1 = nullptr, *dO = nullptr, *loss = nullptr;
    int64_t *dctr = nullptr;         // device step counters: [0] within this train call, [1] Adam steps
    cudaStream_t cap_stream = nullptr;  // private stream for capturing the training step
    // tensor-core operands (BF16 K-major weights + FP32 aux), rebuilt when theta changes
    void *wt16 = nullptr;
    float *aux = nullptr;
    int64_t version = 0, packed = -1;
};

namespace gpbo {

namespace mlp {

__device__ __forceinline__ float gelu(float z) { return z * 0.5f * erfcf(-z * 0.70710678f); }
__device__ __forceinline__ float gelu_grad(float z)
{
    return 0.5f * erfcf(-z * 0.70710678f) + z * 0.39894228f * expf(-0.5f * z * z);
}

struct Off {
    int64_t W1, b1, W2, b2, W3, b3;
};
__host__ __device__ inline Off offsets(int d, int H)
{
    Off f;
    f.W1 = 0;
    f.b1 = f.W1 + (int64_t)d * H;
    f.W2 = f.b1 + H;
    f.b2 = f.W2 + (int64_t)H * H;
    f.W3 = f.b2 + H;
    f.b3 = f.W3 + 2 * (int64_t)H;
    return f;
}

// Glorot-uniform weights from counter stream 5, zero biases.
__global__ void k_init(float *theta, int E, int d, int H, int64_t P, uint64_t seed)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)E * P) return;
    const int64_t i = t % P;
    const Off f = offsets(d, H);
    float fan_in = 0.f, fan_out = 0.f;
    bool bias = false;
    if (i < f.b1) { fan_in = d; fan_out = H; }
    else if (i < f.W2) bias = true;
    else if (i < f.b2) { fan_in = H; fan_out = H; }
    else if (i < f.W3) bias = true;
    else if (i < f.b3) { fan_in = H; fan_out = 2; }
    else bias = true;
    if (bias) { theta[t] = 0.0f; return; }
    const float a = sqrtf(6.0f / (fan_in + fan_out));
    theta[t] = (2.0f * uniform24f(seed, 5, (uint64_t)t) - 1.0f) * a;
}

// C[e] = epi( op(A[e]) op(B[e]) + bias[e] ), all row-major; op transposes when the flag is set.
// epi: 0 store C; 1 store Z = C + bias and H = gelu(Z) (Z may be null); 2 store C * gelu'(Zref).
// 64 x 64 CTA tile, K steps of 16; thread (ty, tx) owns the contiguous 4 x 4 block at rows
// 4 ty, columns 4 tx, read from transposed shared tiles 128 bits at a time; the next K step's
// global loads (128-bit where the operand is contiguous along the loaded dimension and in
// range) are held in registers while the current one is multiplied.  Each output sums over k
// in order, for any M, N, K.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm(const float *__restrict__ A, int64_t sA, int lda,
                                              const float *__restrict__ B, int64_t sB, int ldb, float *__restrict__ C,
                                              int64_t sC, int ldc, const float *__restrict__ bias, int64_t sbias,
                                              float *__restrict__ H, const float *__restrict__ Zref, int M, int N, int K,
                                              int epi)
{
    constexpr int BM = 64, BN = 64, BK = 16, PAD = 4;
    __shared__ __align__(16) float As[2][BK][BM + PAD];
    __shared__ __align__(16) float Bs[2][BK][BN + PAD];
    const int e = blockIdx.z;
    A += e * sA;
    B += e * sB;
    C += e * sC;
    if (H) H += e * sC;
    if (Zref) Zref += e * sC;
    if (bias) bias += e * sbias;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const bool va = ((uintptr_t)A % 16 == 0) && (lda % 4 == 0);
    const bool vb = ((uintptr_t)B % 16 == 0) && (ldb % 4 == 0);
    // loader roles: a quad of 4 consecutive elements along the operand's contiguous dimension
    //   A (M x K):  !TA -> row m = tid/4, k = 4 (tid%4);  TA -> k = tid/16, m = 4 (tid%16)
    //   B (K x N):  !TB -> k = tid/16, n = 4 (tid%16);    TB -> n = tid/4, k = 4 (tid%4)
    const int am = TA ? 4 * (tid % 16) : tid / 4, ak = TA ? tid / 16 : 4 * (tid % 4);
    const int bk = TB ? 4 * (tid % 4) : tid / 16, bn = TB ? tid / 4 : 4 * (tid % 16);
    float pa[4], pb[4];
    auto fetch = [&](int k0) {
        if (!TA) {
            const int gr = m0 + am, gc = k0 + ak;
            const float *src = A + (int64_t)gr * lda + gc;
            if (va && gr < M && gc + 3 < K) {
                const float4 f = *reinterpret_cast<const float4 *>(src);
                pa[0] = f.x; pa[1] = f.y; pa[2] = f.z; pa[3] = f.w;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) pa[q] = (gr < M && gc + q < K) ? src[q] : 0.f;
            }
        } else {
            const int gk = k0 + ak, gm = m0 + am;
            const float *src = A + (int64_t)gk * lda + gm;
            if (va && gk < K && gm + 3 < M) {
                const float4 f = *reinterpret_cast<const float4 *>(src);
                pa[0] = f.x; pa[1] = f.y; pa[2] = f.z; pa[3] = f.w;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) pa[q] = (gk < K && gm + q < M) ? src[q] : 0.f;
            }
        }
        if (!TB) {
            const int gk = k0 + bk, gn = n0 + bn;
            const float *src = B + (int64_t)gk * ldb + gn;
            if (vb && gk < K && gn + 3 < N) {
                const float4 f = *reinterpret_cast<const float4 *>(src);
                pb[0] = f.x; pb[1] = f.y; pb[2] = f.z; pb[3] = f.w;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) pb[q] = (gk < K && gn + q < N) ? src[q] : 0.f;
            }
        } else {
            const int gn = n0 + bn, gk = k0 + bk;
            const float *src = B + (int64_t)gn * ldb + gk;
            if (vb && gn < N && gk + 3 < K) {
                const float4 f = *reinterpret_cast<const float4 *>(src);
                pb[0] = f.x; pb[1] = f.y; pb[2] = f.z; pb[3] = f.w;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) pb[q] = (gn < N && gk + q < K) ? src[q] : 0.f;
            }
        }
    };
    auto stash = [&](int buf) {
        if (!TA) {
#pragma unroll
            for (int q = 0; q < 4; ++q) As[buf][ak + q][am] = pa[q];
        } else {
            *reinterpret_cast<float4 *>(&As[buf][ak][am]) = make_float4(pa[0], pa[1], pa[2], pa[3]);
        }
        if (!TB) {
            *reinterpret_cast<float4 *>(&Bs[buf][bk][bn]) = make_float4(pb[0], pb[1], pb[2], pb[3]);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) Bs[buf][bk + q][bn] = pb[q];
        }
    };
    float acc[4][4] = {};
    int buf = 0;
    if (K > 0) {
        fetch(0);
        stash(0);
    }
    __syncthreads();
    for (int k0 = 0; k0 < K; k0 += BK) {
        const bool more = k0 + BK < K;
        if (more) fetch(k0 + BK);
#pragma unroll
        for (int t = 0; t < BK; ++t) {
            const float4 x = *reinterpret_cast<const float4 *>(&As[buf][t][ty * 4]);
            const float4 y = *reinterpret_cast<const float4 *>(&Bs[buf][t][tx * 4]);
            const float xa[4] = {x.x, x.y, x.z, x.w}, ya[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[u][w] = fmaf(xa[u], ya[w], acc[u][w]);
        }
        if (more) stash(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int gr = m0 + ty * 4 + u, gc = n0 + tx * 4 + w;
            if (gr >= M || gc >= N) continue;
            const int64_t at = (int64_t)gr * ldc + gc;
            float v = acc[u][w] + (bias ? bias[gc] : 0.f);
            if (epi == 1) {
                if (C) C[at] = v;
                H[at] = gelu(v);
            } else if (epi == 2) {
                C[at] = v * gelu_grad(Zref[at]);
            } else {
                C[at] = v;
            }
        }
}

__global__ void k_out_grad(const float *o, const float *t, int B, float *dO, float *loss)
{
    const int e = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (i < 2 * B) {
        const float r = o[(int64_t)e * 2 * B + i] - t[i];
        dO[(int64_t)e * 2 * B + i] = r / B;
        l = 0.5f * r * r / B;
    }
    for (int s = 16; s; s >>= 1) l += __shfl_xor_sync(0xffffffffu, l, s);
    if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(loss + e, l);
}

// Column sums of a B x N row-major matrix (bias gradients): out[e][j] = sum_b X[e][b][j].
__global__ void k_colsum(const float *X, int64_t sX, int B, int N, float *out, int64_t sOut)
{
    const int e = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += X[e * sX + (int64_t)b * N + j];
    out[e * sOut + j] = s;
}

// Adam step t = adam_steps + 1 (bias corrections 1 - 0.9^t, 1 - 0.999^t).
__global__ void k_adam(float *theta, const float *g, float *m, float *v, int64_t count, float lr,
                       const int64_t *adam_steps)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float t = (float)(*adam_steps + 1);
    const float c1 = 1.0f - powf(0.9f, t), c2 = 1.0f - powf(0.999f, t);
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

// Minibatch: rows drawn with replacement (counter stream 7) from X (N x d) and the targets.
// Advance the step counters (after every kernel of the step has read them).
__global__ void k_step_inc(int64_t *ctr)
{
    ctr[0] += 1;
    ctr[1] += 1;
}

__global__ void k_gather_batch(const float *X, const float *T, int64_t N, int d, int B, uint64_t seed,
                               const int64_t *step_dev, float *bx, float *bt)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const uint64_t step = (uint64_t)*step_dev;
    const uint64_t r = splitmix64(seed, 7, step * (uint64_t)B + b);
    const int64_t i = (int64_t)((r >> 11) % (uint64_t)N);
    for (int k = 0; k < d; ++k) bx[(int64_t)b * d + k] = X[i * d + k];
    bt[2 * b] = T[2 * i];
    bt[2 * b + 1] = T[2 * i + 1];
}

// Targets: t0 = (mu - mean) / sd, t1 = (log sigma - mean) / sd, statistics over all N rows.
__global__ void __launch_bounds__(1024) k_target_stats(const float *mu, const float *sigma, int64_t N, double *stats)
{
    __shared__ double red[4][32];
    double s[4] = {0, 0, 0, 0};
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const double a = mu[i], b = log(fmax((double)sigma[i], 1e-30));
        s[0] += a; s[1] += a * a; s[2] += b; s[3] += b * b;
    }
    for (int q = 0; q < 4; ++q) {
        double v = s[q];
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[4] = {0, 0, 0, 0};
        for (int w = 0; w < (int)(blockDim.x / 32); ++w)
            for (int q = 0; q < 4; ++q) t[q] += red[q][w];
        const double m0 = t[0] / N, m1 = t[2] / N;
        const double sd0 = sqrt(fmax(t[1] / N - m0 * m0, 1e-24)), sd1 = sqrt(fmax(t[3] / N - m1 * m1, 1e-24));
        stats[0] = m0; stats[1] = sd0; stats[2] = m1; stats[3] = sd1;
    }
}

__global__ void k_make_targets(const float *mu, const float *sigma, int64_t N, const double *stats, float *T)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    T[2 * i] = (float)((mu[i] - stats[0]) / stats[1]);
    T[2 * i + 1] = (float)((log(fmax((double)sigma[i], 1e-30)) - stats[2]) / stats[3]);
}

// Ensemble EI per candidate from the networks' standardised outputs O [E][C][2]; the sums
// are taken about the first network's mean so that var_e mu_e does not cancel.
__global__ void k_ensemble_ei(const float *O, int E, int64_t C, int64_t c0, float n0, float n1, float n2, float n3,
                              float tau, float xi, float *ei, float *mu_out, float *sigma_out)
{
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= C) return;
    float shift = 0.f, sm = 0.f, sm2 = 0.f, sv = 0.f;
    for (int e = 0; e < E; ++e) {
        const float mu = O[((int64_t)e * C + c) * 2] * n1 + n0;
        const float ls = O[((int64_t)e * C + c) * 2 + 1] * n3 + n2;
        const float s = expf(ls);
        if (e == 0) shift = mu;
        const float dm = mu - shift;
        sm += dm;
        sm2 = fmaf(dm, dm, sm2);
        sv = fmaf(s, s, sv);
    }
    const float invE = 1.0f / (float)E, mm = sm * invE;
    const float mbar = shift + mm;
    const float sbar = sqrtf(sv * invE + fmaxf(sm2 * invE - mm * mm, 0.f));
    ei[c0 + c] = ei_minf(mbar, sbar, tau, xi);
    if (mu_out) mu_out[c0 + c] = mbar;
    if (sigma_out) sigma_out[c0 + c] = sbar;
}

__global__ void k_gen_rows(uint64_t seed, int64_t c0, int64_t C, int d, float *X)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= C * d) return;
    const int64_t c = t / d;
    const int k = (int)(t - c * d);
    X[t] = uniform24f(seed, 2, (uint64_t)((c0 + c) * d + k));
}

// ------------------------------------------------------------------ top-k (radix select)
// keys: EI >= 0 as float bits (order-preserving for non-negative floats); NaN counts as 0.
__device__ __forceinline__ uint32_t key_of(float v) { return v > 0.f ? __float_as_uint(v) : 0u; }

// pass p: histogram of digit p among keys whose higher digits equal the prefix chosen so far.
// digits: bits [20,32) (4096 bins), [8,20) (4096), [0,8) (256).
__global__ void k_radix_hist(const float *ei, int64_t M, int pass, const uint32_t *sel, uint32_t *hist)
{
    __shared__ uint32_t sh[4096];
    for (int i = threadIdx.x; i < 4096; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const uint32_t prefix = sel[0];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = key_of(ei[i]);
        uint32_t dig;
        bool in;
        if (pass == 0) { dig = k >> 20; in = true; }
        else if (pass == 1) { dig = (k >> 8) & 0xFFFu; in = (k >> 20) == prefix; }
        else { dig = k & 0xFFu; in = (k >> 8) == prefix; }
        if (in) atomicAdd(&sh[dig], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4096; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// Single thread: choose the digit where the running count from the top reaches `need`,
// extend the prefix, and leave the remaining count for the next pass.  sel = {prefix, need}.
__global__ void k_radix_pick(uint32_t *hist, int bins, int pass, uint32_t *sel)
{
    uint32_t need = sel[1];
    uint32_t cum = 0;
    int b = bins - 1;
    for (; b > 0; --b) {
        if (cum + hist[b] >= need) break;
        cum += hist[b];
    }
    const uint32_t shift = pass == 2 ? 8u : 12u;
    sel[0] = pass == 0 ? (uint32_t)b : (sel[0] << shift) | (uint32_t)b;
    sel[1] = need - cum;
    for (int i = 0; i < bins; ++i) hist[i] = 0;
}

// Keys above the threshold key T = sel[0] all go in; keys equal to T fill the remaining sel[1].
__global__ void k_radix_gather(const float *ei, int64_t M, const uint32_t *sel, uint32_t *counters, int k,
                               int64_t *out)
{
    const uint32_t T = sel[0];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t key = key_of(ei[i]);
        if (key > T) {
            const uint32_t p = atomicAdd(&counters[0], 1u);
            if (p < (uint32_t)k) out[p] = i;
        } else if (key == T) {
            const uint32_t q = atomicAdd(&counters[1], 1u);
            if (q < sel[1]) {
                const uint32_t p = atomicAdd(&counters[0], 1u);
                if (p < (uint32_t)k) out[p] = i;
            }
        }
    }
}

__global__ void k_rows_from_index(const int64_t *idx, int k, uint64_t seed, int d, float *X)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= k * d) return;
    const int r = t / d, c = t - r * d;
    X[t] = uniform24f(seed, 2, (uint64_t)(idx[r] * d + c));
}

}  // namespace mlp

using namespace mlp;

static unsigned nb(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, cdiv64(n, t)); }

static int ensure_batch(gpbo_mlp *net, int B)
{
    if (B <= net->cap) return GPBO_OK;
    float **bufs[] = {&net->bx, &net->bt, &net->z1, &net->h1, &net->z2, &net->h2, &net->o, &net->d2, &net->d1, &net->dO};
    for (float **b : bufs)
        if (*b) { cudaFree(*b); *b = nullptr; }
    const int64_t EBH = (int64_t)net->E * B * net->H;
    GPBO_CUDA_TRY(cudaMalloc(&net->bx, sizeof(float) * (size_t)B * net->d));
    GPBO_CUDA_TRY(cudaMalloc(&net->bt, sizeof(float) * (size_t)B * 2));
    GPBO_CUDA_TRY(cudaMalloc(&net->z1, sizeof(float) * EBH));
    GPBO_CUDA_TRY(cudaMalloc(&net->h1, sizeof(float) * EBH));
    GPBO_CUDA_TRY(cudaMalloc(&net->z2, sizeof(float) * EBH));
    GPBO_CUDA_TRY(cudaMalloc(&net->h2, sizeof(float) * EBH));
    GPBO_CUDA_TRY(cudaMalloc(&net->o, sizeof(float) * (size_t)net->E * B * 2));
    GPBO_CUDA_TRY(cudaMalloc(&net->d2, sizeof(float) * EBH));
    GPBO_CUDA_TRY(cudaMalloc(&net->d1, sizeof(float) * EBH));
    GPBO_CUDA_TRY(cudaMalloc(&net->dO, sizeof(float) * (size_t)net->E * B * 2));
    net->cap = B;
    return GPBO_OK;
}

// Forward of every network on B rows of X (shared by the networks).  keep: store Z for backward.
static int forward(gpbo_ctx *ctx, gpbo_mlp *net, const float *X, int B, float *z1, float *h1, float *z2, float *h2,
                   float *o, bool keep, cudaStream_t stream = nullptr)
{
    const int E = net->E, d = net->d, H = net->H;
    const Off f = offsets(d, H);
    const int64_t P = net->P, BH = (int64_t)B * H;
    cudaStream_t st = stream ? stream : ctx->stream;
    dim3 g1(nb(H, 64), nb(B, 64), E);
    k_gemm<false, false><<<g1, 256, 0, st>>>(X, 0, d, net->theta + f.W1, P, H, keep ? z1 : nullptr, BH, H,
                                             net->theta + f.b1, P, h1, nullptr, B, H, d, 1);
    GPBO_LAUNCH_CHECK(ctx);
    k_gemm<false, false><<<g1, 256, 0, st>>>(h1, BH, H, net->theta + f.W2, P, H, keep ? z2 : nullptr, BH, H,
                                             net->theta + f.b2, P, h2, nullptr, B, H, H, 1);
    GPBO_LAUNCH_CHECK(ctx);
    dim3 g3(1, nb(B, 64), E);
    k_gemm<false, false><<<g3, 256, 0, st>>>(h2, BH, H, net->theta + f.W3, P, 2, o, (int64_t)B * 2, 2,
                                             net->theta + f.b3, P, nullptr, nullptr, B, 2, H, 0);
    GPBO_LAUNCH_CHECK(ctx);
    return GPBO_OK;
}

// Gradients of every network for the batch in net->bx / net->bt (B rows) into net->grad.
static int backward(gpbo_ctx *ctx, gpbo_mlp *net, int B, cudaStream_t stream = nullptr)
{
    const int E = net->E, d = net->d, H = net->H;
    const Off f = offsets(d, H);
    const int64_t P = net->P, BH = (int64_t)B * H;
    cudaStream_t st = stream ? stream : ctx->stream;
    GPBO_TRY(forward(ctx, net, net->bx, B, net->z1, net->h1, net->z2, net->h2, net->o, true, st));
    GPBO_CUDA_TRY(cudaMemsetAsync(net->loss, 0, sizeof(float) * E, st));
    k_out_grad<<<dim3(nb(2 * B), E), 256, 0, st>>>(net->o, net->bt, B, net->dO, net->loss);
    GPBO_LAUNCH_CHECK(ctx);
    float *G = net->grad;
    // dW3 = h2^T dO, db3 = sum dO
    k_gemm<true, false><<<dim3(1, nb(H, 64), E), 256, 0, st>>>(net->h2, BH, H, net->dO, (int64_t)B * 2, 2, G + f.W3, P, 2,
                                                               nullptr, 0, nullptr, nullptr, H, 2, B, 0);
    GPBO_LAUNCH_CHECK(ctx);
    k_colsum<<<dim3(1, E), 32, 0, st>>>(net->dO, (int64_t)B * 2, B, 2, G + f.b3, P);
    GPBO_LAUNCH_CHECK(ctx);
    // dZ2 = (dO W3^T) * gelu'(z2)
    k_gemm<false, true><<<dim3(nb(H, 64), nb(B, 64), E), 256, 0, st>>>(net->dO, (int64_t)B * 2, 2, net->theta + f.W3, P, 2,
                                                                       net->d2, BH, H, nullptr, 0, nullptr, net->z2, B,
                                                                       H, 2, 2);
    GPBO_LAUNCH_CHECK(ctx);
    // dW2 = h1^T dZ2, db2 = sum dZ2
    k_gemm<true, false><<<dim3(nb(H, 64), nb(H, 64), E), 256, 0, st>>>(net->h1, BH, H, net->d2, BH, H, G + f.W2, P, H,
                                                                       nullptr, 0, nullptr, nullptr, H, H, B, 0);
    GPBO_LAUNCH_CHECK(ctx);
    k_colsum<<<dim3(nb(H), E), 256, 0, st>>>(net->d2, BH, B, H, G + f.b2, P);
    GPBO_LAUNCH_CHECK(ctx);
    // dZ1 = (dZ2 W2^T) * gelu'(z1)
    k_gemm<false, true><<<dim3(nb(H, 64), nb(B, 64), E), 256, 0, st>>>(net->d2, BH, H, net->theta + f.W2, P, H, net->d1,
                                                                       BH, H, nullptr, 0, nullptr, net->z1, B, H, H, 2);
    GPBO_LAUNCH_CHECK(ctx);
    // dW1 = x^T dZ1, db1 = sum dZ1
    k_gemm<true, false><<<dim3(nb(H, 64), nb(d, 64), E), 256, 0, st>>>(net->bx, 0, d, net->d1, BH, H, G + f.W1, P, H,
                                                                       nullptr, 0, nullptr, nullptr, d, H, B, 0);
    GPBO_LAUNCH_CHECK(ctx);
    k_colsum<<<dim3(nb(H), E), 256, 0, st>>>(net->d1, BH, B, H, G + f.b1, P);
    GPBO_LAUNCH_CHECK(ctx);
    return GPBO_OK;
}

static int ensure_packed(gpbo_ctx *ctx, gpbo_mlp *net)
{
    if (!mlp_tc_usable(net->d, net->H, net->E)) return GPBO_ENOTSUP;
    if (!net->wt16) {
        GPBO_CUDA_TRY(cudaMalloc(&net->wt16, mlp_tc_weight_bytes(net->E)));
        GPBO_CUDA_TRY(cudaMalloc(&net->aux, sizeof(float) * mlp_tc_aux_floats(net->E)));
    }
    if (net->packed != net->version) {
        const Off f = offsets(net->d, net->H);
        const int64_t off[6] = {f.W1, f.b1, f.W2, f.b2, f.W3, f.b3};
        GPBO_TRY(mlp_tc_pack(ctx, net->theta, net->E, net->d, net->P, off, net->wt16, net->aux));
        net->packed = net->version;
    }
    return GPBO_OK;
}

// Ensemble (mu_bar, sigma_bar, EI) for M candidates: rows of X (device) or, when X is null,
// pool candidates 0 .. M-1 drawn from seed.  F16: one tensor-core launch; F32: CUDA-core
// forward in chunks.  Outputs are pool-indexed device arrays (mu, sigma may be null).
static int score_pool(gpbo_ctx *ctx, gpbo_mlp *net, const float *X, int64_t M, uint64_t seed, double tau, double xi,
                      int prec, float *ei, float *mu, float *sigma)
{
    cudaStream_t st = ctx->stream;
    const double *nm = net->norm;
    if (prec == GPBO_PREC_F16) {
        GPBO_TRY(ensure_packed(ctx, net));
        return mlp_tc_score(ctx, net->wt16, net->aux, net->E, net->d, nm, X, seed, 0, M, tau, xi, ei, mu, sigma);
    }
    if (prec != GPBO_PREC_F32) return GPBO_EINVAL;
    const int C = 32768;  // candidates per chunk
    GPBO_TRY(ensure_batch(net, C));
    for (int64_t c0 = 0; c0 < M; c0 += C) {
        const int Cc = (int)std::min<int64_t>(C, M - c0);
        const float *xb = X ? X + c0 * net->d : net->bx;
        if (!X) {
            k_gen_rows<<<nb((int64_t)Cc * net->d), 256, 0, st>>>(seed, c0, Cc, net->d, net->bx);
            GPBO_LAUNCH_CHECK(ctx);
        }
        GPBO_TRY(forward(ctx, net, xb, Cc, nullptr, net->h1, nullptr, net->h2, net->o, false));
        k_ensemble_ei<<<nb(Cc), 256, 0, st>>>(net->o, net->E, Cc, c0, (float)nm[0], (float)nm[1], (float)nm[2],
                                              (float)nm[3], (float)tau, (float)xi, ei, mu, sigma);
        GPBO_LAUNCH_CHECK(ctx);
    }
    return GPBO_OK;
}

}  // namespace gpbo

using namespace gpbo;

extern "C" {

int mlp_create(gpbo_ctx *ctx, int E, int d, int H, uint64_t seed, gpbo_mlp **out)
{
    if (!ctx || !out || E < 1 || E > 64 || d < 1 || d > GPBO_MAX_D || H < 1 || H > 4096) return GPBO_EINVAL;
    GPBO_CUDA_TRY(cudaSetDevice(ctx->device));
    gpbo_mlp *net = new gpbo_mlp();
    net->ctx = ctx;
    net->E = E;
    net->d = d;
    net->H = H;
    net->P = (int64_t)d * H + H + (int64_t)H * H + H + 2 * (int64_t)H + 2;
    const size_t bytes = sizeof(float) * (size_t)E * net->P;
    if (cudaMalloc(&net->theta, bytes) != cudaSuccess || cudaMalloc(&net->grad, bytes) != cudaSuccess ||
        cudaMalloc(&net->m, bytes) != cudaSuccess || cudaMalloc(&net->v, bytes) != cudaSuccess ||
        cudaMalloc(&net->loss, sizeof(float) * E) != cudaSuccess ||
        cudaMalloc(&net->dctr, sizeof(int64_t) * 2) != cudaSuccess) {
        mlp_free(net);
        return GPBO_ENOMEM;
    }
    cudaMemsetAsync(net->m, 0, bytes, ctx->stream);
    cudaMemsetAsync(net->v, 0, bytes, ctx->stream);
    k_init<<<nb((int64_t)E * net->P), 256, 0, ctx->stream>>>(net->theta, E, d, H, net->P, seed);
    ctx->launches++;
    if (cudaGetLastError() != cudaSuccess) {
        mlp_free(net);
        return GPBO_ECUDA;
    }
    *out = net;
    return GPBO_OK;
}

int mlp_free(gpbo_mlp *net)
{
    if (!net) return GPBO_EINVAL;
    cudaStreamSynchronize(net->ctx->stream);
    float *bufs[] = {net->theta, net->grad, net->m,  net->v,  net->loss, net->bx, net->bt,
                     net->z1,    net->h1,   net->z2, net->h2, net->o,    net->d2, net->d1, net->dO};
    for (float *b : bufs)
        if (b) cudaFree(b);
    if (net->wt16) cudaFree(net->wt16);
    if (net->aux) cudaFree(net->aux);
    if (net->dctr) cudaFree(net->dctr);
    if (net->cap_stream) cudaStreamDestroy(net->cap_stream);
    delete net;
    return GPBO_OK;
}

int mlp_params(gpbo_mlp *net, float *host_out, const float *host_in)
{
    if (!net) return GPBO_EINVAL;
    gpbo_ctx *ctx = net->ctx;
    const size_t bytes = sizeof(float) * (size_t)net->E * net->P;
    if (host_in) {
        GPBO_CUDA_TRY(cudaMemcpyAsync(net->theta, host_in, bytes, cudaMemcpyHostToDevice, ctx->stream));
        net->version++;
    }
    if (host_out) GPBO_CUDA_TRY(cudaMemcpyAsync(host_out, net->theta, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    GPBO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return GPBO_OK;
}

int mlp_forward(gpbo_ctx *ctx, gpbo_mlp *net, const float *X, int B, float *out)
{
    if (!ctx || !net || !X || !out || B < 1) return GPBO_EINVAL;
    GPBO_TRY(ensure_batch(net, B));
    GPBO_TRY(forward(ctx, net, X, B, nullptr, net->h1, nullptr, net->h2, out, false));
    GPBO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return GPBO_OK;
}

int mlp_gradients(gpbo_ctx *ctx, gpbo_mlp *net, const float *X, const float *T, int B, float *grads_host,
                  float *loss_host)
{
    if (!ctx || !net || !X || !T || B < 1) return GPBO_EINVAL;
    GPBO_TRY(ensure_batch(net, B));
    GPBO_CUDA_TRY(cudaMemcpyAsync(net->bx, X, sizeof(float) * (size_t)B * net->d, cudaMemcpyDeviceToDevice, ctx->stream));
    GPBO_CUDA_TRY(cudaMemcpyAsync(net->bt, T, sizeof(float) * (size_t)B * 2, cudaMemcpyDeviceToDevice, ctx->stream));
    GPBO_TRY(backward(ctx, net, B));
    if (grads_host)
        GPBO_CUDA_TRY(cudaMemcpyAsync(grads_host, net->grad, sizeof(float) * (size_t)net->E * net->P,
                                      cudaMemcpyDeviceToHost, ctx->stream));
    if (loss_host)
        GPBO_CUDA_TRY(cudaMemcpyAsync(loss_host, net->loss, sizeof(float) * net->E, cudaMemcpyDeviceToHost, ctx->stream));
    GPBO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return GPBO_OK;
}

int mlp_train(gpbo_ctx *ctx, gpbo_mlp *net, const float *X, const float *mu, const float *sigma, int64_t N, int steps,
              int batch, float lr, uint64_t seed, float *final_loss)
{
    if (!ctx || !net || !X || !mu || !sigma || N < 1 || steps < 1 || batch < 1 || !(lr > 0)) return GPBO_EINVAL;
    GPBO_TRY(ensure_batch(net, batch));
    float *T = nullptr;
    double *stats = nullptr;
    GPBO_CUDA_TRY(cudaMalloc(&T, sizeof(float) * 2 * (size_t)N));
    GPBO_CUDA_TRY(cudaMalloc(&stats, sizeof(double) * 4));
    cudaStream_t st = ctx->stream;
    k_target_stats<<<1, 1024, 0, st>>>(mu, sigma, N, stats);
    GPBO_LAUNCH_CHECK(ctx);
    k_make_targets<<<nb(N), 256, 0, st>>>(mu, sigma, N, stats, T);
    GPBO_LAUNCH_CHECK(ctx);
    int rc = GPBO_OK;
    const int64_t count = (int64_t)net->E * net->P;
    // One training step (minibatch draw, forward, backward, Adam, counter advance) is captured
    // once into a CUDA graph on a private stream and replayed `steps` times on the context's
    // stream; the step counters live on the device so every replay draws its own batch.
    const int64_t ctr0[2] = {0, net->step};
    GPBO_CUDA_TRY(cudaMemcpyAsync(net->dctr, ctr0, sizeof(ctr0), cudaMemcpyHostToDevice, st));
    if (!net->cap_stream) GPBO_CUDA_TRY(cudaStreamCreateWithFlags(&net->cap_stream, cudaStreamNonBlocking));
    const int64_t launches0 = ctx->launches;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    GPBO_CUDA_TRY(cudaStreamBeginCapture(net->cap_stream, cudaStreamCaptureModeThreadLocal));
    {
        cudaStream_t cs = net->cap_stream;
        k_gather_batch<<<nb(batch), 256, 0, cs>>>(X, T, N, net->d, batch, seed, net->dctr, net->bx, net->bt);
        ctx->launches++;
        rc = backward(ctx, net, batch, cs);
        k_adam<<<nb(count), 256, 0, cs>>>(net->theta, net->grad, net->m, net->v, count, lr, net->dctr + 1);
        k_step_inc<<<1, 1, 0, cs>>>(net->dctr);
        ctx->launches += 2;
    }
    cudaError_t ce = cudaStreamEndCapture(net->cap_stream, &graph);
    if (rc == GPBO_OK && ce != cudaSuccess) rc = GPBO_ECUDA;
    if (rc == GPBO_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) rc = GPBO_ECUDA;
    const int64_t per_step = ctx->launches - launches0;
    for (int s = 0; s < steps && rc == GPBO_OK; ++s)
        if (cudaGraphLaunch(exec, st) != cudaSuccess) rc = GPBO_ECUDA;
    if (rc == GPBO_OK) ctx->launches += per_step * (steps - 1);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (rc == GPBO_OK) net->step += steps;
    net->version++;
    if (rc == GPBO_OK && cudaGetLastError() != cudaSuccess) rc = GPBO_ECUDA;
    double hs[4];
    if (rc == GPBO_OK && cudaMemcpyAsync(hs, stats, sizeof(hs), cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = GPBO_ECUDA;
    std::vector<float> l(net->E);
    if (rc == GPBO_OK && cudaMemcpyAsync(l.data(), net->loss, sizeof(float) * net->E, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = GPBO_ECUDA;
    cudaStreamSynchronize(st);
    cudaFree(T);
    cudaFree(stats);
    if (rc != GPBO_OK) return rc;
    for (int q = 0; q < 4; ++q) net->norm[q] = hs[q];
    if (final_loss) {
        double m = 0;
        for (float x : l) m += x;
        *final_loss = (float)(m / net->E);
    }
    return GPBO_OK;
}

int mlp_norm(const gpbo_mlp *net, double *norm4)
{
    if (!net || !norm4) return GPBO_EINVAL;
    for (int q = 0; q < 4; ++q) norm4[q] = net->norm[q];
    return GPBO_OK;
}

int mlp_score(gpbo_ctx *ctx, gpbo_mlp *net, const float *X, int64_t M, uint64_t seed, double y_best, double xi, int prec,
              float *ei, float *mu, float *sigma)
{
    if (!ctx || !net || !ei || M < 1 || M > 0x7fffffffll) return GPBO_EINVAL;
    if (prec == GPBO_PREC_BF16) return GPBO_ENOTSUP;  // the tensor-core forward uses FP16 operands
    if (prec != GPBO_PREC_F16 && prec != GPBO_PREC_F32) return GPBO_EINVAL;
    GPBO_CUDA_TRY(cudaSetDevice(ctx->device));
    GPBO_TRY(score_pool(ctx, net, X, M, seed, y_best, xi, prec, ei, mu, sigma));
    GPBO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    unsigned bits = 0;
    GPBO_TRY(take_device_status(ctx, &bits));
    if (bits & DEV_TIMEOUT) return GPBO_ETIMEOUT;
    return GPBO_OK;
}

int surrogate_screen(gpbo_ctx *ctx, const gp_model *model, gpbo_mlp *net, int64_t M, uint64_t seed, int k,
                     double y_best, double xi, float *ei_pool, int64_t *top_idx, int64_t *argmax, double *ei_max)
{
    if (!ctx || !model || !net || !argmax || !ei_max || M < 1 || M > 0x7fffffffll || k < 1 || k > 1 << 20 ||
        (int64_t)k > M || net->d != model->d)
        return GPBO_EINVAL;
    if (model->prec == GPBO_PREC_F64) return GPBO_ENOTSUP;
    GPBO_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const int d = net->d;
    float *ei = ei_pool;
    float *own = nullptr;
    int64_t *idx = nullptr;
    uint32_t *hist = nullptr;
    float *Xk = nullptr;
    int rc = GPBO_OK;
    auto dalloc = [&](void **p, size_t bytes) {
        if (rc != GPBO_OK) return;
        const cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            note_cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
            rc = e == cudaErrorMemoryAllocation ? GPBO_ENOMEM : GPBO_ECUDA;
        }
    };
    if (!ei) {
        dalloc((void **)&own, sizeof(float) * (size_t)M);
        ei = own;
    }
    dalloc((void **)&idx, sizeof(int64_t) * (size_t)k);
    dalloc((void **)&hist, sizeof(uint32_t) * (4096 + 4));
    dalloc((void **)&Xk, sizeof(float) * (size_t)k * d);
    uint32_t *sel = hist + 4096, *counters = hist + 4098;
    const int prec = mlp_tc_usable(d, net->H, net->E) ? GPBO_PREC_F16 : GPBO_PREC_F32;
    if (rc == GPBO_OK) rc = score_pool(ctx, net, nullptr, M, seed, y_best, xi, prec, ei, nullptr, nullptr);
    if (rc == GPBO_OK) {
        // a bounded wait that gave up in the network's forward leaves part of the pool unscored:
        // report it here rather than select from it (or leave the bit for a later call)
        unsigned bits = 0;
        rc = take_device_status(ctx, &bits);
        if (rc == GPBO_OK && (bits & DEV_TIMEOUT)) rc = GPBO_ETIMEOUT;
    }
    // top k by the surrogate's EI
    if (rc == GPBO_OK) {
        uint32_t init[8] = {0, (uint32_t)k, 0, 0, 0, 0, 0, 0};
        cudaMemsetAsync(hist, 0, sizeof(uint32_t) * 4096, st);
        cudaMemcpyAsync(sel, init, sizeof(uint32_t) * 4, cudaMemcpyHostToDevice, st);
        for (int pass = 0; pass < 3; ++pass) {
            k_radix_hist<<<std::min<unsigned>(nb(M), ctx->sm_count * 8), 256, 0, st>>>(ei, M, pass, sel, hist);
            k_radix_pick<<<1, 1, 0, st>>>(hist, pass == 2 ? 256 : 4096, pass, sel);
            ctx->launches += 2;
        }
        k_radix_gather<<<std::min<unsigned>(nb(M), ctx->sm_count * 8), 256, 0, st>>>(ei, M, sel, counters, k, idx);
        k_rows_from_index<<<nb((int64_t)k * d), 256, 0, st>>>(idx, k, seed, d, Xk);
        ctx->launches += 2;
        if (cudaGetLastError() != cudaSuccess) rc = GPBO_ECUDA;
    }
    int64_t am = -1;
    double em = 0.0;
    if (rc == GPBO_OK) rc = score_model(ctx, model, Xk, k, 0, y_best, nullptr, xi, nullptr, nullptr, nullptr, &am, &em);
    if (rc == GPBO_OK) {
        int64_t pool = -1;
        if (cudaMemcpyAsync(&pool, idx + am, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = GPBO_ECUDA;
        if (top_idx && rc == GPBO_OK &&
            cudaMemcpyAsync(top_idx, idx, sizeof(int64_t) * (size_t)k, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            rc = GPBO_ECUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) rc = GPBO_ECUDA;
        *argmax = pool;
        *ei_max = em;
    }
    cudaStreamSynchronize(st);
    if (idx) cudaFree(idx);
    if (hist) cudaFree(hist);
    if (Xk) cudaFree(Xk);
    if (own) cudaFree(own);
    return rc;
}

}  // extern "C"
