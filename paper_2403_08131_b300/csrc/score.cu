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
#include "score_kernels.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <mutex>

namespace gpbo {

__global__ void k_gen_candidates(uint64_t seed, int64_t first, int64_t M, int d, float *__restrict__ out)
{
    k_gen_candidates_body(seed, first, M, d, out, blockIdx.x, blockIdx.y, gridDim.x);
}

int gen_candidates(gpbo_ctx *ctx, uint64_t seed, int64_t first, int64_t M, int d, float *out)
{
    int64_t total = M * d;
    unsigned grid = (unsigned)std::min<int64_t>(cdiv64(total, 256), (int64_t)ctx->sm_count * 16);
    k_gen_candidates<<<std::max(1u, grid), 256, 0, ctx->stream>>>(seed, first, M, d, out);
    GPBO_LAUNCH_CHECK(ctx);
    return GPBO_OK;
}

template <typename Acc, typename Out>
__global__ void __launch_bounds__(256) k_xkern(const float *__restrict__ Xc, uint64_t seed, int64_t c0, int64_t C,
                                               int d, const Acc *__restrict__ Xs, const Acc *__restrict__ alpha,
                                               int n, int n_pad, Acc s2, Lengthscales_inv ls, Out *__restrict__ Kst,
                                               Acc *__restrict__ mu)
{
    k_xkern_body<Acc, Out>(Xc, seed, c0, C, d, Xs, alpha, n, n_pad, s2, ls, Kst, mu, blockIdx.x, blockIdx.y, gridDim.x);
}

template <typename Out>
__global__ void __launch_bounds__(256, 4) k_xkern32(const float *__restrict__ Xc, uint64_t seed, int64_t c0, int64_t C,
                                                 int d, const float *__restrict__ Xs, const float *__restrict__ alpha,
                                                 int n, int n_pad, float s2, Lengthscales_inv ls, Out *__restrict__ Kst,
                                                 float *__restrict__ mu)
{
    k_xkern32_body<Out>(Xc, seed, c0, C, d, Xs, alpha, n, n_pad, s2, ls, Kst, mu, blockIdx.x, blockIdx.y, gridDim.x);
}

// Candidates per CTA of the variance kernel: FP32 uses the 128-candidate tile of
// k_var_f32_body, FP64 the 64-candidate k_var_simt_body.
constexpr int VAR_BM32 = 128;
template <typename T> constexpr int var_bm() { return sizeof(T) == 4 ? VAR_BM32 : 64; }

template <typename T>
__global__ void __launch_bounds__(256, 2) k_var_simt(const T *__restrict__ Kst, int64_t C, int64_t c0, int n_pad,
                                                  const T *__restrict__ Linv, const T *__restrict__ mu, T s2,
                                                  double y_best, const double *__restrict__ tau_dev, T xi,
                                                  T *__restrict__ sigma_out, T *__restrict__ ei_out,
                                                  T *__restrict__ part_ei, int64_t *__restrict__ part_idx,
                                                  int part_base)
{
    if constexpr (sizeof(T) == 4)
        k_var_f32_body<VAR_BM32>(Kst, C, c0, n_pad, Linv, mu, s2, y_best, tau_dev, xi, sigma_out, ei_out, part_ei,
                                 part_idx, part_base, blockIdx.x);
    else
        k_var_simt_body<T>(Kst, C, c0, n_pad, Linv, mu, s2, y_best, tau_dev, xi, sigma_out, ei_out, part_ei, part_idx,
                           part_base, blockIdx.x, blockIdx.y, gridDim.x);
}

template <typename T>
__global__ void __launch_bounds__(1024) k_argmax_final(const T *__restrict__ part_ei, const int64_t *__restrict__ part_idx,
                                                       int np, double *__restrict__ out_ei, int64_t *__restrict__ out_idx)
{
    k_argmax_final_body<T>(part_ei, part_idx, np, out_ei, out_idx, blockIdx.x, blockIdx.y, gridDim.x);
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
        const size_t smem = sizeof(float) * (192 * (size_t)m->d + 128);
        GPBO_TRY(ensure_smem((const void *)k_xkern32<Out>, ctx->device, (int)smem));
        k_xkern32<Out><<<(unsigned)cdiv64(C, 64), 256, smem, ctx->stream>>>(Xc, seed, c0, C, m->d, Xs, alpha, m->n,
                                                                             m->n_pad, (float)m->s2, ls, Kst, mu);
        GPBO_LAUNCH_CHECK(ctx);
        return GPBO_OK;
    }
    const size_t smem = sizeof(Acc) * ((size_t)32 * m->d + (size_t)m->d * 128 + 128);
    GPBO_TRY(ensure_smem((const void *)k_xkern<Acc, Out>, ctx->device, (int)smem));
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
    if constexpr (sizeof(T) == 4) {
        // whole waves of the FP32 variance kernel (two CTAs of VAR_BM32 candidates per SM), so
        // that no chunk ends on a partly filled wave
        const int64_t wave = (int64_t)2 * ctx->sm_count * VAR_BM32;
        if (C < M && C >= wave) C = C / wave * wave;
    }
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
        const unsigned g = (unsigned)cdiv64(Cc, var_bm<T>());
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
        const unsigned g = (unsigned)cdiv64(Cc, var_bm<T>());
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

