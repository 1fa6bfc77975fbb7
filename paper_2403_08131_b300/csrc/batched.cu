// Batched BO step: G independent sub-searches of uneven dimension and size in one graph
// launch.  The paper runs the independent and merged searches that its interdependence
// analysis produces in parallel (§IV-D, "which can be conducted in parallel"); here every
// kernel of the step covers all G problems at once (blockIdx.y = problem), with the same
// device bodies as the single-problem path, so each problem's results are bit-identical to
// a search_step call on it.  The whole sequence is captured once per set of shapes into a
// CUDA graph; later calls copy the new inputs and replay it.
//
// Work per step: standardise y, kernel matrix, blocked FP64 Cholesky (step k for every
// problem with more than k blocks), refined alpha, FP32 L^-1 (one merged recursion plan),
// FP32 cross-kernel + mean, FP32 variance + EI, per-problem argmax and x_next.
#include "fit_kernels.cuh"
#include "score_kernels.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <vector>

namespace gpbo {

struct BProb {
    int n, d, n_pad, nblk;
    int64_t M;
    uint64_t seed;
    double s2, sn2;
    int64_t off_X, off_y, off_xs, off_sq, off_dinv, off_vec, off_kst, off_mu, off_part, off_rpart;
    int part_count;
    int chunks;  // row chunks of the refinement's X^T u
    // this call's device inputs (n x d, n), gathered into the arenas by the graph's first
    // kernel; null when the host copied them (host inputs)
    const double *X_src, *y_src;
};

struct BatchPlan {
    // shapes (the set that owns the plan holds the key)
    int G = 0;
    std::vector<int> n, d;
    std::vector<int64_t> M;
    double xi = 0.0;     // baked into the captured graph
    // arenas
    BProb *probs_dev = nullptr;
    std::vector<BProb> probs;
    double *dX = nullptr, *dy = nullptr, *dys = nullptr, *tau = nullptr;
    double *Xs64 = nullptr, *K = nullptr, *L = nullptr, *Dinv = nullptr, *vec = nullptr, *lsinv = nullptr;
    double *rpart = nullptr;  // the refinement's row-chunk partial sums
    float *Xs32 = nullptr, *alpha32 = nullptr, *L32 = nullptr, *Linv32 = nullptr, *tmp = nullptr, *Kst = nullptr;
    float *mu = nullptr, *pei = nullptr;
    int64_t *pidx = nullptr;
    double *best_ei = nullptr;
    int64_t *best_idx = nullptr;
    float *xnext = nullptr;
    GemmProb *gemm_dev = nullptr;
    // tensor-core trailing updates (problems with n_pad >= CHOL_TC_UPDATE_MIN_NPAD): every such
    // problem's 7 BF16 slices of a panel in one arena, one pair of tensor maps over it
    CholTcProb *tc_probs = nullptr;
    std::vector<CholTcProb> tc_host;
    void *tc_slices = nullptr;
    int *tc_exps = nullptr;
    alignas(64) unsigned char tc_maps[2][128];
    std::vector<int> lvl_first, lvl_count;
    std::vector<int2> lvl_mm;
    int64_t sum_vec = 0;
    int max_npad = 0, max_nblk = 0, max_tiles64 = 0, max_chunks = 0;
    int64_t max_M = 0;
    int64_t max_sq = 0, max_dn = 0;
    int max_d = 1;                        // the widest problem's d
    int tile_req = 0;    // requested variance tile (0: autotune)
    int var_bm = 128;    // variance tile in use: candidates per CTA
    float tune_ms[3] = {-1.f, -1.f, -1.f};  // autotuner's times for 64, 128, 256
    cudaStream_t cap = nullptr;
    cudaStream_t cap2 = nullptr;     // second capture stream: lookahead column, alpha solve
    cudaStream_t cap3 = nullptr;     // third: the FP64 trailing updates beside the tensor-core ones
    cudaEvent_t ev[7] = {};          // fork / join events between the capture streams
    int64_t kernels = 0;             // kernel nodes in the captured graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<void *> allocs;
};

// ------------------------------------------------------------------ batched kernels
__device__ __forceinline__ Lengthscales_inv ls_of(const double *lsinv, int g, int d)
{
    Lengthscales_inv ls;
    for (int k = 0; k < d; ++k) ls.inv[k] = lsinv[g * GPBO_MAX_D + k];
    return ls;
}

// The call's device inputs into the arenas (one launch for all problems instead of two copies
// each); problems whose inputs the host copied have null sources.
__global__ void b_load_inputs(const BProb *P, double *X, double *y)
{
    const BProb &p = P[blockIdx.y];
    if (!p.X_src) return;
    const int64_t nd = (int64_t)p.n * p.d;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nd + p.n; t += (int64_t)gridDim.x * blockDim.x) {
        if (t < nd) X[p.off_X + t] = p.X_src[t];
        else y[p.off_y + (t - nd)] = p.y_src[t - nd];
    }
}

__global__ void __launch_bounds__(1024) b_standardize(const BProb *P, const double *y, double *ys, double *tau)
{
    const BProb &p = P[blockIdx.x];
    k_standardize_body(y + p.off_y, p.n, ys + p.off_y, tau + blockIdx.x, 0, 0);
}

__global__ void b_scale_x(const BProb *P, const double *X, const double *lsinv, double *Xs64, float *Xs32)
{
    const BProb &p = P[blockIdx.y];
    if ((int64_t)blockIdx.x * blockDim.x >= (int64_t)p.d * p.n_pad) return;
    k_scale_x_body(X + p.off_X, p.n, p.d, p.n_pad, ls_of(lsinv, blockIdx.y, p.d), Xs64 + p.off_xs, Xs32 + p.off_xs,
                   blockIdx.x, 0);
}

__global__ void b_kmat(const BProb *P, const double *Xs64, double *K)
{
    const BProb &p = P[blockIdx.z];
    const int nt = p.n_pad / 32;
    if ((int)blockIdx.x >= nt || (int)blockIdx.y >= nt) return;
    k_kmat_body(Xs64 + p.off_xs, p.n, p.d, p.n_pad, p.s2, p.sn2, K + p.off_sq, blockIdx.x, blockIdx.y);
}

__global__ void __launch_bounds__(256) b_chol_diag(const BProb *P, double *L, double *Dinv, int kb, unsigned *status)
{
    const BProb &p = P[blockIdx.y];
    if (kb >= p.nblk) return;
    k_chol_diag_body(L + p.off_sq, p.n_pad, kb, Dinv + p.off_dinv, status, 0, 0);
}

__global__ void __launch_bounds__(128) b_chol_inv(const BProb *P, const double *L, double *Dinv, int kb)
{
    const BProb &p = P[blockIdx.y];
    if (kb >= p.nblk) return;
    k_chol_inv_body(L + p.off_sq, p.n_pad, kb, Dinv + p.off_dinv, blockIdx.x);
}

__global__ void __launch_bounds__(128) b_chol_panel(const BProb *P, double *L, const double *Dinv, int kb)
{
    const BProb &p = P[blockIdx.y];
    const int T = p.nblk - kb - 1;
    if (T <= 0 || (int)blockIdx.x >= T * (NB / 4)) return;
    k_chol_panel_body(L + p.off_sq, p.n_pad, kb, Dinv + p.off_dinv, blockIdx.x, 0);
}

// The FP64 trailing updates in slabs of B_SLAB_ROWS rows (16 CTAs per 64 x 64 tile), as the
// single-problem path's next-column and small updates: the same arithmetic per element as a
// whole tile, without one CTA per tile holding a late, small step to 64^3 FP64 FMAs on one SM.
// part 1: block column kb+1 (T tiles); part 2: block columns kb+2 .. (T(T-1)/2 tiles), except
// problems whose step kb runs on the tensor cores.
constexpr int B_SLAB_ROWS = 4;
__global__ void __launch_bounds__(256) b_chol_update_slab(const BProb *P, double *L, int kb, int part)
{
    const BProb &p = P[blockIdx.y];
    const int T = p.nblk - kb - 1;
    const int64_t tiles = part == 1 ? T : (int64_t)T * (T - 1) / 2;
    if (T <= 0 || (int64_t)(blockIdx.x / (NB / B_SLAB_ROWS)) >= tiles) return;
    if (part == 2 && chol_tc_step(p.n_pad, p.nblk, kb)) return;
    k_chol_update_slab_body<B_SLAB_ROWS>(L + p.off_sq, p.n_pad, kb, blockIdx.x, part, 0);
}

// Between the factorisation and the inverse's levels, one pass over each problem's n_pad^2
// elements (grid-stride, so a small problem's share of the grid is not idle blocks): the blocks
// of L above its block diagonal set to zero, L32 = (float) L, and the start of Linv32 (the
// diagonal blocks' inverses from Dinv, zeros elsewhere); per element the arithmetic of
// k_zero_upper_blocks, k_cast and k_linv_init.
__global__ void b_prep_inverse(const BProb *P, double *L, float *L32, const double *Dinv, float *Linv)
{
    const BProb &p = P[blockIdx.y];
    const int n_pad = p.n_pad;
    const int64_t sq = (int64_t)n_pad * n_pad;
    double *Lp = L + p.off_sq;
    float *L32p = L32 + p.off_sq, *Lip = Linv + p.off_sq;
    const double *Dp = Dinv + p.off_dinv;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < sq; t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / n_pad), j = (int)(t % n_pad), bi = i / NB, bj = j / NB;
        double v = Lp[t];
        if (bj > bi) {
            v = 0.0;
            Lp[t] = 0.0;
        }
        L32p[t] = (float)v;
        Lip[t] = bi == bj ? (float)Dp[(int64_t)bi * NB * NB + (i % NB) * NB + (j % NB)] : 0.0f;
    }
}

// vec arena per problem: [alpha64 | ypad | work (2 n_pad) | r | dlt]
__global__ void b_pad_copy(const BProb *P, const double *ys, double *vec)
{
    const BProb &p = P[blockIdx.y];
    if ((int)(blockIdx.x * blockDim.x) >= p.n_pad) return;
    k_pad_copy_body(ys + p.off_y, p.n, p.n_pad, vec + p.off_vec + p.n_pad, blockIdx.x, 0);
}

__global__ void b_copy_vec(const BProb *P, double *vec, int src_slot, int dst_slot)
{
    const BProb &p = P[blockIdx.y];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < p.n_pad) vec[p.off_vec + (int64_t)dst_slot * p.n_pad + i] = vec[p.off_vec + (int64_t)src_slot * p.n_pad + i];
}

__global__ void __launch_bounds__(256) b_fwd_step(const BProb *P, const double *L, const double *Dinv, double *vec,
                                                  int b)
{
    const BProb &p = P[blockIdx.y];
    if (b >= p.nblk || (int)blockIdx.x >= max(1, p.nblk - b - 1)) return;
    double *work = vec + p.off_vec + 2 * (int64_t)p.n_pad;
    k_fwd_step_body(L + p.off_sq, Dinv + p.off_dinv, p.n_pad, b, work, work + p.n_pad, blockIdx.x, 0);
}

__global__ void __launch_bounds__(256) b_bwd_step(const BProb *P, const double *L, const double *Dinv, double *vec,
                                                  int s, int out_slot)
{
    const BProb &p = P[blockIdx.y];
    const int b = p.nblk - 1 - s;
    if (b < 0 || (int)blockIdx.x >= max(1, b)) return;
    double *work = vec + p.off_vec + 2 * (int64_t)p.n_pad;
    k_bwd_step_body(L + p.off_sq, Dinv + p.off_dinv, p.n_pad, b, work + p.n_pad,
                    vec + p.off_vec + (int64_t)out_slot * p.n_pad, blockIdx.x, 0);
}

__global__ void b_residual(const BProb *P, const double *K, double *vec)
{
    const BProb &p = P[blockIdx.y];
    if ((int)(blockIdx.x * (blockDim.x / 32)) >= p.n_pad) return;
    double *v = vec + p.off_vec;
    k_residual_body(K + p.off_sq, v, v + p.n_pad, p.n_pad, v + 4 * (int64_t)p.n_pad, blockIdx.x, 0);
}

// Refinement correction through the FP32 L^-1 (the single-problem path's arithmetic):
// u = X r (slot 5 from slot 4), part = chunks of X^T u, alpha (slot 0) += their sum.
__global__ void __launch_bounds__(256) b_trmv(const BProb *P, const float *Linv, double *vec)
{
    const BProb &p = P[blockIdx.y];
    if ((int)(blockIdx.x * 8) >= p.n_pad) return;
    double *v = vec + p.off_vec;
    k_trmv_body(Linv + p.off_sq, p.n_pad, v + 4 * (int64_t)p.n_pad, v + 5 * (int64_t)p.n_pad, blockIdx.x);
}

__global__ void __launch_bounds__(256) b_trmv_t_part(const BProb *P, const float *Linv, const double *vec,
                                                     double *rpart)
{
    const BProb &p = P[blockIdx.z];
    if ((int)(blockIdx.x * 32) >= p.n_pad || (int)blockIdx.y >= p.chunks) return;  // whole CTA
    k_trmv_t_part_body(Linv + p.off_sq, p.n_pad, vec + p.off_vec + 5 * (int64_t)p.n_pad, rpart + p.off_rpart,
                       blockIdx.x, blockIdx.y);
}

__global__ void b_trmv_t_sum(const BProb *P, const double *rpart, double *vec, float *alpha32)
{
    const BProb &p = P[blockIdx.y];
    if ((int)(blockIdx.x * blockDim.x) >= p.n_pad) return;
    k_trmv_t_sum_body(rpart + p.off_rpart, p.n_pad, p.chunks, vec + p.off_vec, alpha32 + p.off_vec / 6, blockIdx.x);
}

// The recursion's GEMMs: problems in blockIdx.z, shared body with the single-problem path.
__global__ void __launch_bounds__(256) b_gemm(const float *A, const float *B, float *Cc, const GemmProb *probs, float alpha,
                                              int tri_a, int tri_b)
{
    k_gemm_batched_body<float>(A, B, Cc, 0, 0, 0, probs, alpha, tri_a, tri_b, blockIdx.x, blockIdx.y);
}

__global__ void __launch_bounds__(256) b_gemm128(const float *A, const float *B, float *Cc, const GemmProb *probs,
                                                 float alpha, int tri_a, int tri_b)
{
    k_gemm128_body(A, B, Cc, probs, alpha, tri_a, tri_b, blockIdx.x, blockIdx.y, blockIdx.z);
}

__global__ void __launch_bounds__(256, 4) b_xkern(const BProb *P, const float *Xs32, const float *alpha32, const double *lsinv,
                                               float *Kst, float *mu)
{
    const BProb &p = P[blockIdx.y];
    if ((int64_t)blockIdx.x * 64 >= p.M) return;
    k_xkern32_body<float>(nullptr, p.seed, 0, p.M, p.d, Xs32 + p.off_xs, alpha32 + p.off_vec / 6, p.n, p.n_pad,
                          (float)p.s2, ls_of(lsinv, blockIdx.y, p.d), Kst + p.off_kst, mu + p.off_mu, blockIdx.x, 0, 0);
}

template <int BM>
__global__ void __launch_bounds__(256, BM == 256 ? 1 : 2) b_var(const BProb *P, const float *Kst, const float *Linv, const float *mu,
                                             const double *tau, float xi, float *pei, int64_t *pidx)
{
    const BProb &p = P[blockIdx.y];
    if ((int64_t)blockIdx.x * BM >= p.M) return;
    k_var_f32_body<BM, true>(Kst + p.off_kst, p.M, 0, p.n_pad, Linv + p.off_sq, mu + p.off_mu, (float)p.s2, 0.0,
                       tau + blockIdx.y, xi, nullptr, nullptr, pei + p.off_part, pidx + p.off_part, 0, blockIdx.x);
}

__global__ void __launch_bounds__(1024) b_argmax(const BProb *P, const float *pei, const int64_t *pidx, double *best_ei,
                                                 int64_t *best_idx)
{
    const BProb &p = P[blockIdx.x];
    k_argmax_final_body<float>(pei + p.off_part, pidx + p.off_part, p.part_count, best_ei + blockIdx.x,
                               best_idx + blockIdx.x, 0, 0, 0);
}

// x_next of problem g: its argmax candidate, redrawn from the counter stream.
__global__ void b_gather(const BProb *P, const int64_t *best_idx, float *xnext)
{
    const BProb &p = P[blockIdx.x];
    const int k = threadIdx.x;
    if (k < p.d) xnext[blockIdx.x * GPBO_MAX_D + k] = uniform24f(p.seed, 2, (uint64_t)(best_idx[blockIdx.x] * p.d + k));
}

// ------------------------------------------------------------------ plan
static void free_plan(BatchPlan *pl)
{
    if (!pl) return;
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    if (pl->cap) cudaStreamDestroy(pl->cap);
    if (pl->cap2) cudaStreamDestroy(pl->cap2);
    if (pl->cap3) cudaStreamDestroy(pl->cap3);
    for (cudaEvent_t e : pl->ev)
        if (e) cudaEventDestroy(e);
    for (void *p : pl->allocs) cudaFree(p);
    delete pl;
}

template <typename T>
static int arena(BatchPlan *pl, T **out, int64_t count)
{
    void *p = nullptr;
    GPBO_CUDA_TRY(cudaMalloc(&p, sizeof(T) * std::max<int64_t>(count, 1)));
    pl->allocs.push_back(p);
    *out = (T *)p;
    return GPBO_OK;
}

static int build_plan(gpbo_ctx *ctx, BatchPlan *pl, const gp_hyper *hyp)
{
    const int G = pl->G;
    pl->probs.resize(G);
    int64_t sX = 0, sy = 0, sxs = 0, ssq = 0, sdinv = 0, svec = 0, skst = 0, smu = 0, spart = 0, srpart = 0;
    std::vector<double> lsinv((size_t)G * GPBO_MAX_D, 0.0);
    for (int g = 0; g < G; ++g) {
        BProb &p = pl->probs[g];
        p.n = pl->n[g];
        p.d = pl->d[g];
        p.n_pad = round_up(p.n, NB);
        p.nblk = p.n_pad / NB;
        p.M = pl->M[g];
        p.seed = 0;
        p.s2 = hyp[g].signal_var;
        p.sn2 = hyp[g].noise_var;
        for (int k = 0; k < p.d; ++k) lsinv[(size_t)g * GPBO_MAX_D + k] = 1.0 / hyp[g].lengthscale[k];
        p.off_X = sX;     sX += (int64_t)p.n * p.d;
        p.off_y = sy;     sy += p.n;
        p.off_xs = sxs;   sxs += (int64_t)p.d * p.n_pad;
        p.off_sq = ssq;   ssq += (int64_t)p.n_pad * p.n_pad;
        p.off_dinv = sdinv; sdinv += (int64_t)p.n_pad * NB;
        p.off_vec = svec; svec += 6 * (int64_t)p.n_pad;
        p.off_kst = skst; skst += p.M * p.n_pad;
        p.off_mu = smu;   smu += p.M;
        p.part_count = (int)cdiv64(p.M, 64);
        p.off_part = spart; spart += cdiv64(p.M, 64);  // room for the smallest variance tile
        p.chunks = (p.n_pad + TRMV_ROWS - 1) / TRMV_ROWS;
        p.off_rpart = srpart; srpart += (int64_t)p.chunks * p.n_pad;
        pl->max_chunks = std::max(pl->max_chunks, p.chunks);
        pl->max_npad = std::max(pl->max_npad, p.n_pad);
        pl->max_nblk = std::max(pl->max_nblk, p.nblk);
        pl->max_tiles64 = std::max<int>(pl->max_tiles64, (int)cdiv64(p.M, 64));
        pl->max_M = std::max<int64_t>(pl->max_M, p.M);
        pl->max_sq = std::max<int64_t>(pl->max_sq, (int64_t)p.n_pad * p.n_pad);
        pl->max_dn = std::max<int64_t>(pl->max_dn, (int64_t)p.d * p.n_pad);
        pl->max_d = std::max(pl->max_d, p.d);
    }
    // alpha32 shares the vec offsets divided by 6 (one float per padded row)
    GPBO_TRY(arena(pl, &pl->probs_dev, G));
    GPBO_TRY(arena(pl, &pl->dX, sX));
    GPBO_TRY(arena(pl, &pl->dy, sy));
    GPBO_TRY(arena(pl, &pl->dys, sy));
    GPBO_TRY(arena(pl, &pl->tau, G));
    GPBO_TRY(arena(pl, &pl->Xs64, sxs));
    GPBO_TRY(arena(pl, &pl->Xs32, sxs));
    GPBO_TRY(arena(pl, &pl->K, ssq));
    GPBO_TRY(arena(pl, &pl->L, ssq));
    GPBO_TRY(arena(pl, &pl->Dinv, sdinv));
    GPBO_TRY(arena(pl, &pl->vec, svec));
    GPBO_TRY(arena(pl, &pl->alpha32, svec / 6));
    GPBO_TRY(arena(pl, &pl->rpart, srpart));
    GPBO_TRY(arena(pl, &pl->lsinv, (int64_t)G * GPBO_MAX_D));
    GPBO_TRY(arena(pl, &pl->L32, ssq));
    GPBO_TRY(arena(pl, &pl->Linv32, ssq));
    GPBO_TRY(arena(pl, &pl->tmp, ssq));
    GPBO_TRY(arena(pl, &pl->Kst, skst));
    GPBO_TRY(arena(pl, &pl->mu, smu));
    GPBO_TRY(arena(pl, &pl->pei, spart));
    GPBO_TRY(arena(pl, &pl->pidx, spart));
    GPBO_TRY(arena(pl, &pl->best_ei, G));
    GPBO_TRY(arena(pl, &pl->best_idx, G));
    GPBO_TRY(arena(pl, &pl->xnext, (int64_t)G * GPBO_MAX_D));
    GPBO_CUDA_TRY(cudaMemcpy(pl->lsinv, lsinv.data(), sizeof(double) * lsinv.size(), cudaMemcpyHostToDevice));
    // the tensor-core updates' slice arena (the single-problem path's rule, per problem)
    {
        int64_t rows = 0, nexp = 0;
        pl->tc_host.assign(G, CholTcProb{});
        for (int g = 0; g < G; ++g) {
            const BProb &p = pl->probs[g];
            CholTcProb &t = pl->tc_host[g];
            t.n_pad = p.n_pad;
            t.nblk = p.nblk;
            if (p.n_pad < CHOL_TC_UPDATE_MIN_NPAD) continue;
            t.row_off = rows;
            rows += (int64_t)chol_tc_slice_bytes(p.n_pad) / (2 * NB);
            t.exps = (int *)(intptr_t)nexp;  // offset for now
            nexp += p.n_pad;
        }
        if (rows > 0) {
            GPBO_TRY(arena(pl, (__nv_bfloat16 **)&pl->tc_slices, rows * NB));
            GPBO_TRY(arena(pl, &pl->tc_exps, nexp));
            GPBO_TRY(arena(pl, &pl->tc_probs, G));
            for (int g = 0; g < G; ++g) {
                CholTcProb &t = pl->tc_host[g];
                t.A = pl->L + pl->probs[g].off_sq;
                t.exps = t.n_pad >= CHOL_TC_UPDATE_MIN_NPAD ? pl->tc_exps + (intptr_t)t.exps : nullptr;
            }
            GPBO_CUDA_TRY(cudaMemcpy(pl->tc_probs, pl->tc_host.data(), sizeof(CholTcProb) * G, cudaMemcpyHostToDevice));
            GPBO_TRY(chol_tc_arena_maps(pl->tc_slices, rows, pl->tc_maps[0], pl->tc_maps[1]));
        }
    }
    // merged triangular-inverse plan: level l gathers every problem's runs of 2^l blocks
    std::vector<GemmProb> all;
    for (int run = 1; run < pl->max_nblk; run *= 2) {
        std::vector<GemmProb> first, second;
        int maxm = 0, maxn = 0;
        for (int g = 0; g < G; ++g) {
            const BProb &p = pl->probs[g];
            for (int b0 = 0; b0 + run < p.nblk; b0 += 2 * run) {
                const int r0 = (b0 + run) * NB, sl = run * NB, sr = std::min(run, p.nblk - b0 - run) * NB;
                GemmProb q;
                q.a_off = p.off_sq + (int64_t)r0 * p.n_pad + (int64_t)b0 * NB;
                q.b_off = p.off_sq + (int64_t)b0 * NB * p.n_pad + (int64_t)b0 * NB;
                q.c_off = q.a_off;
                q.m = sr;
                q.n = sl;
                q.k = sl;
                q.ld = p.n_pad;
                first.push_back(q);
                GemmProb q2 = q;
                q2.b_off = q.c_off;
                q2.a_off = p.off_sq + (int64_t)r0 * p.n_pad + r0;
                q2.k = sr;
                second.push_back(q2);
                maxm = std::max(maxm, sr);
                maxn = std::max(maxn, sl);
            }
        }
        if (first.empty()) continue;
        pl->lvl_first.push_back((int)all.size());
        pl->lvl_count.push_back((int)first.size());
        pl->lvl_mm.push_back(make_int2(maxm, maxn));
        all.insert(all.end(), first.begin(), first.end());
        all.insert(all.end(), second.begin(), second.end());
    }
    GPBO_TRY(arena(pl, &pl->gemm_dev, (int64_t)all.size()));
    if (!all.empty())
        GPBO_CUDA_TRY(cudaMemcpy(pl->gemm_dev, all.data(), sizeof(GemmProb) * all.size(), cudaMemcpyHostToDevice));
    GPBO_CUDA_TRY(cudaStreamCreateWithFlags(&pl->cap, cudaStreamNonBlocking));
    GPBO_CUDA_TRY(cudaStreamCreateWithFlags(&pl->cap2, cudaStreamNonBlocking));
    GPBO_CUDA_TRY(cudaStreamCreateWithFlags(&pl->cap3, cudaStreamNonBlocking));
    for (cudaEvent_t &e : pl->ev) GPBO_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return GPBO_OK;
}

static unsigned gb(int64_t count, int threads = 256) { return (unsigned)std::max<int64_t>(1, cdiv64(count, threads)); }

static int launch_var_bm(BatchPlan *pl, cudaStream_t st, float xi, int bm)
{
    const dim3 grid((unsigned)cdiv64(pl->max_M, bm), pl->G);
    const BProb *P = pl->probs_dev;
    if (bm == 64) b_var<64><<<grid, 256, 0, st>>>(P, pl->Kst, pl->Linv32, pl->mu, pl->tau, xi, pl->pei, pl->pidx);
    else if (bm == 256) b_var<256><<<grid, 256, 0, st>>>(P, pl->Kst, pl->Linv32, pl->mu, pl->tau, xi, pl->pei, pl->pidx);
    else b_var<128><<<grid, 256, 0, st>>>(P, pl->Kst, pl->Linv32, pl->mu, pl->tau, xi, pl->pei, pl->pidx);
    GPBO_CUDA_TRY(cudaGetLastError());
    return GPBO_OK;
}

static int launch_var(BatchPlan *pl, cudaStream_t st, float xi) { return launch_var_bm(pl, st, xi, pl->var_bm); }

// Set the variance tile (candidates per CTA) and the per-problem partial-argmax counts.
static void set_tile(BatchPlan *pl, int bm)
{
    pl->var_bm = bm;
    for (BProb &p : pl->probs) p.part_count = (int)cdiv64(p.M, bm);
}

// Autotuner: time each variance tile on the plan's own (zeroed) buffers, three launches
// after one warm-up, and keep the fastest.  The kernel's work and memory traffic do not
// depend on the values, only on the shapes, which are the plan's.
static int autotune(BatchPlan *pl)
{
    static const int tiles[3] = {64, 128, 256};
    GPBO_CUDA_TRY(cudaMemsetAsync(pl->Kst, 0, sizeof(float) * (size_t)(pl->probs.back().off_kst +
                                  pl->probs.back().M * (int64_t)pl->probs.back().n_pad), pl->cap));
    GPBO_CUDA_TRY(cudaMemsetAsync(pl->Linv32, 0, sizeof(float) * (size_t)(pl->probs.back().off_sq +
                                  (int64_t)pl->probs.back().n_pad * pl->probs.back().n_pad), pl->cap));
    GPBO_CUDA_TRY(cudaMemsetAsync(pl->mu, 0, sizeof(float) * (size_t)(pl->probs.back().off_mu + pl->probs.back().M),
                                  pl->cap));
    GPBO_CUDA_TRY(cudaMemsetAsync(pl->tau, 0, sizeof(double) * pl->G, pl->cap));
    cudaEvent_t a = nullptr, b = nullptr;
    GPBO_CUDA_TRY(cudaEventCreate(&a));
    GPBO_CUDA_TRY(cudaEventCreate(&b));
    int best = 128;
    float best_ms = 1e30f;
    int rc = GPBO_OK;
    for (int i = 0; i < 3 && rc == GPBO_OK; ++i) {
        set_tile(pl, tiles[i]);
        if (cudaMemcpyAsync(pl->probs_dev, pl->probs.data(), sizeof(BProb) * pl->G, cudaMemcpyHostToDevice, pl->cap) !=
            cudaSuccess) { rc = GPBO_ECUDA; break; }
        if ((rc = launch_var_bm(pl, pl->cap, 0.f, tiles[i])) != GPBO_OK) break;
        cudaEventRecord(a, pl->cap);
        for (int r = 0; r < 3 && rc == GPBO_OK; ++r) rc = launch_var_bm(pl, pl->cap, 0.f, tiles[i]);
        cudaEventRecord(b, pl->cap);
        if (cudaEventSynchronize(b) != cudaSuccess) { rc = GPBO_ECUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        pl->tune_ms[i] = ms / 3;
        if (ms / 3 < best_ms) { best_ms = ms / 3; best = tiles[i]; }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    set_tile(pl, best);
    return rc;
}

// The batched step's kernels, in order, on stream st (captured into the plan's graph).
static int enqueue_step(gpbo_ctx *ctx, BatchPlan *pl, cudaStream_t st, float xi)
{
    const int G = pl->G;
    const BProb *P = pl->probs_dev;
    const size_t smem1 = sizeof(double) * NB * (NB + 1);
    b_load_inputs<<<dim3(std::max(1u, gb(pl->max_dn + pl->max_npad) / 4), G), 256, 0, st>>>(P, pl->dX, pl->dy);
    b_standardize<<<G, 1024, 0, st>>>(P, pl->dy, pl->dys, pl->tau);
    b_scale_x<<<dim3(gb(pl->max_dn), G), 256, 0, st>>>(P, pl->dX, pl->lsinv, pl->Xs64, pl->Xs32);
    b_kmat<<<dim3(pl->max_npad / 32, pl->max_npad / 32, G), dim3(32, 8), 0, st>>>(P, pl->Xs64, pl->K);
    GPBO_CUDA_TRY(cudaMemcpyAsync(pl->L, pl->K, sizeof(double) * (size_t)(pl->probs.back().off_sq + pl->probs.back().n_pad *
                                  (int64_t)pl->probs.back().n_pad), cudaMemcpyDeviceToDevice, st));
    // Cholesky with a lookahead of one block column (as the single-problem path): the next
    // column's update, its diagonal factor and its panel on the second capture stream, the
    // rest of each trailing update on the main one.
    cudaStream_t s2 = pl->cap2;
    cudaEvent_t ev_fork = pl->ev[0], ev_panel = pl->ev[1], ev_rest = pl->ev[2], ev_join = pl->ev[3];
    const int NBL = pl->max_nblk;
    GPBO_CUDA_TRY(cudaEventRecord(ev_fork, st));
    GPBO_CUDA_TRY(cudaStreamWaitEvent(s2, ev_fork, 0));
    b_chol_diag<<<dim3(1, G), 256, smem1, s2>>>(P, pl->L, pl->Dinv, 0, ctx->dev_status);
    b_chol_inv<<<dim3(NB / 4, G), 128, 0, s2>>>(P, pl->L, pl->Dinv, 0);
    if (NBL > 1) b_chol_panel<<<dim3((NBL - 1) * (NB / 4), G), 128, 0, s2>>>(P, pl->L, pl->Dinv, 0);
    GPBO_CUDA_TRY(cudaEventRecord(ev_panel, s2));
    for (int kb = 0; kb + 1 < NBL; ++kb) {
        const int T = NBL - kb - 1;
        GPBO_CUDA_TRY(cudaStreamWaitEvent(st, ev_panel, 0));
        if (kb > 0) GPBO_CUDA_TRY(cudaStreamWaitEvent(s2, ev_rest, 0));
        b_chol_update_slab<<<dim3((unsigned)T * (NB / B_SLAB_ROWS), G), 256, 0, s2>>>(P, pl->L, kb, 1);
        b_chol_diag<<<dim3(1, G), 256, smem1, s2>>>(P, pl->L, pl->Dinv, kb + 1, ctx->dev_status);
        b_chol_inv<<<dim3(NB / 4, G), 128, 0, s2>>>(P, pl->L, pl->Dinv, kb + 1);
        if (T > 1) b_chol_panel<<<dim3((T - 1) * (NB / 4), G), 128, 0, s2>>>(P, pl->L, pl->Dinv, kb + 1);
        GPBO_CUDA_TRY(cudaEventRecord(ev_panel, s2));
        if (T > 1) {
            // problems with a tensor-core update at this step (the single-problem rule), and
            // beside it, on the third capture stream, the FP64 update of the others (disjoint
            // problems, so the two branches of the graph run concurrently)
            int max_rows = 0;
            int64_t max_tiles = 0;
            if (pl->tc_probs)
                for (int g = 0; g < G; ++g) {
                    const CholTcProb &t = pl->tc_host[g];
                    if (!chol_tc_step(t.n_pad, t.nblk, kb)) continue;
                    max_rows = std::max(max_rows, t.n_pad - (kb + 2) * NB);
                    max_tiles = std::max(max_tiles, chol_tc_tiles(t.nblk, kb));
                }
            // the FP64 update's grid covers the largest problem it updates (the kernel skips the
            // tensor-core ones by the same rule)
            int64_t slab_tiles = 0;
            for (int g = 0; g < G; ++g) {
                const BProb &q = pl->probs[g];
                const int64_t Tg = q.nblk - kb - 1;
                if (Tg > 1 && !chol_tc_step(q.n_pad, q.nblk, kb)) slab_tiles = std::max(slab_tiles, Tg * (Tg - 1) / 2);
            }
            GPBO_CUDA_TRY(cudaEventRecord(pl->ev[5], st));
            GPBO_CUDA_TRY(cudaStreamWaitEvent(pl->cap3, pl->ev[5], 0));
            if (slab_tiles > 0)
                b_chol_update_slab<<<dim3((unsigned)(slab_tiles * (NB / B_SLAB_ROWS)), G), 256, 0, pl->cap3>>>(
                    P, pl->L, kb, 2);
            GPBO_CUDA_TRY(cudaEventRecord(pl->ev[6], pl->cap3));
            GPBO_TRY(chol_tc_update_batched(ctx, st, pl->tc_probs, G, kb, max_rows, max_tiles, pl->tc_slices,
                                            pl->tc_maps[0], pl->tc_maps[1]));
            GPBO_CUDA_TRY(cudaStreamWaitEvent(st, pl->ev[6], 0));
            GPBO_CUDA_TRY(cudaEventRecord(ev_rest, st));
        }
    }
    GPBO_CUDA_TRY(cudaEventRecord(ev_join, s2));
    GPBO_CUDA_TRY(cudaStreamWaitEvent(st, ev_join, 0));
    b_prep_inverse<<<dim3(std::max(1u, gb(pl->max_sq) / 8), G), 256, 0, st>>>(P, pl->L, pl->L32, pl->Dinv, pl->Linv32);
    // alpha = K^-1 y' with one step of iterative refinement (as the single-problem path): the
    // FP64 solve and residual on the second stream, under the L^-1 products, then the
    // correction through L^-1; vec slots: 0 alpha, 1 ypad, 2-3 work, 4 r, 5 u
    GPBO_CUDA_TRY(cudaEventRecord(ev_fork, st));
    GPBO_CUDA_TRY(cudaStreamWaitEvent(s2, ev_fork, 0));
    b_pad_copy<<<dim3(gb(pl->max_npad), G), 256, 0, s2>>>(P, pl->dys, pl->vec);
    b_copy_vec<<<dim3(gb(pl->max_npad), G), 256, 0, s2>>>(P, pl->vec, 1, 2);
    for (int b = 0; b < NBL; ++b)
        b_fwd_step<<<dim3(std::max(1, NBL - b - 1), G), 256, 0, s2>>>(P, pl->L, pl->Dinv, pl->vec, b);
    for (int s = 0; s < NBL; ++s)
        b_bwd_step<<<dim3(std::max(1, NBL - 1 - s), G), 256, 0, s2>>>(P, pl->L, pl->Dinv, pl->vec, s, 0);
    b_residual<<<dim3((pl->max_npad + 7) / 8, G), 256, 0, s2>>>(P, pl->K, pl->vec);
    // FP32 L^-1 (L32 and the start of Linv32 from b_prep_inverse)
    for (size_t l = 0; l < pl->lvl_first.size(); ++l) {
        if (pl->lvl_mm[l].y >= 128) {  // the single-problem path's rule: 128 x 128 tiles on large levels
            dim3 g((pl->lvl_mm[l].y + 127) / 128, (pl->lvl_mm[l].x + 127) / 128, pl->lvl_count[l]);
            b_gemm128<<<g, 256, 0, st>>>(pl->L32, pl->Linv32, pl->tmp, pl->gemm_dev + pl->lvl_first[l], 1.0f, 0, 1);
            b_gemm128<<<g, 256, 0, st>>>(pl->Linv32, pl->tmp, pl->Linv32,
                                         pl->gemm_dev + pl->lvl_first[l] + pl->lvl_count[l], -1.0f, 1, 0);
            continue;
        }
        dim3 grid((pl->lvl_mm[l].y + 63) / 64, (pl->lvl_mm[l].x + 63) / 64, pl->lvl_count[l]);
        b_gemm<<<grid, 256, 0, st>>>(pl->L32, pl->Linv32, pl->tmp, pl->gemm_dev + pl->lvl_first[l], 1.0f, 0, 1);
        b_gemm<<<grid, 256, 0, st>>>(pl->Linv32, pl->tmp, pl->Linv32, pl->gemm_dev + pl->lvl_first[l] + pl->lvl_count[l],
                                     -1.0f, 1, 0);
    }
    GPBO_CUDA_TRY(cudaEventRecord(pl->ev[4], st));
    GPBO_CUDA_TRY(cudaStreamWaitEvent(s2, pl->ev[4], 0));
    b_trmv<<<dim3((pl->max_npad + 7) / 8, G), 256, 0, s2>>>(P, pl->Linv32, pl->vec);
    b_trmv_t_part<<<dim3(pl->max_npad / 32, pl->max_chunks, G), 256, 0, s2>>>(P, pl->Linv32, pl->vec, pl->rpart);
    b_trmv_t_sum<<<dim3(gb(pl->max_npad), G), 256, 0, s2>>>(P, pl->rpart, pl->vec, pl->alpha32);
    GPBO_CUDA_TRY(cudaEventRecord(ev_join, s2));
    GPBO_CUDA_TRY(cudaStreamWaitEvent(st, ev_join, 0));
    // scoring
    const size_t xkern_smem = sizeof(float) * (192 * (size_t)pl->max_d + 128);
    GPBO_TRY(ensure_smem((const void *)b_xkern, ctx->device, (int)xkern_smem));
    b_xkern<<<dim3(pl->max_tiles64, G), 256, xkern_smem, st>>>(P, pl->Xs32, pl->alpha32, pl->lsinv,
                                                                                    pl->Kst, pl->mu);
    GPBO_TRY(launch_var(pl, st, xi));
    b_argmax<<<G, 1024, 0, st>>>(P, pl->pei, pl->pidx, pl->best_ei, pl->best_idx);
    b_gather<<<G, GPBO_MAX_D, 0, st>>>(P, pl->best_idx, pl->xnext);
    GPBO_CUDA_TRY(cudaGetLastError());
    return GPBO_OK;
}

// Kernel nodes of a captured graph (one graph replay launches that many kernels).
static int64_t count_kernel_nodes(cudaGraph_t g)
{
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) return 0;
    std::vector<cudaGraphNode_t> nodes(n);
    if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return 0;
    int64_t k = 0;
    for (cudaGraphNode_t node : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(node, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

// The call's problems split by size into at most two plans whose graphs run concurrently, on
// streams of low and high priority: the small problems' whole step (factorisation, inverse,
// scoring) runs beside the large ones' factorisation, whose chain of latency-bound launches
// leaves most SMs idle.  Each problem's kernels and arithmetic are those of one plan, so every
// result is the same as with one plan.
constexpr int B_SMALL_NPAD = 512;
struct BatchSet {
    // key
    int G = 0;
    double xi = 0.0;
    std::vector<int> n, d;
    std::vector<int64_t> M;
    std::vector<double> key_hyp;
    int tile_req = 0;
    BatchPlan *pl[2] = {};       // [0]: problems of n_pad <= B_SMALL_NPAD, [1]: the others (either may be null)
    std::vector<int> idx[2];     // each plan's problems' positions in the call
    cudaStream_t st[2] = {};     // [0] lowest priority, [1] highest
    cudaEvent_t ev[3] = {};      // fork, and each plan's end
    void *host = nullptr;        // pinned: per problem its best EI, index and x_next, then the status word
};

static void free_set(BatchSet *bs)
{
    if (!bs) return;
    for (int c = 0; c < 2; ++c) {
        free_plan(bs->pl[c]);
        if (bs->st[c]) cudaStreamDestroy(bs->st[c]);
    }
    for (cudaEvent_t e : bs->ev)
        if (e) cudaEventDestroy(e);
    if (bs->host) cudaFreeHost(bs->host);
    delete bs;
}

static bool same_key(const BatchSet *bs, int G, const int *n, const int *d, const int64_t *M, const gp_hyper *hyp,
                     double xi)
{
    if (!bs || bs->G != G || bs->xi != xi) return false;
    std::vector<double> kh;
    for (int g = 0; g < G; ++g) {
        if (bs->n[g] != n[g] || bs->d[g] != d[g] || bs->M[g] != M[g]) return false;
        kh.push_back(hyp[g].signal_var);
        kh.push_back(hyp[g].noise_var);
        for (int k = 0; k < d[g]; ++k) kh.push_back(hyp[g].lengthscale[k]);
    }
    return kh == bs->key_hyp;
}

// Pinned readback of a set: G best EIs, G indices, G x GPBO_MAX_D floats of x_next, the status.
static size_t set_host_bytes(int G)
{
    return (sizeof(double) + sizeof(int64_t) + sizeof(float) * GPBO_MAX_D) * (size_t)G + 16;
}

// A new set for this call's shapes: the split, each part's plan (arenas, autotuned tile), the
// streams and events.
static int build_set(gpbo_ctx *ctx, BatchSet *bs, const gp_hyper *hyp)
{
    for (int g = 0; g < bs->G; ++g) bs->idx[round_up(bs->n[g], NB) <= B_SMALL_NPAD ? 0 : 1].push_back(g);
    int lo = 0, hi = 0;
    GPBO_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    for (int c = 0; c < 2; ++c) {
        GPBO_CUDA_TRY(cudaStreamCreateWithPriority(&bs->st[c], cudaStreamNonBlocking, c == 0 ? lo : hi));
        if (bs->idx[c].empty()) continue;
        BatchPlan *pl = new BatchPlan();
        bs->pl[c] = pl;
        pl->G = (int)bs->idx[c].size();
        pl->xi = bs->xi;
        std::vector<gp_hyper> h;
        for (int g : bs->idx[c]) {
            pl->n.push_back(bs->n[g]);
            pl->d.push_back(bs->d[g]);
            pl->M.push_back(bs->M[g]);
            h.push_back(hyp[g]);
        }
        pl->tile_req = bs->tile_req;
        GPBO_TRY(build_plan(ctx, pl, h.data()));
        if (pl->tile_req) set_tile(pl, pl->tile_req);
        else GPBO_TRY(autotune(pl));
    }
    for (cudaEvent_t &e : bs->ev) GPBO_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    GPBO_CUDA_TRY(cudaMallocHost(&bs->host, set_host_bytes(bs->G)));
    return GPBO_OK;
}

// Enqueue one plan's step on stream s: its inputs (host: a copy each; device: read by the
// graph's first kernel), its problem table, and its graph (captured on first use).
static int enqueue_plan(gpbo_ctx *ctx, BatchPlan *pl, const std::vector<int> &idx, cudaStream_t s,
                        const double *const *X, const double *const *y, const uint64_t *seed, bool host)
{
    for (int k = 0; k < pl->G; ++k) {
        const int g = idx[k];
        BProb &p = pl->probs[k];
        p.seed = seed[g];
        p.X_src = host ? nullptr : X[g];
        p.y_src = host ? nullptr : y[g];
        if (host) {
            GPBO_CUDA_TRY(cudaMemcpyAsync(pl->dX + p.off_X, X[g], sizeof(double) * p.n * p.d, cudaMemcpyHostToDevice, s));
            GPBO_CUDA_TRY(cudaMemcpyAsync(pl->dy + p.off_y, y[g], sizeof(double) * p.n, cudaMemcpyHostToDevice, s));
        }
    }
    GPBO_CUDA_TRY(cudaMemcpyAsync(pl->probs_dev, pl->probs.data(), sizeof(BProb) * pl->G, cudaMemcpyHostToDevice, s));
    if (!pl->exec) {
        // capture the step once; the probe table and arenas keep their addresses from here on
        GPBO_CUDA_TRY(cudaStreamSynchronize(s));
        GPBO_CUDA_TRY(cudaFuncSetAttribute(b_chol_diag, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(sizeof(double) * 2 * NB * (NB + 1))));
        GPBO_CUDA_TRY(cudaStreamBeginCapture(pl->cap, cudaStreamCaptureModeThreadLocal));
        int st = enqueue_step(ctx, pl, pl->cap, (float)pl->xi);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(pl->cap, &graph);
        if (st != GPBO_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            note_cuda_error(e, "batched capture", __FILE__, __LINE__);
            return st != GPBO_OK ? st : GPBO_ECUDA;
        }
        pl->graph = graph;
        pl->kernels = count_kernel_nodes(graph);
        GPBO_CUDA_TRY(cudaGraphInstantiate(&pl->exec, graph, 0));
    }
    GPBO_CUDA_TRY(cudaGraphLaunch(pl->exec, s));
    ctx->launches += pl->kernels;
    return GPBO_OK;
}

}  // namespace gpbo

using namespace gpbo;

static BatchSet *g_last_set_for_ctx(gpbo_ctx *ctx) { return (BatchSet *)ctx->batch_plan; }

extern "C" int search_step_batched(gpbo_ctx *ctx, int G, const double *const *X, const double *const *y, const int *n,
                                   const int *d, const gp_hyper *hyp, const int64_t *M, const uint64_t *seed, double xi,
                                   gpbo_prec prec, unsigned flags, double *x_next, double *ei_max, int64_t *argmax)
{
    if (!ctx || G < 1 || G > 4096 || !X || !y || !n || !d || !hyp || !M || !seed || !x_next || !ei_max) return GPBO_EINVAL;
    if (prec != GPBO_PREC_F32) return GPBO_ENOTSUP;
    for (int g = 0; g < G; ++g) {
        if (!X[g] || !y[g] || n[g] < 1 || n[g] > GPBO_MAX_N || d[g] < 1 || d[g] > GPBO_MAX_D || M[g] < 1 ||
            M[g] > 0x7fffffffll || hyp[g].d != d[g] || !hyp[g].lengthscale || !(hyp[g].signal_var > 0) ||
            !(hyp[g].noise_var >= 0))
            return GPBO_EINVAL;
        for (int k = 0; k < d[g]; ++k)
            if (!(hyp[g].lengthscale[k] > 0)) return GPBO_EINVAL;
    }
    GPBO_CUDA_TRY(cudaSetDevice(ctx->device));
    BatchSet *bs = g_last_set_for_ctx(ctx);
    if (!same_key(bs, G, n, d, M, hyp, xi) || bs->tile_req != ctx->batch_tile) {
        cudaStreamSynchronize(ctx->stream);
        free_set(bs);
        ctx->batch_plan = nullptr;
        bs = new BatchSet();
        bs->G = G;
        bs->xi = xi;
        bs->n.assign(n, n + G);
        bs->d.assign(d, d + G);
        bs->M.assign(M, M + G);
        for (int g = 0; g < G; ++g) {
            bs->key_hyp.push_back(hyp[g].signal_var);
            bs->key_hyp.push_back(hyp[g].noise_var);
            for (int k = 0; k < d[g]; ++k) bs->key_hyp.push_back(hyp[g].lengthscale[k]);
        }
        bs->tile_req = ctx->batch_tile;
        const int st = build_set(ctx, bs, hyp);
        if (st != GPBO_OK) {
            free_set(bs);
            return st;
        }
        ctx->batch_plan = bs;
    }
    // both plans' steps, forked from and joined back into the context stream
    const bool host = flags & GPBO_HOST_PTRS;
    GPBO_CUDA_TRY(cudaEventRecord(bs->ev[0], ctx->stream));
    for (int c = 1; c >= 0; --c) {  // the large problems' step first, on the high-priority stream
        if (!bs->pl[c]) continue;
        GPBO_CUDA_TRY(cudaStreamWaitEvent(bs->st[c], bs->ev[0], 0));
        GPBO_TRY(enqueue_plan(ctx, bs->pl[c], bs->idx[c], bs->st[c], X, y, seed, host));
        GPBO_CUDA_TRY(cudaEventRecord(bs->ev[1 + c], bs->st[c]));
    }
    for (int c = 0; c < 2; ++c)
        if (bs->pl[c]) GPBO_CUDA_TRY(cudaStreamWaitEvent(ctx->stream, bs->ev[1 + c], 0));
    // every plan's results and the status word into pinned memory, then one synchronisation
    double *be = (double *)bs->host;
    int64_t *bi = (int64_t *)(be + G);
    float *xn = (float *)(bi + G);
    unsigned *bits = (unsigned *)(xn + (size_t)G * GPBO_MAX_D);
    int off = 0;
    for (int c = 0; c < 2; ++c) {
        const BatchPlan *pl = bs->pl[c];
        if (!pl) continue;
        GPBO_CUDA_TRY(cudaMemcpyAsync(be + off, pl->best_ei, sizeof(double) * pl->G, cudaMemcpyDeviceToHost, ctx->stream));
        GPBO_CUDA_TRY(cudaMemcpyAsync(bi + off, pl->best_idx, sizeof(int64_t) * pl->G, cudaMemcpyDeviceToHost, ctx->stream));
        GPBO_CUDA_TRY(cudaMemcpyAsync(xn + (size_t)off * GPBO_MAX_D, pl->xnext, sizeof(float) * GPBO_MAX_D * pl->G,
                                      cudaMemcpyDeviceToHost, ctx->stream));
        off += pl->G;
    }
    GPBO_CUDA_TRY(cudaMemcpyAsync(bits, ctx->dev_status, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
    GPBO_CUDA_TRY(cudaMemsetAsync(ctx->dev_status, 0, sizeof(unsigned), ctx->stream));
    GPBO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (*bits & DEV_NOTSPD) return GPBO_ENOTSPD;
    off = 0;
    for (int c = 0; c < 2; ++c) {
        if (!bs->pl[c]) continue;
        for (size_t k = 0; k < bs->idx[c].size(); ++k, ++off) {
            const int g = bs->idx[c][k];
            ei_max[g] = be[off];
            if (argmax) argmax[g] = bi[off];
            for (int q = 0; q < GPBO_MAX_D; ++q)
                x_next[(size_t)g * GPBO_MAX_D + q] = q < d[g] ? (double)xn[(size_t)off * GPBO_MAX_D + q] : 0.0;
        }
    }
    return GPBO_OK;
}

extern "C" int search_step_batched_tile(gpbo_ctx *ctx, int tile)
{
    if (!ctx || !(tile == 0 || tile == 64 || tile == 128 || tile == 256)) return GPBO_EINVAL;
    ctx->batch_tile = tile;
    return GPBO_OK;
}

// The plan with the larger problems (the one with most of the variance work).
extern "C" int search_step_batched_tuning(const gpbo_ctx *ctx, int *tile, float *ms3, int *members)
{
    if (!ctx || !tile) return GPBO_EINVAL;
    const BatchSet *bs = (const BatchSet *)ctx->batch_plan;
    const int c = bs && bs->pl[1] ? 1 : 0;
    const BatchPlan *pl = bs ? bs->pl[c] : nullptr;
    if (!pl) return GPBO_EINVAL;
    *tile = pl->var_bm;
    if (ms3)
        for (int i = 0; i < 3; ++i) ms3[i] = pl->tune_ms[i];
    if (members) {
        for (int g = 0; g < bs->G; ++g) members[g] = 0;
        for (int g : bs->idx[c]) members[g] = 1;
    }
    return GPBO_OK;
}

namespace gpbo {
void batch_plan_free(void *p) { free_set((BatchSet *)p); }
}  // namespace gpbo
