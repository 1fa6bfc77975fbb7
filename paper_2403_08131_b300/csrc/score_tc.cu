// Posterior variance, EI and argmax on the 5th-generation tensor cores (tcgen05).
//
// For a chunk of C candidates whose cross-kernel rows K* (C x n_pad, BF16 or FP16,
// observation index contiguous) and means are ready, computes
//     V = K* (L^-1)^T             (C x n_pad; only the lower triangle of L^-1 is read)
//     sigma_c^2 = s2 - sum_i V_ci^2,  EI_c, and the chunk's (EI, index) winners.
// This is the triangular solve v = L^-1 k* of the GP posterior variance (Rasmussen &
// Williams 2006, Alg. 2.1) written as a GEMM with many right-hand sides, so that it is a
// dense contraction and belongs on the tensor cores.
//
// Kernel shape: clusters of two CTAs (one per SM), persistent over tiles of 256 candidates, the
// pair running one tensor-core MMA of M = 256 (cta_group::2): each CTA holds its own 128
// candidates (its TMEM lanes) and half of the 256 L^-1 rows of the output chunk, so a CTA stages
// 32 KiB per 64 of K instead of 48 KiB for the same MMA time.
//   warp 0      TMA producer (both CTAs): K* tile (128 x 128) and half the L^-1 tile (128 x 128)
//               per stage as 64-wide sub-tiles, 128-byte swizzle, 3 stages of 64 KiB
//   warp 1      both CTAs allocate 512 TMEM columns together; in the first CTA one lane issues
//               the pair's tcgen05.mma (M=256, N=256, K=16, FP32 accumulate) into one of two
//               256-column accumulators once both CTAs' copies of a stage have landed; in the
//               second CTA one lane forwards each landed stage to the first CTA's barrier
//   warps 2..5  epilogue (both CTAs): tcgen05.ld the accumulator, square and sum into the
//               candidate's running |v|^2 (one TMEM lane = one candidate = one thread), then
//               sigma, EI and the per-CTA argmax
// For output chunk q (L^-1 rows 256q .. 256q+255) only K columns < 256(q+1) are read:
// the triangle's zero blocks are never loaded or multiplied.  Successive passes over K run in
// opposite directions, so a pass starts on the K* columns the previous one read last (in L2).
// BF16 models carry a compensated inverse, hi = bf16(L^-1) and lo = bf16(L^-1 - hi); the
// K loop then runs twice (hi, then lo) into the same accumulator, so only K*'s rounding
// remains (twice the MMA work).  FP16 models run a single pass.
//
// Every mbarrier wait is bounded (the context's wait limit, about 2 s of SM clock by
// default).  On timeout the kernel sets DEV_TIMEOUT in the context's status word, every
// role leaves its loop, the producer waits (bounded by the default limit) for copies it
// issued, the MMA issuer drains its MMAs (and both CTAs wait for that), and the allocating
// warps free TMEM before the CTAs exit.  gpbo_inject_wait_stall makes the epilogue wait on a
// barrier that nothing arrives at, so that tests can run this path without a fault.
#include "tc_common.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>

namespace gpbo {

namespace tc {

constexpr int BM = 128;        // candidates per CTA (TMEM lanes); a pair covers 2 BM
constexpr int BN = TC_NCHUNK;  // L^-1 rows per output chunk (MMA N)
constexpr int BNH = BN / 2;    // rows of the chunk each CTA of the pair stages
constexpr int BK = 128;        // K elements per stage
constexpr int KSUB = BK / 64;  // sub-tiles of 64 (128 bytes of 16-bit values: the swizzle span)
constexpr int STAGES = 3;
constexpr int A_SUB = BM * 64 * 2;
constexpr int B_SUB = BNH * 64 * 2;
constexpr int A_BYTES = KSUB * A_SUB;
constexpr int B_BYTES = KSUB * B_SUB;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int THREADS = 192;
constexpr int TMEM_COLS = 512;
constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES + 1024 /*align*/ + 512 /*barriers*/;

struct Shared {
    uint64_t full[STAGES];   // this CTA's copies of the stage have landed
    uint64_t pfull[STAGES];  // first CTA: the second CTA's copies of the stage have landed
    uint64_t empty[STAGES];  // the pair's MMAs are done with the stage (both CTAs)
    uint64_t acc_full[2];    // accumulator a is complete (both CTAs)
    uint64_t acc_empty[2];   // first CTA: both CTAs' epilogues have read accumulator a
    uint64_t drain;          // every MMA of the pair is complete (both CTAs)
    uint64_t never;          // failure injection: a barrier that nothing arrives at
    uint32_t tmem_base;
    int abort;
    float best_v[4];
    int64_t best_i[4];
};
static_assert(sizeof(Shared) <= 512, "barrier area");

using namespace tcx;

// Instruction descriptor for this kernel's MMA: N = 256, M = 256 (the pair's two halves).
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt) { return idesc_f16(fmt, BN, 2 * BM); }

struct Params {
    int64_t C;        // candidates in this chunk
    int64_t c0;       // pool index of the chunk's first candidate
    int n_pad;
    int num_tiles;    // tiles of 2 BM candidates
    float s2;
    float xi;
    double y_best;
    const double *tau_dev;
    const float *mu;  // pool-indexed
    float *sigma_out; // pool-indexed, may be null
    float *ei_out;    // pool-indexed, may be null
    float *part_ei;   // one per CTA
    int64_t *part_idx;
    unsigned *status;
    uint32_t idesc;
    int split;        // 1: V = K* hi^T + K* lo^T (compensated BF16 inverse), 0: single pass
};

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(THREADS, 1)
    k_var_ei_tc(const __grid_constant__ CUtensorMap map_k, const __grid_constant__ CUtensorMap map_l,
                const __grid_constant__ CUtensorMap map_l2, Params P)
{
    extern __shared__ unsigned char smraw[];
    unsigned char *tiles = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    Shared *sh = (Shared *)(tiles + (size_t)STAGES * STAGE_BYTES);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int nq = P.n_pad / BN;
    const uint32_t rank = cluster_rank();  // 0: issues the pair's MMAs
    const int pair = (int)(blockIdx.x >> 1), npairs = (int)(gridDim.x >> 1);
    const int passes = 1 + P.split;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&sh->full[s], 1);
            mbar_init(&sh->pfull[s], 1);
            mbar_init(&sh->empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&sh->acc_full[a], 1);
            mbar_init(&sh->acc_empty[a], 8);
        }
        mbar_init(&sh->drain, 1);
        mbar_init(&sh->never, 1);
        sh->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        // one warp of each CTA of the pair allocates, together, the same columns in both
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh->tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();  // both CTAs' barriers are initialised before either signals the other
    tc_fence_after();
    const uint32_t tmem = sh->tmem_base;
    volatile int *abort_flag = &sh->abort;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&map_k) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&map_l) : "memory");
            if (P.split) asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&map_l2) : "memory");
            int stage = 0;
            uint32_t phase = 0;
            uint32_t armed = 0, armed_par = 0;  // bit s: stage s has a copy issued, and its phase
            bool ok = true;
            for (int t = pair; ok && t < P.num_tiles; t += npairs) {
                const int arow = t * (2 * BM) + (int)rank * BM;
                for (int q = 0; ok && q < nq; ++q) {
                    const int ksteps = (q + 1) * (BN / BK);
                    const int brow = q * BN + (int)rank * BNH;
                    for (int h = 0; ok && h < passes; ++h) {
                        const bool down = ((q * passes + h) & 1) != 0;
                        const CUtensorMap *mb = h ? &map_l2 : &map_l;
                        for (int i = 0; i < ksteps; ++i) {
                            const int ks = down ? ksteps - 1 - i : i;
                            if (!mbar_wait_fast(&sh->empty[stage], phase ^ 1u, abort_flag, P.status)) { ok = false; break; }
                            unsigned char *a = tiles + (size_t)stage * STAGE_BYTES;
                            unsigned char *b = a + A_BYTES;
                            mbar_arrive_expect_tx(&sh->full[stage], STAGE_BYTES);
                            armed |= 1u << stage;
                            armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
#pragma unroll
                            for (int u = 0; u < KSUB; ++u) {
                                tma_load_2d(a + u * A_SUB, &map_k, ks * BK + 64 * u, arow, &sh->full[stage]);
                                tma_load_2d(b + u * B_SUB, mb, ks * BK + 64 * u, brow, &sh->full[stage]);
                            }
                            if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                        }
                    }
                }
            }
            // leave no copy in flight: wait for the last arming of every stage
            for (int s = 0; s < STAGES; ++s)
                if ((armed >> s) & 1u) mbar_wait(&sh->full[s], (armed_par >> s) & 1u, abort_flag, P.status, false);
        }
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) {
            // ---------------- MMA issuer of the pair
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool ok = true;
            for (int t = pair; ok && t < P.num_tiles; t += npairs) {
                for (int q = 0; ok && q < nq; ++q) {
                    // CTA-scope acquire on the barriers that the second CTA signals: a cluster-scope
                    // poll costs about as much as a K step's MMAs, and each signal covers work that
                    // the signalling CTA completed on its own side (its TMEM reads; its copies, which
                    // its own wait saw land) before signalling
                    if (!mbar_wait_fast(&sh->acc_empty[acc], acc_phase ^ 1u, abort_flag, P.status)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t d_tmem = tmem + (uint32_t)(acc * BN);
                    const int ksteps = (q + 1) * (BN / BK) * passes;
                    for (int ks = 0; ks < ksteps; ++ks) {
                        if (!mbar_wait_fast(&sh->full[stage], phase, abort_flag, P.status)) { ok = false; break; }
                        if (!mbar_wait_fast(&sh->pfull[stage], phase, abort_flag, P.status)) { ok = false; break; }
                        tc_fence_after();
                        const unsigned char *a = tiles + (size_t)stage * STAGE_BYTES;
                        const unsigned char *b = a + A_BYTES;
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk)
                            mma_f16_pair(d_tmem, smem_desc(a + (kk >> 2) * A_SUB + (kk & 3) * 32),
                                         smem_desc(b + (kk >> 2) * B_SUB + (kk & 3) * 32), P.idesc,
                                         (ks > 0 || kk > 0) ? 1u : 0u);
                        mma_commit_pair(&sh->empty[stage], 3);
                        if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                    }
                    if (!ok) break;
                    mma_commit_pair(&sh->acc_full[acc], 3);
                    if (++acc == 2) { acc = 0; acc_phase ^= 1u; }
                }
            }
            // every MMA this thread issued completes before either CTA releases TMEM or exits
            mma_commit_pair(&sh->drain, 3);
            mbar_wait(&sh->drain, 0, abort_flag, P.status, false);
        } else if (lane == 0) {
            // ---------------- the second CTA: forward each landed stage to the first CTA
            const uint32_t pfull0 = cluster_addr(&sh->pfull[0], 0);
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int t = pair; ok && t < P.num_tiles; t += npairs) {
                for (int q = 0; ok && q < nq; ++q) {
                    const int ksteps = (q + 1) * (BN / BK) * passes;
                    for (int ks = 0; ks < ksteps; ++ks) {
                        if (!mbar_wait_fast(&sh->full[stage], phase, abort_flag, P.status)) { ok = false; break; }
                        // the copies have landed in this CTA's shared memory (this wait saw them);
                        // the signal itself publishes nothing, so it needs no release fence
                        mbar_arrive_cluster_relaxed(pfull0 + (uint32_t)(stage * sizeof(uint64_t)));
                        if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                    }
                }
            }
            mbar_wait(&sh->drain, 0, abort_flag, P.status, false);
        }
    } else {
        // ---------------- epilogue: warps 2..5, TMEM lane quadrant = warp % 4
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(quad * 32) << 16;
        const uint32_t acc_empty0 = cluster_addr(&sh->acc_empty[0], 0);
        const float tau = P.tau_dev ? (float)*P.tau_dev : (float)P.y_best;
        float best_v = -1.0f;
        int64_t best_i = INT64_MAX;
        int acc = 0;
        uint32_t acc_phase = 0;
        bool ok = true;
        if (injected_faults(P.status) & 1u) {
            // failure injection for tests of this error path: the wait runs out after the
            // context's wait limit, and every role leaves as on a real timeout
            const bool got = mbar_wait_inl(&sh->never, 0, abort_flag, P.status);
            ok = __all_sync(0xffffffffu, got);
        }
        for (int t = pair; ok && t < P.num_tiles; t += npairs) {
            float ss = 0.0f;
            for (int q = 0; q < nq; ++q) {
                // every lane waits; the warp leaves together so tcgen05.ld stays warp-uniform
                const bool got = mbar_wait_inl(&sh->acc_full[acc], acc_phase, abort_flag, P.status);
                if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
                tc_fence_after();
#pragma unroll 1
                for (int cb = 0; cb < BN / 32; ++cb) {
                    float v[32];
                    tmem_ld32(tmem + lane_addr + (uint32_t)(acc * BN + cb * 32), v);
#pragma unroll
                    for (int j = 0; j < 32; ++j) ss = fmaf(v[j], v[j], ss);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(acc_empty0 + (uint32_t)(acc * sizeof(uint64_t)));
                if (++acc == 2) { acc = 0; acc_phase ^= 1u; }
            }
            if (!ok) break;
            const int64_t cl = (int64_t)t * (2 * BM) + (int64_t)rank * BM + row;
            if (cl < P.C) {
                const int64_t c = P.c0 + cl;
                const float var = P.s2 - ss;
                const float sg = var > 0.0f ? sqrtf(var) : 0.0f;
                const float e = ei_minf(P.mu[c], sg, tau, P.xi);
                if (P.sigma_out) P.sigma_out[c] = sg;
                if (P.ei_out) P.ei_out[c] = e;
                if (better(e, c, best_v, best_i)) { best_v = e; best_i = c; }
            }
        }
        for (int o = 16; o; o >>= 1) {
            float ov = __shfl_xor_sync(0xffffffffu, best_v, o);
            int64_t oi = __shfl_xor_sync(0xffffffffu, best_i, o);
            if (better(ov, oi, best_v, best_i)) { best_v = ov; best_i = oi; }
        }
        if (lane == 0) {
            sh->best_v[warp - 2] = best_v;
            sh->best_i[warp - 2] = best_i;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        float bv = sh->best_v[0];
        int64_t bi = sh->best_i[0];
        for (int w = 1; w < 4; ++w)
            if (better(sh->best_v[w], sh->best_i[w], bv, bi)) { bv = sh->best_v[w]; bi = sh->best_i[w]; }
        P.part_ei[blockIdx.x] = bv;
        P.part_idx[blockIdx.x] = bi;
    }
    // neither CTA leaves while the other may still signal its barriers
    cluster_sync();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

}  // namespace tc

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static int get_encoder()
{
    if (g_encode) return GPBO_OK;
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    GPBO_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !fn) return GPBO_ENOTSUP;
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return GPBO_OK;
}

// 2-D row-major 16-bit matrix (rows x cols, cols contiguous), box = box_rows x 64 cols.
int encode_2d(CUtensorMap *map, CUtensorMapDataType dt, const void *base, uint64_t rows, uint64_t cols,
                     uint32_t box_rows)
{
    return encode_2d_box(map, dt, base, rows, cols, box_rows, 64, CU_TENSOR_MAP_SWIZZLE_128B);
}

int encode_2d_box(CUtensorMap *map, CUtensorMapDataType dt, const void *base, uint64_t rows, uint64_t cols,
                  uint32_t box_rows, uint32_t box_cols, CUtensorMapSwizzle swizzle)
{
    GPBO_TRY(get_encoder());
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {cols * 2};
    cuuint32_t box[2] = {box_cols, box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = g_encode(map, dt, 2, const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        fprintf(stderr, "gpbo: cuTensorMapEncodeTiled failed (%d)\n", (int)r);
        return GPBO_ECUDA;
    }
    return GPBO_OK;
}

int tc_variance_ei(gpbo_ctx *ctx, const gp_model *m, const void *Kstar, int64_t C, int64_t c0, const float *mu,
                   double y_best, const double *tau_dev, double xi, float *sigma_out, float *ei_out, float *part_ei,
                   int64_t *part_idx, int *n_parts)
{
    if (m->n_pad % tc::BN != 0 || C <= 0 || C > 0x7fffffffll) return GPBO_EINVAL;
    if (((uintptr_t)Kstar & 15) || ((uintptr_t)m->Linv16 & 15)) return GPBO_EINVAL;
    const CUtensorMapDataType dt =
        m->prec == GPBO_PREC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    CUtensorMap mk, ml, ml2;
    const int split = m->prec == GPBO_PREC_BF16 ? 1 : 0;
    const size_t sq = (size_t)m->n_pad * m->n_pad;
    GPBO_TRY(encode_2d(&mk, dt, Kstar, (uint64_t)C, (uint64_t)m->n_pad, tc::BM));
    GPBO_TRY(encode_2d(&ml, dt, m->Linv16, (uint64_t)m->n_pad, (uint64_t)m->n_pad, tc::BNH));
    GPBO_TRY(encode_2d(&ml2, dt, (const uint16_t *)m->Linv16 + (split ? sq : 0), (uint64_t)m->n_pad,
                       (uint64_t)m->n_pad, tc::BNH));
    GPBO_TRY(ensure_smem((const void *)tc::k_var_ei_tc, ctx->device, (int)tc::SMEM_BYTES));
    tc::Params P;
    P.C = C;
    P.c0 = c0;
    P.n_pad = m->n_pad;
    P.num_tiles = (int)cdiv64(C, 2 * tc::BM);
    P.s2 = (float)m->s2;
    P.xi = (float)xi;
    P.y_best = y_best;
    P.tau_dev = tau_dev;
    P.mu = mu;
    P.sigma_out = sigma_out;
    P.ei_out = ei_out;
    P.part_ei = part_ei;
    P.part_idx = part_idx;
    P.status = ctx->dev_status;
    P.idesc = tc::instr_desc(m->prec == GPBO_PREC_BF16 ? 1u : 0u);
    P.split = split;
    // clusters of two CTAs, one per SM: as many pairs as can be resident at once (a pair must
    // sit in one GPC, so this can be below half the SMs)
    int pairs = 0;
    {
        static std::mutex mu;
        static int cached[64] = {};
        std::lock_guard<std::mutex> lk(mu);
        if (ctx->device >= 0 && ctx->device < 64 && cached[ctx->device] > 0) {
            pairs = cached[ctx->device];
        } else {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(2 * (ctx->sm_count / 2));
            cfg.blockDim = dim3(tc::THREADS);
            cfg.dynamicSmemBytes = tc::SMEM_BYTES;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = 2;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            GPBO_CUDA_TRY(cudaOccupancyMaxActiveClusters(&pairs, (const void *)tc::k_var_ei_tc, &cfg));
            if (pairs < 1) return GPBO_ENOTSUP;
            if (ctx->device >= 0 && ctx->device < 64) cached[ctx->device] = pairs;
        }
    }
    const int grid = 2 * std::max(1, std::min(P.num_tiles, pairs));
    tc::k_var_ei_tc<<<grid, tc::THREADS, tc::SMEM_BYTES, ctx->stream>>>(mk, ml, ml2, P);
    GPBO_LAUNCH_CHECK(ctx);
    *n_parts = grid;
    return GPBO_OK;
}

}  // namespace gpbo
