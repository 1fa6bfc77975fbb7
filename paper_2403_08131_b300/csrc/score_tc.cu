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
// Kernel shape (one CTA per SM, persistent over 128-candidate tiles):
//   warp 0      TMA producer: K* tile (128 x 64) and L^-1 tile (256 x 64) per stage,
//               128-byte swizzle, 4 stages of 48 KiB in shared memory
//   warp 1      allocates 512 TMEM columns; one lane issues tcgen05.mma (M=128, N=256,
//               K=16, FP32 accumulate) into one of two 256-column accumulators
//   warps 2..5  epilogue: tcgen05.ld the accumulator, square and sum into the candidate's
//               running |v|^2 (one TMEM lane = one candidate = one thread), then sigma,
//               EI and the per-CTA argmax
// For output chunk q (L^-1 rows 256q .. 256q+255) only K columns < 256(q+1) are read:
// the triangle's zero blocks are never loaded or multiplied.
// BF16 models carry a compensated inverse, hi = bf16(L^-1) and lo = bf16(L^-1 - hi); the
// K loop then runs twice (hi, then lo) into the same accumulator, so only K*'s rounding
// remains (twice the MMA work).  FP16 models run a single pass.
//
// Every mbarrier wait is bounded (the context's wait limit, about 2 s of SM clock by
// default).  On timeout the kernel sets DEV_TIMEOUT in the context's status word, every
// role leaves its loop, the producer waits (bounded by the default limit) for copies it
// issued, the MMA issuer drains its MMAs, and the allocating warp frees TMEM before the
// CTA exits.  gpbo_inject_wait_stall makes the epilogue wait on a barrier that nothing
// arrives at, so that tests can run this path without a fault.
#include "tc_common.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

namespace gpbo {

namespace tc {

constexpr int BM = 128;        // candidates per tile (MMA M, TMEM lanes)
constexpr int BN = TC_NCHUNK;  // L^-1 rows per output chunk (MMA N)
constexpr int BK = 64;         // K elements per stage (128 bytes of 16-bit values)
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int THREADS = 192;
constexpr int TMEM_COLS = 512;
constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;

struct Shared {
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint64_t drain;
    uint64_t never;    // failure injection: a barrier that nothing arrives at
    uint32_t tmem_base;
    int abort;
    float best_v[4];
    int64_t best_i[4];
};

using namespace tcx;

// Instruction descriptor for this kernel's MMA: N = 256, M = 128.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt) { return idesc_f16(fmt, BN, BM); }

struct Params {
    int64_t C;        // candidates in this chunk
    int64_t c0;       // pool index of the chunk's first candidate
    int n_pad;
    int num_tiles;
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

__global__ void __launch_bounds__(THREADS, 1)
    k_var_ei_tc(const __grid_constant__ CUtensorMap map_k, const __grid_constant__ CUtensorMap map_l,
                const __grid_constant__ CUtensorMap map_l2, Params P)
{
    extern __shared__ unsigned char smraw[];
    unsigned char *tiles = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    Shared *sh = (Shared *)(tiles + (size_t)STAGES * STAGE_BYTES);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int nq = P.n_pad / BN;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&sh->full[s], 1);
            mbar_init(&sh->empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&sh->acc_full[a], 1);
            mbar_init(&sh->acc_empty[a], 4);
        }
        mbar_init(&sh->drain, 1);
        mbar_init(&sh->never, 1);
        sh->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh->tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
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
            int armed[STAGES];
            uint32_t armed_par[STAGES];
            for (int s = 0; s < STAGES; ++s) armed[s] = 0, armed_par[s] = 0;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < P.num_tiles; t += gridDim.x) {
                for (int q = 0; ok && q < nq; ++q) {
                    const int ksteps = (q + 1) * (BN / BK);
                    // the compensated form runs the K loop twice: hi operand, then lo
                    for (int ks2 = 0; ks2 < ksteps * (1 + P.split); ++ks2) {
                        const int ks = ks2 < ksteps ? ks2 : ks2 - ksteps;
                        if (!mbar_wait_fast(&sh->empty[stage], phase ^ 1u, abort_flag, P.status)) { ok = false; break; }
                        unsigned char *a = tiles + (size_t)stage * STAGE_BYTES;
                        unsigned char *b = a + A_BYTES;
                        mbar_arrive_expect_tx(&sh->full[stage], STAGE_BYTES);
                        armed[stage] = 1;
                        armed_par[stage] = phase;
                        tma_load_2d(a, &map_k, ks * BK, t * BM, &sh->full[stage]);
                        tma_load_2d(b, ks2 < ksteps ? &map_l : &map_l2, ks * BK, q * BN, &sh->full[stage]);
                        if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                    }
                }
            }
            // leave no copy in flight: wait for the last arming of every stage
            for (int s = 0; s < STAGES; ++s)
                if (armed[s]) mbar_wait(&sh->full[s], armed_par[s], abort_flag, P.status, false);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < P.num_tiles; t += gridDim.x) {
                for (int q = 0; ok && q < nq; ++q) {
                    if (!mbar_wait_fast(&sh->acc_empty[acc], acc_phase ^ 1u, abort_flag, P.status)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t d_tmem = tmem + (uint32_t)(acc * BN);
                    const int ksteps = (q + 1) * (BN / BK) * (1 + P.split);
                    for (int ks = 0; ks < ksteps; ++ks) {
                        if (!mbar_wait_fast(&sh->full[stage], phase, abort_flag, P.status)) { ok = false; break; }
                        tc_fence_after();
                        const unsigned char *a = tiles + (size_t)stage * STAGE_BYTES;
                        const unsigned char *b = a + A_BYTES;
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk)
                            mma_f16(d_tmem, smem_desc(a + kk * 32), smem_desc(b + kk * 32), P.idesc,
                                    (ks > 0 || kk > 0) ? 1u : 0u);
                        mma_commit(&sh->empty[stage]);
                        if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                    }
                    if (!ok) break;
                    mma_commit(&sh->acc_full[acc]);
                    if (++acc == 2) { acc = 0; acc_phase ^= 1u; }
                }
            }
            // drain every MMA this thread issued before TMEM is released
            mma_commit(&sh->drain);
            mbar_wait(&sh->drain, 0, abort_flag, P.status, false);
        }
    } else {
        // ---------------- epilogue: warps 2..5, TMEM lane quadrant = warp % 4
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(quad * 32) << 16;
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
        for (int t = blockIdx.x; ok && t < P.num_tiles; t += gridDim.x) {
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
                if (lane == 0) mbar_arrive(&sh->acc_empty[acc]);
                if (++acc == 2) { acc = 0; acc_phase ^= 1u; }
            }
            if (!ok) break;
            const int64_t cl = (int64_t)t * BM + row;
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
    tc_fence_after();
    if (threadIdx.x == 0) {
        float bv = sh->best_v[0];
        int64_t bi = sh->best_i[0];
        for (int w = 1; w < 4; ++w)
            if (better(sh->best_v[w], sh->best_i[w], bv, bi)) { bv = sh->best_v[w]; bi = sh->best_i[w]; }
        P.part_ei[blockIdx.x] = bv;
        P.part_idx[blockIdx.x] = bi;
    }
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
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
    GPBO_TRY(encode_2d(&ml, dt, m->Linv16, (uint64_t)m->n_pad, (uint64_t)m->n_pad, tc::BN));
    GPBO_TRY(encode_2d(&ml2, dt, (const uint16_t *)m->Linv16 + (split ? sq : 0), (uint64_t)m->n_pad,
                       (uint64_t)m->n_pad, tc::BN));
    GPBO_TRY(ensure_smem((const void *)tc::k_var_ei_tc, ctx->device, (int)tc::SMEM_BYTES));
    tc::Params P;
    P.C = C;
    P.c0 = c0;
    P.n_pad = m->n_pad;
    P.num_tiles = (int)cdiv64(C, tc::BM);
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
    const int grid = std::min(P.num_tiles, ctx->sm_count);
    tc::k_var_ei_tc<<<grid, tc::THREADS, tc::SMEM_BYTES, ctx->stream>>>(mk, ml, ml2, P);
    GPBO_LAUNCH_CHECK(ctx);
    *n_parts = grid;
    return GPBO_OK;
}

}  // namespace gpbo
