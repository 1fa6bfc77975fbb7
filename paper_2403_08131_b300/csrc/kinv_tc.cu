// K^-1 = L^-T L^-1 on the tensor cores at FP64 accuracy, for the gradient of the log marginal
// likelihood: [K^-1]_pq = sum_k L^-1_kp L^-1_kq, a dense contraction over k >= max(p, q).
//
// The same error-free splitting as the tensor-core Cholesky update (Ozaki, Ogita, Oishi and
// Rump 2012): column p of L^-1 is 2^(e_p - 7) times 7 integer slices of at most 8 bits (exact in
// BF16), e_p putting the column's largest |entry| just below 2^e_p.  Slice products are exact
// integers; the 34 pairs with s + t <= 9 are summed per level s + t in eight FP32 accumulators
// (512 TMEM columns).  Over 128 values of k a level's sum stays below 7 x 128 x 2^14 < 2^24, so
// every FP32 partial sum is an exact integer; after each 128 of k the levels are read back as
// integers and folded into two int64 sums per element (hi: levels 2..5, lo: 6..9, by Horner),
// and the next 128 start from zero.  At the end
//     K^-1_pq = 2^(e_p + e_q - 38) hi + 2^(e_p + e_q - 70) lo,
// each part built as a double on the integer pipe and added in FP64.
//
//   k_kinv_split   (L^-1)^T's rows (= L^-1's columns): exponent and 7 BF16 slices, slice-major
//                  [s][p][k], through a 32 x 32 shared-memory transpose
//   k_kinv_tc      one CTA per 128 x 64 lower tile (two block rows, one block column); k runs
//                  from max(row0, col0) in chunks of 64: TMA of 7 + 7 slice tiles (168 KiB),
//                  34 x 4 MMAs (M = 128, N = 64, K = 16), fold every two chunks; the next
//                  chunk's copies start while the fold runs
// Every mbarrier wait is bounded; on timeout DEV_TIMEOUT is raised, the CTA waits (bounded) for
// its copies and MMAs and frees TMEM.
#include "tc_common.cuh"

#include <cuda_bf16.h>

namespace gpbo {

namespace ktc {

constexpr int SLICES = 7;
constexpr int LEVEL_MAX = 9;
constexpr int BM = 128, BN = 64, BK = 64;
constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
constexpr int THREADS = 256;
constexpr int TMEM_COLS = 512;
constexpr size_t SMEM_BYTES = (size_t)SLICES * (A_BYTES + B_BYTES) + 1024 + 1024;

using namespace tcx;

// Pass 1: e_p for each column p of L^-1 (n_pad x n_pad row-major).  One CTA of 256 threads per
// 32 columns: 8 row groups, warp-coalesced reads of 32 consecutive columns.
__global__ void __launch_bounds__(256) k_kinv_exp(const double *__restrict__ Li, int n_pad, int *__restrict__ exps)
{
    __shared__ unsigned long long mx[8][32];
    const int p = blockIdx.x * 32 + (threadIdx.x & 31), rg = threadIdx.x >> 5;
    unsigned long long m = 0;
    for (int k = rg; k < n_pad; k += 8) m = max(m, (unsigned long long)mag_bits(Li[(int64_t)k * n_pad + p]));
    mx[rg][threadIdx.x & 31] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        for (int g = 1; g < 8; ++g) m = max(m, mx[g][threadIdx.x]);
        exps[p] = exp_of_mag(m);
    }
}

// Pass 2: slices.  CTA (bx, by) handles columns 32 bx .. and k rows 32 by ..: reads the 32 x 32
// block row-wise, writes slice s of output row p (= column p) contiguously in k.
__global__ void __launch_bounds__(256) k_kinv_split(const double *__restrict__ Li, int n_pad, const int *__restrict__ exps,
                                                    __nv_bfloat16 *__restrict__ slices)
{
    __shared__ double t[32][33];
    const int p0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < 32; r += 8) t[r][tx] = Li[(int64_t)(k0 + r) * n_pad + p0 + tx];  // t[k][p]
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int p = p0 + r;
        uint16_t d[SLICES];
        split7(fixed55(t[tx][r], exps[p]), d);  // element (k0 + tx, p)
        uint16_t *out = reinterpret_cast<uint16_t *>(slices);
#pragma unroll
        for (int s = 0; s < SLICES; ++s) out[((int64_t)s * n_pad + p) * n_pad + k0 + tx] = d[s];
    }
}

struct Shared {
    uint64_t full;  // a chunk's copies have landed (one phase per chunk)
    uint64_t done;  // a chunk's MMAs have completed (one phase per chunk; thread 0 only)
    uint64_t fold;  // the MMAs before a fold have completed (one phase per fold)
    uint32_t tmem_base;
    int abort;
    int er[BM];
    int ec[BN];
};

struct Params {
    double *C;  // n_pad x n_pad, lower tiles written
    const int *exps;
    unsigned *status;
    int n_pad, nblk;
    uint32_t idesc;
};

// Tile t -> (strip i2, block column jb), strips of two block rows over the whole matrix.
__device__ __forceinline__ void tile_coords(int t, int nblk, int &i2, int &jb)
{
    i2 = 0;
    for (;; ++i2) {
        const int c = min(2 * i2 + 2, nblk);
        if (t < c) break;
        t -= c;
    }
    jb = t;
}

__global__ void __launch_bounds__(THREADS, 1)
    k_kinv_tc(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b, Params P)
{
    extern __shared__ unsigned char smraw[];
    unsigned char *tiles = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char *sa = tiles, *sb = tiles + (size_t)SLICES * A_BYTES;
    Shared *sh = (Shared *)(sb + (size_t)SLICES * B_BYTES);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    int i2, jb;
    tile_coords(blockIdx.x, P.nblk, i2, jb);
    const int row0 = 2 * i2 * NB, col0 = jb * NB;
    const int kbeg = max(row0, col0), nchunk = (P.n_pad - kbeg) / BK;

    if (threadIdx.x == 0) {
        mbar_init(&sh->full, 1);
        mbar_init(&sh->done, 1);
        mbar_init(&sh->fold, 1);
        sh->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    for (int i = threadIdx.x; i < BM; i += THREADS) sh->er[i] = row0 + i < P.n_pad ? P.exps[row0 + i] : 0;
    for (int i = threadIdx.x; i < BN; i += THREADS) sh->ec[i] = P.exps[col0 + i];
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

    const int quad = warp & 3, half = warp >> 2;
    const int row = quad * 32 + lane;
    const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16);
    long long hi[32], lo[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) hi[j] = lo[j] = 0;

    // thread 0: copies of chunk c (the buffers are free once chunk c-1's MMAs completed)
    auto load = [&](int c) {
        mbar_arrive_expect_tx(&sh->full, SLICES * (A_BYTES + B_BYTES));
        const int k = kbeg + c * BK;
        for (int s = 0; s < SLICES; ++s) {
            tma_load_2d(sa + (size_t)s * A_BYTES, &map_a, k, s * P.n_pad + row0, &sh->full);
            tma_load_2d(sb + (size_t)s * B_BYTES, &map_b, k, s * P.n_pad + col0, &sh->full);
        }
    };
    bool ok = true;
    int armed = 0;  // chunks whose copies were issued
    if (threadIdx.x == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&map_a) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&map_b) : "memory");
        if (nchunk > 0) {
            load(0);
            armed = 1;
        }
    }
    for (int c = 0; c < nchunk; ++c) {
        if (threadIdx.x == 0 && ok) {
            if (!mbar_wait(&sh->full, (uint32_t)c & 1u, abort_flag, P.status)) {
                ok = false;
            } else {
                tc_fence_after();
                for (int l = 2; l <= LEVEL_MAX; ++l) {
                    const uint32_t d = tmem + (uint32_t)((l - 2) * BN);
                    bool first = (c & 1) == 0;  // each 128 of k starts the levels from zero
                    for (int s = 1; s <= SLICES; ++s) {
                        const int t = l - s;
                        if (t < 1 || t > SLICES) continue;
                        const unsigned char *a = sa + (size_t)(s - 1) * A_BYTES;
                        const unsigned char *b = sb + (size_t)(t - 1) * B_BYTES;
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk)
                            mma_f16(d, smem_desc(a + kk * 32), smem_desc(b + kk * 32), P.idesc,
                                    (first && kk == 0) ? 0u : 1u);
                        first = false;
                    }
                }
                mma_commit(&sh->done);
                // the warps that fold wait on a barrier of their own: one that only moves at folds
                // can never be two phases ahead of them (a parity wait cannot tell those apart)
                if ((c & 1) == 1 || c + 1 == nchunk) mma_commit(&sh->fold);
                // the next chunk's copies once these MMAs have read the buffers
                if (c + 1 < nchunk) {
                    if (!mbar_wait(&sh->done, (uint32_t)c & 1u, abort_flag, P.status)) {
                        ok = false;
                    } else {
                        load(c + 1);
                        armed = c + 2;
                    }
                }
            }
            if (!ok) *abort_flag = 1;
        }
        // fold after every second chunk and after the last
        if ((c & 1) == 1 || c + 1 == nchunk) {
            const bool got = mbar_wait_inl(&sh->fold, (uint32_t)(c >> 1) & 1u, abort_flag, P.status);
            if (!__all_sync(0xffffffffu, got)) {
                ok = false;
                break;
            }
            tc_fence_after();
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                const int c0 = half * 32 + g * 16;
                long long h16[16], l16[16];
                uint32_t v[16];
                tmem_ld16_nw(taddr + (uint32_t)c0, v);
                tmem_wait();
                pin16(v);
#pragma unroll
                for (int j = 0; j < 16; ++j) h16[j] = __float2int_rn(__uint_as_float(v[j]));
#pragma unroll 1
                for (int l = 3; l <= 5; ++l) {
                    tmem_ld16_nw(taddr + (uint32_t)((l - 2) * BN + c0), v);
                    tmem_wait();
                    pin16(v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) h16[j] = h16[j] * 256 + __float2int_rn(__uint_as_float(v[j]));
                }
                tmem_ld16_nw(taddr + (uint32_t)(4 * BN + c0), v);
                tmem_wait();
                pin16(v);
#pragma unroll
                for (int j = 0; j < 16; ++j) l16[j] = __float2int_rn(__uint_as_float(v[j]));
#pragma unroll 1
                for (int l = 7; l <= LEVEL_MAX; ++l) {
                    tmem_ld16_nw(taddr + (uint32_t)((l - 2) * BN + c0), v);
                    tmem_wait();
                    pin16(v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) l16[j] = l16[j] * 256 + __float2int_rn(__uint_as_float(v[j]));
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    hi[g * 16 + j] += h16[j];
                    lo[g * 16 + j] += l16[j];
                }
            }
            tc_fence_before();
            __syncthreads();  // every warp has read TMEM before the next MMAs overwrite it
            tc_fence_after();
            if (*abort_flag) {
                ok = false;
                break;
            }
        }
    }
    // ---- write the tile's lower blocks
    if (ok) {
        const int r = row0 + row;
        if (r < P.n_pad && r / NB >= jb) {
            const int er = sh->er[row];
            double *dst = P.C + (int64_t)r * P.n_pad + col0 + half * 32;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int E = er + sh->ec[half * 32 + j];
                dst[j] = scaled_to_double(hi[j], E - 38) + scaled_to_double(lo[j], E - 70);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        // leave no copy or MMA in flight before TMEM and the CTA go away
        if (armed > 0) mbar_wait(&sh->full, (uint32_t)(armed - 1) & 1u, abort_flag, P.status, false);
        if (nchunk > 0) mbar_wait(&sh->done, (uint32_t)(nchunk - 1) & 1u, abort_flag, P.status, false);
    }
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

}  // namespace ktc

size_t kinv_tc_slice_bytes(int n_pad) { return (size_t)ktc::SLICES * n_pad * n_pad * 2; }

// C (n_pad x n_pad, lower 64 x 64 tiles) = L^-T L^-1 from Linv (n_pad x n_pad FP64, lower).
// slices: kinv_tc_slice_bytes(n_pad) bytes; exps: n_pad ints (both device scratch).
int kinv_tc(gpbo_ctx *ctx, cudaStream_t st, const double *Linv, int n_pad, void *slices, int *exps, double *C)
{
    if (n_pad % 128 != 0) return GPBO_EINVAL;
    GPBO_TRY(ensure_smem((const void *)ktc::k_kinv_tc, ctx->device, (int)ktc::SMEM_BYTES));
    ktc::k_kinv_exp<<<n_pad / 32, 256, 0, st>>>(Linv, n_pad, exps);
    GPBO_LAUNCH_CHECK(ctx);
    ktc::k_kinv_split<<<dim3(n_pad / 32, n_pad / 32), 256, 0, st>>>(Linv, n_pad, exps, (__nv_bfloat16 *)slices);
    GPBO_LAUNCH_CHECK(ctx);
    CUtensorMap ma, mb;
    const uint64_t rows = (uint64_t)ktc::SLICES * n_pad;
    GPBO_TRY(encode_2d_box(&ma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, slices, rows, (uint64_t)n_pad, ktc::BM, ktc::BK,
                           CU_TENSOR_MAP_SWIZZLE_128B));
    GPBO_TRY(encode_2d_box(&mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, slices, rows, (uint64_t)n_pad, ktc::BN, ktc::BK,
                           CU_TENSOR_MAP_SWIZZLE_128B));
    ktc::Params P;
    P.C = C;
    P.exps = exps;
    P.status = ctx->dev_status;
    P.n_pad = n_pad;
    P.nblk = n_pad / NB;
    P.idesc = tcx::idesc_f16(1u, ktc::BN, ktc::BM);
    int64_t tiles = 0;
    for (int i2 = 0; 2 * i2 < P.nblk; ++i2) tiles += std::min(2 * i2 + 2, P.nblk);
    ktc::k_kinv_tc<<<(unsigned)tiles, ktc::THREADS, ktc::SMEM_BYTES, st>>>(ma, mb, P);
    GPBO_LAUNCH_CHECK(ctx);
    return GPBO_OK;
}

}  // namespace gpbo
