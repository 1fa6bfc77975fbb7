// Trailing update of the FP64 Cholesky factorisation on the tensor cores (tcgen05), at FP64
// accuracy, by exact products of 8-bit integer slices (the error-free splitting of Ozaki, Ogita,
// Oishi and Rump, Numer. Algorithms 59, 2012).
//
// Step kb of the right-looking factorisation subtracts P P^T from the trailing lower tiles,
// P = L[rows below, block column kb] (64 columns).  Each row r of P is written as
//     P_r = 2^(e_r - 7) (a_1 + 2^-8 a_2 + ... + 2^-48 a_7) + rest,    |a_s| <= 128 integers,
// with e_r the exponent that puts the row's largest |entry| just below 2^e_r and a_1 .. a_7 the
// balanced base-256 digits of the integer round(x 2^(55 - e_r)), taken on the integer pipe from
// the bits of x (|rest| <= 2^(e_r - 56)).  A slice is exact in BF16, a product of two is an integer below 2^14, and up to
// 7 x 64 of them sum below 2^23: every partial sum of a tensor-core MMA with FP32 accumulation
// is an exact integer, whatever the order or rounding mode.  Products of slices s and t carry
// the weight 2^(e_r + e_c - 14 - 8 (s + t - 2)); the kernel keeps the 34 pairs with
// s + t <= 9, summing each level s + t in its own FP32 accumulator (8 levels x 64 columns = 512
// TMEM columns), and combines the levels exactly in int64 before two FP64 FMAs per element.  The terms left out weigh
// below 2^-56 |P_r| |P_c| per product, and the result is within a small multiple of FP64
// rounding of the exact P P^T (measured on Cholesky panels of the Matern kernel matrices: at
// or below the error of an FP64 dot product, relative to |P_r| |P_c|).
//
//   k_chol_split      one warp per row of P: e_r and the seven BF16 slices, stored slice-major
//                     (slice s, row r: 64 contiguous values, 128 bytes)
//   k_chol_update_tc  one CTA per 128 x 64 output tile (two block rows, one block column) of
//                     block columns kb+2 .. (the next column is updated on the side stream):
//                     TMA of the 7 + 7 slice tiles (168 KiB), one thread issues 34 x 4 MMAs
//                     (M = 128, N = 64, K = 16, BF16, FP32 accumulate), then 8 warps read the
//                     8 accumulators back, combine them and subtract from A.
// Every mbarrier wait is bounded; on timeout DEV_TIMEOUT is raised, the copies and MMAs the
// CTA issued are waited for (bounded) and TMEM is freed before the CTA exits.
#include "tc_common.cuh"

#include <cuda_bf16.h>

#include <algorithm>

namespace gpbo {

namespace ctc {

constexpr int SLICES = 7;
constexpr int LEVEL_MAX = 9;         // keep slice pairs s + t <= 9
constexpr int BM = 128, BN = 64, BK = 64;
constexpr int A_BYTES = BM * BK * 2;  // one slice of the row strip
constexpr int B_BYTES = BN * BK * 2;  // one slice of the column block
constexpr int THREADS = 256;
constexpr int TMEM_COLS = 512;
constexpr size_t SMEM_BYTES = (size_t)SLICES * (A_BYTES + B_BYTES) + 1024 + 1024;

struct Shared {
    uint64_t full;
    uint64_t done;
    uint32_t tmem_base;
    int abort;
    int er[BM];
    int ec[BN];
};

using namespace tcx;

// Rows r0 .. n_pad - 1 of panel kb of A: one warp per row (warp index w = r - r0).
__device__ __forceinline__ void chol_split_row(const double *__restrict__ A, int n_pad, int kb, int r0, int w,
                                               __nv_bfloat16 *__restrict__ slices, int *__restrict__ exps)
{
    const int lane = threadIdx.x & 31;
    const int r = r0 + w;
    if (r >= n_pad) return;
    const double *row = A + (int64_t)r * n_pad + (int64_t)kb * NB;
    const double2 v = *reinterpret_cast<const double2 *>(row + 2 * lane);
    unsigned long long mx = max(mag_bits(v.x), mag_bits(v.y));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int e = exp_of_mag(mx);
    uint16_t d0[SLICES], d1[SLICES];
    split7(fixed55(v.x, e), d0);
    split7(fixed55(v.y, e), d1);
#pragma unroll
    for (int s = 0; s < SLICES; ++s)
        *reinterpret_cast<uint32_t *>(slices + ((int64_t)s * n_pad + r) * BK + 2 * lane) =
            (uint32_t)d0[s] | ((uint32_t)d1[s] << 16);
    if (lane == 0) exps[r] = e;
}

__global__ void __launch_bounds__(256) k_chol_split(const double *__restrict__ A, int n_pad, int kb, int r0,
                                                    __nv_bfloat16 *__restrict__ slices, int *__restrict__ exps)
{
    chol_split_row(A, n_pad, kb, r0, (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), slices, exps);
}

// The batched form: problem blockIdx.y, its slices at row row_off of the arena.
__global__ void __launch_bounds__(256) k_chol_split_batched(const CholTcProb *__restrict__ probs, int kb,
                                                            __nv_bfloat16 *__restrict__ arena)
{
    const CholTcProb p = probs[blockIdx.y];
    if (!chol_tc_step(p.n_pad, p.nblk, kb)) return;
    chol_split_row(p.A, p.n_pad, kb, (kb + 2) * NB, (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5),
                   arena + p.row_off * BK, p.exps);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct Params {
    CholTcProb one;            // the problem of a single launch
    const CholTcProb *probs;   // or, batched: problem blockIdx.y (device)
    unsigned *status;
    int kb;                    // step: block rows / columns kb + 2 .. are updated by panel kb
    uint32_t idesc;
};

// Tile t -> (strip i2, block column jb): strip i2 covers block rows b0 + 2 i2 and b0 + 2 i2 + 1
// and meets block columns b0 .. min(b0 + 2 i2 + 1, nblk - 1).
__device__ __forceinline__ void tile_coords(int t, int b0, int nblk, int &i2, int &jb)
{
    const int T2 = nblk - b0;
    i2 = 0;
    for (;; ++i2) {
        const int c = min(2 * i2 + 2, T2);
        if (t < c) break;
        t -= c;
    }
    jb = b0 + t;
}

__global__ void __launch_bounds__(THREADS, 1)
    k_chol_update_tc(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b, Params P)
{
    extern __shared__ unsigned char smraw[];
    unsigned char *tiles = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char *sa = tiles;                                 // SLICES x A_BYTES
    unsigned char *sb = tiles + (size_t)SLICES * A_BYTES;      // SLICES x B_BYTES
    Shared *sh = (Shared *)(sb + (size_t)SLICES * B_BYTES);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const CholTcProb pr = P.probs ? P.probs[blockIdx.y] : P.one;
    // a problem without a tensor-core update at this step, or a tile beyond its count, leaves
    // before any barrier or tensor memory is touched
    if (!chol_tc_step(pr.n_pad, pr.nblk, P.kb) || (int64_t)blockIdx.x >= chol_tc_tiles(pr.nblk, P.kb)) return;
    const int n_pad = pr.n_pad, b0 = P.kb + 2;
    int i2, jb;
    tile_coords(blockIdx.x, b0, pr.nblk, i2, jb);
    const int row0 = (b0 + 2 * i2) * NB;  // first row of the strip
    const int col0 = jb * NB;

    if (threadIdx.x == 0) {
        mbar_init(&sh->full, 1);
        mbar_init(&sh->done, 1);
        sh->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    for (int i = threadIdx.x; i < BM; i += THREADS) sh->er[i] = row0 + i < n_pad ? pr.exps[row0 + i] : 0;
    for (int i = threadIdx.x; i < BN; i += THREADS) sh->ec[i] = pr.exps[col0 + i];
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

    bool issued = false;
    if (threadIdx.x == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&map_a) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&map_b) : "memory");
        mbar_arrive_expect_tx(&sh->full, SLICES * (A_BYTES + B_BYTES));
        for (int s = 0; s < SLICES; ++s) {
            const int base = (int)(pr.row_off + (int64_t)s * n_pad);
            tma_load_2d(sa + (size_t)s * A_BYTES, &map_a, 0, base + row0, &sh->full);
            tma_load_2d(sb + (size_t)s * B_BYTES, &map_b, 0, base + col0, &sh->full);
        }
        if (mbar_wait(&sh->full, 0, abort_flag, P.status)) {
            tc_fence_after();
            for (int l = 2; l <= LEVEL_MAX; ++l) {
                const uint32_t d = tmem + (uint32_t)((l - 2) * BN);
                bool first = true;
                for (int s = 1; s <= SLICES; ++s) {
                    const int t = l - s;
                    if (t < 1 || t > SLICES) continue;
                    const unsigned char *a = sa + (size_t)(s - 1) * A_BYTES;
                    const unsigned char *b = sb + (size_t)(t - 1) * B_BYTES;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk)
                        mma_f16(d, smem_desc(a + kk * 32), smem_desc(b + kk * 32), P.idesc, (first && kk == 0) ? 0u : 1u);
                    first = false;
                }
            }
            mma_commit(&sh->done);
            issued = true;
        } else {
            *abort_flag = 1;
            mbar_wait(&sh->full, 0, abort_flag, P.status, false);  // no copy left in flight
        }
    }

    // ---------------- epilogue: all 8 warps; TMEM lane quadrant = warp % 4, column half = warp / 4.
    // The accumulators hold exact integers below 2^23; they are read back as integers and folded
    // by Horner in int64, levels 2..5 into hi and 6..9 into lo (each below 2^47, so exact).  Then
    // C = hi 2^16 + floor(lo / 2^16) < 2^63 is the level sum times 2^40 to within one unit
    // (2^-54 |P_r|max |P_c|max in A's units, below the terms already left out), and
    // A -= C 2^(E - 40), E = e_r + e_c - 14, with the double built on the integer pipe: one FP64
    // operation per element, since the FP64 pipe is the scarce one.
    {
        const int quad = warp & 3, half = warp >> 2;
        const int row = quad * 32 + lane;
        const int r = row0 + row;
        const int ib = r / NB;
        const bool live = r < n_pad && ib >= jb;
        const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16);
        // this thread's 32 values of A, loaded while the copies and MMAs are in flight
        double2 pre[2][8];
        {
            const double *src = pr.A + (int64_t)r * n_pad + col0 + half * 32;
#pragma unroll
            for (int g = 0; g < 2; ++g)
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    pre[g][q] = live ? *reinterpret_cast<const double2 *>(src + g * 16 + 2 * q) : make_double2(0.0, 0.0);
        }
        const bool got = mbar_wait_inl(&sh->done, 0, abort_flag, P.status);
        if (__all_sync(0xffffffffu, got)) {
            tc_fence_after();
            const int er = sh->er[row];
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                const int c0 = half * 32 + g * 16;
                long long hi[16], lo[16];
                uint32_t v[16];
                tmem_ld16(taddr + (uint32_t)c0, v);
#pragma unroll
                for (int j = 0; j < 16; ++j) hi[j] = __float2int_rn(__uint_as_float(v[j]));
#pragma unroll 1
                for (int l = 3; l <= 5; ++l) {
                    tmem_ld16(taddr + (uint32_t)((l - 2) * BN + c0), v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) hi[j] = hi[j] * 256 + __float2int_rn(__uint_as_float(v[j]));
                }
                tmem_ld16(taddr + (uint32_t)(4 * BN + c0), v);
#pragma unroll
                for (int j = 0; j < 16; ++j) lo[j] = __float2int_rn(__uint_as_float(v[j]));
#pragma unroll 1
                for (int l = 7; l <= LEVEL_MAX; ++l) {
                    tmem_ld16(taddr + (uint32_t)((l - 2) * BN + c0), v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) lo[j] = lo[j] * 256 + __float2int_rn(__uint_as_float(v[j]));
                }
                if (live) {
                    double *dst = pr.A + (int64_t)r * n_pad + col0 + c0;
#pragma unroll
                    for (int j = 0; j < 16; j += 2) {
                        double2 a = pre[g][j / 2];
                        const long long C0 = hi[j] * 65536 + (lo[j] >> 16), C1 = hi[j + 1] * 65536 + (lo[j + 1] >> 16);
                        a.x -= scaled_to_double(C0, er + sh->ec[c0 + j] - 54);
                        a.y -= scaled_to_double(C1, er + sh->ec[c0 + j + 1] - 54);
                        *reinterpret_cast<double2 *>(dst + j) = a;
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && issued) mbar_wait(&sh->done, 0, abort_flag, P.status, false);  // MMAs drained
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// ---------------------------------------------------------------------------------------------
// The persistent form of the update (single model).  Same slice pairs, levels and per-element
// arithmetic as k_chol_update_tc, so the two give the same bits; what changes is the schedule
// and the shape of the MMAs.  A tcgen05 MMA of M = 128 costs the tensor pipe about as much to
// read its operands as a product of N = 128 takes to compute, so the 34 pairs are not issued
// as 34 narrow products.  For each row slice s, one MMA multiplies a_s by the tile's column
// slices t = 1 .. n_s stacked along N (n_s = min(7, 9 - s)); the product of pair (s, t) lands
// in columns 32 (s + t - 2) .. of the accumulator, the block of level s + t, so each level's
// pairs still sum in their own FP32 accumulator, exactly.  Per K step of 16: 7 MMAs of
// N = 32 n_s (1088 columns in all, the 34 pairs and nothing else).  The first MMA of a tile
// (s = 1, first K step) overwrites the accumulator: it also covers level 9's block, with a
// zero block kept after each stage's seventh slice as its B rows.
// One CTA per SM walks work items: an item is up to PCH tiles of 128 rows x 32 columns in one
// strip, whose 7 row slices (112 KiB) are loaded once for the item while the column slices
// (28 KiB per tile) stream through PSTAGES stages.  Two accumulators of 8 levels x 32 columns
// fill the 512 TMEM columns: the epilogue of one tile overlaps the MMAs of the next.
//   warp 0       TMA producer
//   warp 1       allocates 512 TMEM columns; one lane issues the 28 MMAs of each tile and
//                commits them to the stage, accumulator and item barriers
//   warps 2..17  epilogue: TMEM lane quadrant warp % 4, columns 8 ((warp - 2) / 4) .. of the tile
// The launch leaves CHAIN_SMS SMs free for the 64 x 64 kernels of the factorisation's chain.
constexpr int PBN = 32;                         // output columns per tile
constexpr int PCH = 8;                          // tiles per work item, at most
constexpr int PSTAGES = 3;
constexpr int CHAIN_SMS = 8;                    // SMs left to the factorisation's chain
constexpr int PB_SLICE = PBN * BK * 2;          // one slice of a tile's column rows (4 KiB)
constexpr int PB_STAGE = (SLICES + 1) * PB_SLICE;  // 7 slices and the zero block
constexpr int PA_BYTES = SLICES * A_BYTES;
constexpr int PEPI_WARPS = 16;
constexpr int PCOLS = PBN / (PEPI_WARPS / 4);   // columns per epilogue thread
static_assert(PCOLS == 8, "the epilogue reads 8 column exponents as two int4");
constexpr int PTHREADS = 32 * (2 + PEPI_WARPS);
constexpr int ACC_COLS = (LEVEL_MAX - 1) * PBN; // one accumulator: levels 2 .. 9
static_assert(2 * ACC_COLS <= TMEM_COLS, "tensor memory");
constexpr size_t PSMEM_BYTES = 1024 + (size_t)PA_BYTES + (size_t)PSTAGES * PB_STAGE + 256;

struct PShared {
    uint64_t a_full;      // the item's row slices have landed
    uint64_t a_empty;     // the item's MMAs are complete (the row-slice buffer may be refilled)
    uint64_t b_full[PSTAGES], b_empty[PSTAGES];
    uint64_t acc_full[2], acc_empty[2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
};
static_assert(sizeof(PShared) <= 256, "barrier area");

struct PItem {
    int row0;   // first row of the strip
    int tile0;  // first tile, in units of PBN columns
    int nt;     // tiles
};

// Work items of one step: strips of two block rows from block row b0 (the last may hold one),
// strip i2 meeting block columns c0 .. min(b0 + 2 i2 + 1, nblk - 1), each cut into items of at
// most PCH tiles; the strips that meet the most columns come first.
__host__ __device__ inline int p_strip_tiles(int i2, int b0, int c0, int nblk)
{
    const int last = b0 + 2 * i2 + 1 < nblk - 1 ? b0 + 2 * i2 + 1 : nblk - 1;
    return (NB / PBN) * (last - c0 + 1);
}
__host__ __device__ inline int p_items(int b0, int c0, int nblk)
{
    int n = 0;
    for (int i2 = 0; b0 + 2 * i2 < nblk; ++i2) n += (p_strip_tiles(i2, b0, c0, nblk) + PCH - 1) / PCH;
    return n;
}
__device__ inline bool p_item(int it, int b0, int c0, int nblk, PItem &out)
{
    const int S = (nblk - b0 + 1) / 2;
    for (int i2 = S - 1; i2 >= 0; --i2) {
        const int nt = p_strip_tiles(i2, b0, c0, nblk), ch = (nt + PCH - 1) / PCH;
        if (it < ch) {
            out.row0 = (b0 + 2 * i2) * NB;
            out.tile0 = (NB / PBN) * c0 + it * PCH;
            out.nt = nt - it * PCH < PCH ? nt - it * PCH : PCH;
            return true;
        }
        it -= ch;
    }
    return false;
}

struct PParams {
    double *A;
    const int *exps;
    unsigned *status;
    int n_pad, nblk, kb;
    int b0, c0;        // first block row / block column updated
    int items;
};

__device__ __forceinline__ void tmem_ld8_nw(uint32_t taddr, uint32_t *r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
__device__ __forceinline__ void pin8(uint32_t *r)
{
    asm volatile("" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]));
}

// An exact integer |x| <= 2^22 held in FP32, as an int: x + 1.5 2^23 lies in [2^23, 2^24], where
// FP32 steps by 1, so the sum is exact and its low bits are x + 2^22 (one FP32 add and one
// integer subtract instead of a conversion).  Levels 2 .. 5 stay within this range: at most
// 4 pairs x 64 products of |a_s a_t| <= 2^14.
__device__ __forceinline__ int small_int_of(uint32_t bits)
{
    return (int)(__float_as_uint(__fadd_rn(__uint_as_float(bits), 12582912.0f)) - 0x4B400000u);
}

__global__ void __launch_bounds__(PTHREADS, 1)
    k_chol_update_tcp(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b, PParams P)
{
    extern __shared__ unsigned char smraw[];
    unsigned char *sa = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);  // SLICES x A_BYTES
    unsigned char *sb = sa + PA_BYTES;                                                      // PSTAGES x PB_STAGE
    PShared *sh = (PShared *)(sb + (size_t)PSTAGES * PB_STAGE);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int n_pad = P.n_pad;

    // the zero block after each stage's seventh slice (never written by the copies)
    for (int i = threadIdx.x; i < PSTAGES * PB_SLICE / 16; i += PTHREADS) {
        const int st = i / (PB_SLICE / 16), o = i % (PB_SLICE / 16);
        *reinterpret_cast<uint4 *>(sb + (size_t)st * PB_STAGE + (size_t)SLICES * PB_SLICE + (size_t)o * 16) =
            make_uint4(0u, 0u, 0u, 0u);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        mbar_init(&sh->a_full, 1);
        mbar_init(&sh->a_empty, 1);
        for (int s = 0; s < PSTAGES; ++s) {
            mbar_init(&sh->b_full[s], 1);
            mbar_init(&sh->b_empty[s], 1);
        }
        for (int u = 0; u < 2; ++u) {
            mbar_init(&sh->acc_full[u], 1);
            mbar_init(&sh->acc_empty[u], PEPI_WARPS);
        }
        mbar_init(&sh->drain, 1);
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
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&map_a) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&map_b) : "memory");
            int a_armed = 0, b_armed = 0;
            bool ok = true;
            for (int it = blockIdx.x; ok && it < P.items; it += gridDim.x) {
                PItem w;
                p_item(it, P.b0, P.c0, P.nblk, w);
                // the row-slice buffer is free once the previous item's MMAs are complete
                if (a_armed > 0 && !mbar_wait(&sh->a_empty, (a_armed - 1) & 1, abort_flag, P.status)) break;
                mbar_arrive_expect_tx(&sh->a_full, PA_BYTES);
                ++a_armed;
                for (int s = 0; s < SLICES; ++s)
                    tma_load_2d(sa + (size_t)s * A_BYTES, &map_a, 0, s * n_pad + w.row0, &sh->a_full);
                for (int t = 0; t < w.nt; ++t) {
                    const int st = b_armed % PSTAGES, use = b_armed / PSTAGES;
                    if (use > 0 && !mbar_wait(&sh->b_empty[st], (use - 1) & 1, abort_flag, P.status)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&sh->b_full[st], SLICES * PB_SLICE);
                    ++b_armed;
                    const int col = (w.tile0 + t) * PBN;
                    for (int s = 0; s < SLICES; ++s)
                        tma_load_2d(sb + (size_t)st * PB_STAGE + (size_t)s * PB_SLICE, &map_b, 0, s * n_pad + col,
                                    &sh->b_full[st]);
                }
            }
            // every copy issued has landed before the CTA may exit (a no-op unless aborted)
            if (a_armed > 0) mbar_wait(&sh->a_full, (a_armed - 1) & 1, abort_flag, P.status, false);
            for (int st = 0; st < PSTAGES; ++st) {
                const int uses = (b_armed - st + PSTAGES - 1) / PSTAGES;
                if (uses > 0) mbar_wait(&sh->b_full[st], (uses - 1) & 1, abort_flag, P.status, false);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int ia = 0, bc = 0, tcount = 0;
            bool ok = true, issued = false;
            for (int it = blockIdx.x; ok && it < P.items; it += gridDim.x, ++ia) {
                PItem w;
                p_item(it, P.b0, P.c0, P.nblk, w);
                if (!mbar_wait(&sh->a_full, ia & 1, abort_flag, P.status)) break;
                tc_fence_after();
                for (int t = 0; t < w.nt; ++t, ++bc, ++tcount) {
                    const int st = bc % PSTAGES, u = tcount & 1;
                    if (tcount >= 2 && !mbar_wait(&sh->acc_empty[u], ((tcount >> 1) - 1) & 1, abort_flag, P.status)) {
                        ok = false;
                        break;
                    }
                    if (!mbar_wait(&sh->b_full[st], (bc / PSTAGES) & 1, abort_flag, P.status)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d0 = tmem + (uint32_t)(u * ACC_COLS);
                    const unsigned char *bst = sb + (size_t)st * PB_STAGE;
#pragma unroll 1
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint64_t bdesc = smem_desc(bst + kk * 32);
#pragma unroll
                        for (int s = 1; s <= SLICES; ++s) {
                            const bool init = kk == 0 && s == 1;
                            const int nt = init ? LEVEL_MAX - 1 : (SLICES < LEVEL_MAX - s ? SLICES : LEVEL_MAX - s);
                            mma_f16(d0 + (uint32_t)((s - 1) * PBN), smem_desc(sa + (size_t)(s - 1) * A_BYTES + kk * 32),
                                    bdesc, idesc_f16(1u, nt * PBN, BM), init ? 0u : 1u);
                        }
                    }
                    issued = true;
                    mma_commit(&sh->b_empty[st]);
                    mma_commit(&sh->acc_full[u]);
                }
                mma_commit(&sh->a_empty);
            }
            if (issued) {
                mma_commit(&sh->drain);
                mbar_wait(&sh->drain, 0, abort_flag, P.status, false);  // every MMA complete
            }
        }
    } else {
        // epilogue: the sums of k_chol_update_tc's fold (the same integers: the four levels of
        // each half combined as two int32 pairs, (L_l 256 + L_l+1) 2^16 + (L_l+2 256 + L_l+3)),
        // then the same FP64 build, for PCOLS columns of one row per thread
        const int q = warp & 3, g = (warp - 2) >> 2;
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
        int tcount = 0;
        bool ok = true;
        for (int it = blockIdx.x; ok && it < P.items; it += gridDim.x) {
            PItem w;
            p_item(it, P.b0, P.c0, P.nblk, w);
            const int r = w.row0 + q * 32 + lane;
            const bool rin = r < n_pad;
            const int er = rin ? P.exps[r] : 0;
            for (int t = 0; t < w.nt; ++t, ++tcount) {
                const int u = tcount & 1;
                const int c0 = (w.tile0 + t) * PBN + PCOLS * g;
                const bool live = rin && r / NB >= c0 / NB;
                double *dst = P.A + (int64_t)r * n_pad + c0;
                double2 pre[PCOLS / 2];
#pragma unroll
                for (int j = 0; j < PCOLS / 2; ++j)
                    pre[j] = live ? *reinterpret_cast<const double2 *>(dst + 2 * j) : make_double2(0.0, 0.0);
                const int4 e0 = *reinterpret_cast<const int4 *>(P.exps + c0);
                const int4 e1 = *reinterpret_cast<const int4 *>(P.exps + c0 + 4);
                const bool got = mbar_wait_inl(&sh->acc_full[u], (tcount >> 1) & 1, abort_flag, P.status);
                if (!__all_sync(0xffffffffu, got)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t ta = tl + (uint32_t)(u * ACC_COLS + PCOLS * g);
                long long hi[PCOLS], lo[PCOLS];
                {
                    uint32_t v[4][PCOLS];
#pragma unroll
                    for (int k = 0; k < 4; ++k) tmem_ld8_nw(ta + (uint32_t)(k * PBN), v[k]);  // levels 2..5
                    tmem_wait();
#pragma unroll
                    for (int k = 0; k < 4; ++k) pin8(v[k]);
#pragma unroll
                    for (int j = 0; j < PCOLS; ++j) {
                        const int t0 = small_int_of(v[0][j]) * 256 + small_int_of(v[1][j]);
                        const int t1 = small_int_of(v[2][j]) * 256 + small_int_of(v[3][j]);
                        hi[j] = (long long)t0 * 65536 + t1;
                    }
                }
                {
                    uint32_t v[4][PCOLS];
#pragma unroll
                    for (int k = 0; k < 4; ++k) tmem_ld8_nw(ta + (uint32_t)((4 + k) * PBN), v[k]);  // levels 6..9
                    tmem_wait();
#pragma unroll
                    for (int k = 0; k < 4; ++k) pin8(v[k]);
                    // this warp is done with the accumulator
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sh->acc_empty[u]);
#pragma unroll
                    for (int j = 0; j < PCOLS; ++j) {
                        const int t0 =
                            __float2int_rn(__uint_as_float(v[0][j])) * 256 + __float2int_rn(__uint_as_float(v[1][j]));
                        const int t1 =
                            __float2int_rn(__uint_as_float(v[2][j])) * 256 + __float2int_rn(__uint_as_float(v[3][j]));
                        lo[j] = (long long)t0 * 65536 + t1;
                    }
                }
                if (live) {
                    const int ec[PCOLS] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
#pragma unroll
                    for (int j = 0; j < PCOLS; j += 2) {
                        double2 a = pre[j / 2];
                        const long long C0 = hi[j] * 65536 + (lo[j] >> 16), C1 = hi[j + 1] * 65536 + (lo[j + 1] >> 16);
                        a.x -= scaled_to_double(C0, er + ec[j] - 54);
                        a.y -= scaled_to_double(C1, er + ec[j + 1] - 54);
                        *reinterpret_cast<double2 *>(dst + j) = a;
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

}  // namespace ctc

bool chol_tc_enabled(const gp_model *m) { return m->cslices != nullptr; }

size_t chol_tc_slice_bytes(int n_pad) { return (size_t)ctc::SLICES * n_pad * ctc::BK * 2; }

int chol_tc_maps(const gp_model *m, void *map_a, void *map_b)
{
    const uint64_t rows = (uint64_t)ctc::SLICES * m->n_pad;
    GPBO_TRY(encode_2d_box((CUtensorMap *)map_a, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, m->cslices, rows, ctc::BK, ctc::BM,
                           ctc::BK, CU_TENSOR_MAP_SWIZZLE_128B));
    GPBO_TRY(encode_2d_box((CUtensorMap *)map_b, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, m->cslices, rows, ctc::BK, ctc::PBN,
                           ctc::BK, CU_TENSOR_MAP_SWIZZLE_128B));
    return GPBO_OK;
}

// Split panel kb (rows of block rows min(c0, kb + 2) ..), then update block columns c0 .. of the
// rows of block rows kb + 2 .. on stream st with the persistent kernel.
int chol_tc_update(gpbo_ctx *ctx, gp_model *m, int kb, int c0, cudaStream_t st, const void *map_a, const void *map_b)
{
    const int n_pad = m->n_pad, nblk = n_pad / NB, b0 = kb + 2;
    if (b0 >= nblk) return GPBO_OK;
    GPBO_TRY(ensure_smem((const void *)ctc::k_chol_update_tcp, ctx->device, (int)ctc::PSMEM_BYTES));
    const int r0 = (c0 < b0 ? c0 : b0) * NB, rows = n_pad - r0;
    ctc::k_chol_split<<<(unsigned)cdiv64((int64_t)rows * 32, 256), 256, 0, st>>>(
        m->L, n_pad, kb, r0, (__nv_bfloat16 *)m->cslices, m->cexps);
    GPBO_LAUNCH_CHECK(ctx);
    ctc::PParams P;
    P.A = m->L;
    P.exps = m->cexps;
    P.status = ctx->dev_status;
    P.n_pad = n_pad;
    P.nblk = nblk;
    P.kb = kb;
    P.b0 = b0;
    P.c0 = c0;
    P.items = ctc::p_items(b0, c0, nblk);
    const int sms = ctx->sm_count > 2 * ctc::CHAIN_SMS ? ctx->sm_count - ctc::CHAIN_SMS : ctx->sm_count;
    const int grid = P.items < sms ? P.items : sms;
    ctc::k_chol_update_tcp<<<(unsigned)grid, ctc::PTHREADS, ctc::PSMEM_BYTES, st>>>(
        *(const CUtensorMap *)map_a, *(const CUtensorMap *)map_b, P);
    GPBO_LAUNCH_CHECK(ctx);
    return GPBO_OK;
}

int chol_tc_arena_maps(const void *slices, int64_t rows, void *map_a, void *map_b)
{
    GPBO_TRY(encode_2d_box((CUtensorMap *)map_a, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, slices, (uint64_t)rows, ctc::BK,
                           ctc::BM, ctc::BK, CU_TENSOR_MAP_SWIZZLE_128B));
    GPBO_TRY(encode_2d_box((CUtensorMap *)map_b, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, slices, (uint64_t)rows, ctc::BK,
                           ctc::BN, ctc::BK, CU_TENSOR_MAP_SWIZZLE_128B));
    return GPBO_OK;
}

// Step kb of every problem that takes a tensor-core update there: split its panel kb, then
// update its block columns kb + 2 .. (one launch each, blockIdx.y = problem).
int chol_tc_update_batched(gpbo_ctx *ctx, cudaStream_t st, const CholTcProb *probs, int G, int kb, int max_rows,
                           int64_t max_tiles, void *slices, const void *map_a, const void *map_b)
{
    if (max_rows <= 0 || max_tiles <= 0) return GPBO_OK;
    GPBO_TRY(ensure_smem((const void *)ctc::k_chol_update_tc, ctx->device, (int)ctc::SMEM_BYTES));
    ctc::k_chol_split_batched<<<dim3((unsigned)cdiv64((int64_t)max_rows * 32, 256), G), 256, 0, st>>>(
        probs, kb, (__nv_bfloat16 *)slices);
    GPBO_LAUNCH_CHECK(ctx);
    ctc::Params P = {};
    P.probs = probs;
    P.status = ctx->dev_status;
    P.kb = kb;
    P.idesc = tcx::idesc_f16(1u, ctc::BN, ctc::BM);
    ctc::k_chol_update_tc<<<dim3((unsigned)max_tiles, G), ctc::THREADS, ctc::SMEM_BYTES, st>>>(
        *(const CUtensorMap *)map_a, *(const CUtensorMap *)map_b, P);
    GPBO_LAUNCH_CHECK(ctx);
    return GPBO_OK;
}

}  // namespace gpbo
