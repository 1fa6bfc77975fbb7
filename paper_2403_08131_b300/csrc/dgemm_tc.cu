// Batched GEMMs at FP64 accuracy on the tensor cores, for the large levels of the FP64
// triangular inverse (L^-1 by recursive doubling: T = L21 X11, then X21 = -X22 T).
//
// C_q = alpha A_q B_q for each problem q of a level, A_q (m x k) and B_q (k x n) FP64 with
// leading dimension ld.  The slice products of the tensor-core Cholesky update and of K^-1
// (Ozaki, Ogita, Oishi and Rump 2012): each row of A_q and each column of B_q is 2^(e - 7) times
// 7 integer slices of at most 8 bits (exact in BF16), e per row / per column over its k values;
// the 34 slice pairs with s + t <= 9 accumulate per level s + t in FP32 (exact integers while a
// fold covers at most 128 of k), fold into two int64 sums per element, and the result is built
// as a double on the integer pipe.  Triangular operands skip their zero parts: with B lower
// triangular (B_kj = 0 for k < j) a tile's k starts at its first column; with A lower
// triangular (A_ik = 0 for k > i) it ends after its last row.
//
//   k_dtc_split_rows  one warp per row of A_q: exponent, then the slices (zero past k)
//   k_dtc_exp_cols    per column of B_q: exponent
//   k_dtc_split_cols  B_q's columns as slice rows, through a 32 x 32 shared-memory transpose
//   k_dtc_gemm        one CTA per 128 x 64 tile of C_q, k in chunks of 64, fold every two chunks
// Every mbarrier wait is bounded; a timeout raises DEV_TIMEOUT and the CTA waits (bounded) for
// its copies and MMAs and frees TMEM.
#include "tc_common.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

namespace gpbo {

namespace dtc {

constexpr int SLICES = 7;
constexpr int LEVEL_MAX = 9;
constexpr int BM = 128, BN = 64, BK = 64;
constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
constexpr int THREADS = 256;
constexpr int TMEM_COLS = 512;
constexpr size_t SMEM_BYTES = (size_t)SLICES * (A_BYTES + B_BYTES) + 1024 + 1024;
constexpr int TRI_B_LOWER = 1, TRI_A_LOWER = 2;

using namespace tcx;

struct Prob {
    int64_t a_off, b_off, c_off;  // element offsets of A_q, B_q, C_q (leading dimension ld)
    int a_row0, b_row0;           // first slice row of A_q / of B_q's columns
    int m, n, k;
};

// One warp per row r of A_q (blockIdx.y = q): e_r over the row's k values, then the slices
// for k' < KA (zero from k on).
__global__ void __launch_bounds__(256) k_dtc_split_rows(const double *__restrict__ A, int ld, const Prob *__restrict__ P,
                                                        int KA, int RA, __nv_bfloat16 *__restrict__ S, int *__restrict__ ex)
{
    const Prob p = P[blockIdx.y];
    const int r = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (r >= p.m) return;
    const double *row = A + p.a_off + (int64_t)r * ld;
    double mx = 0.0;
    for (int j = lane; j < p.k; j += 32) mx = fmax(mx, fabs(row[j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int e = mx > 0.0 ? ilogb(mx) + 1 : 0;
    if (lane == 0) ex[p.a_row0 + r] = e;
    for (int j = lane; j < KA; j += 32) {
        double v = j < p.k ? scalbn(row[j], 7 - e) : 0.0;
        for (int s = 0; s < SLICES; ++s) {
            const double a = rint(v);
            S[((int64_t)s * RA + p.a_row0 + r) * KA + j] = __double2bfloat16(a);
            v = (v - a) * 256.0;
        }
    }
}

// e_j over column j's k values of B_q: CTA (bx, q) handles columns 32 bx .., 8 row groups.
__global__ void __launch_bounds__(256) k_dtc_exp_cols(const double *__restrict__ B, int ld, const Prob *__restrict__ P,
                                                      int *__restrict__ ex)
{
    __shared__ double mx[8][32];
    const Prob p = P[blockIdx.y];
    const int j = blockIdx.x * 32 + (threadIdx.x & 31), rg = threadIdx.x >> 5;
    double m = 0.0;
    if (j < p.n)
        for (int kk = rg; kk < p.k; kk += 8) m = fmax(m, fabs(B[p.b_off + (int64_t)kk * ld + j]));
    mx[rg][threadIdx.x & 31] = m;
    __syncthreads();
    if (threadIdx.x < 32 && j < p.n) {
        for (int g = 1; g < 8; ++g) m = fmax(m, mx[g][threadIdx.x]);
        ex[p.b_row0 + j] = m > 0.0 ? ilogb(m) + 1 : 0;
    }
}

// Slices of B_q's columns: CTA (bx, by, q) covers columns 32 bx .. and k values 32 by ..
// (k' < KA; zero from k on).
__global__ void __launch_bounds__(256) k_dtc_split_cols(const double *__restrict__ B, int ld, const Prob *__restrict__ P,
                                                        int KA, int RB, const int *__restrict__ ex,
                                                        __nv_bfloat16 *__restrict__ S)
{
    __shared__ double t[32][33];
    const Prob p = P[blockIdx.z];
    const int j0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    if (j0 >= p.n) return;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < 32; r += 8) {
        const int kk = k0 + r, j = j0 + tx;
        t[r][tx] = (kk < p.k && j < p.n) ? B[p.b_off + (int64_t)kk * ld + j] : 0.0;  // t[k][j]
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int j = j0 + r;
        if (j >= p.n) continue;
        double v = scalbn(t[tx][r], 7 - ex[p.b_row0 + j]);
        for (int s = 0; s < SLICES; ++s) {
            const double a = rint(v);
            S[((int64_t)s * RB + p.b_row0 + j) * KA + k0 + tx] = __double2bfloat16(a);
            v = (v - a) * 256.0;
        }
    }
}

struct Shared {
    uint64_t full;  // one phase per chunk
    uint64_t done;  // one phase per chunk (thread 0)
    uint64_t fold;  // one phase per fold (every warp)
    uint32_t tmem_base;
    int abort;
    int er[BM];
    int ec[BN];
};

struct Params {
    double *C;
    const Prob *probs;
    const int *exa, *exb;
    unsigned *status;
    int ld, RA, RB, tri;
    double alpha;
    uint32_t idesc;
};

__global__ void __launch_bounds__(THREADS, 1)
    k_dtc_gemm(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b, Params P)
{
    const Prob pr = P.probs[blockIdx.z];
    const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
    if (row0 >= pr.m || col0 >= pr.n) return;  // whole CTA, before any barrier
    int kbeg = (P.tri & TRI_B_LOWER) ? col0 : 0;
    int kend = (P.tri & TRI_A_LOWER) ? min(pr.k, row0 + BM) : pr.k;
    kend = (kend + BK - 1) / BK * BK;
    const int nchunk = kend > kbeg ? (kend - kbeg) / BK : 0;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int quad = warp & 3, half = warp >> 2;
    const int row = quad * 32 + lane;
    if (nchunk == 0) {  // the tile is all zero
        const int r = row0 + row;
        if (r < pr.m)
            for (int j = 0; j < 32; ++j)
                if (col0 + half * 32 + j < pr.n) P.C[pr.c_off + (int64_t)r * P.ld + col0 + half * 32 + j] = 0.0;
        return;
    }
    extern __shared__ unsigned char smraw[];
    unsigned char *tiles = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char *sa = tiles, *sb = tiles + (size_t)SLICES * A_BYTES;
    Shared *sh = (Shared *)(sb + (size_t)SLICES * B_BYTES);
    if (threadIdx.x == 0) {
        mbar_init(&sh->full, 1);
        mbar_init(&sh->done, 1);
        mbar_init(&sh->fold, 1);
        sh->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    for (int i = threadIdx.x; i < BM; i += THREADS) sh->er[i] = P.exa[pr.a_row0 + row0 + i];
    for (int i = threadIdx.x; i < BN; i += THREADS) sh->ec[i] = P.exb[pr.b_row0 + col0 + i];
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
    const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16);
    long long hi[32], lo[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) hi[j] = lo[j] = 0;

    auto load = [&](int c) {
        mbar_arrive_expect_tx(&sh->full, SLICES * (A_BYTES + B_BYTES));
        const int k = kbeg + c * BK;
        for (int s = 0; s < SLICES; ++s) {
            tma_load_2d(sa + (size_t)s * A_BYTES, &map_a, k, s * P.RA + pr.a_row0 + row0, &sh->full);
            tma_load_2d(sb + (size_t)s * B_BYTES, &map_b, k, s * P.RB + pr.b_row0 + col0, &sh->full);
        }
    };
    bool ok = true;
    int armed = 0;
    if (threadIdx.x == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&map_a) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&map_b) : "memory");
        load(0);
        armed = 1;
    }
    for (int c = 0; c < nchunk; ++c) {
        const bool fold_here = (c & 1) == 1 || c + 1 == nchunk;
        if (threadIdx.x == 0 && ok) {
            if (!mbar_wait(&sh->full, (uint32_t)c & 1u, abort_flag, P.status)) {
                ok = false;
            } else {
                tc_fence_after();
                for (int l = 2; l <= LEVEL_MAX; ++l) {
                    const uint32_t d = tmem + (uint32_t)((l - 2) * BN);
                    bool first = (c & 1) == 0;
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
                if (fold_here) mma_commit(&sh->fold);
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
        if (fold_here) {
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
            __syncthreads();
            tc_fence_after();
            if (*abort_flag) {
                ok = false;
                break;
            }
        }
    }
    if (ok) {
        const int r = row0 + row;
        if (r < pr.m) {
            const int er = sh->er[row];
            double *dst = P.C + pr.c_off + (int64_t)r * P.ld + col0 + half * 32;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (col0 + half * 32 + j >= pr.n) break;
                const int E = er + sh->ec[half * 32 + j];
                dst[j] = P.alpha * (scaled_to_double(hi[j], E - 38) + scaled_to_double(lo[j], E - 70));
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        if (armed > 0) mbar_wait(&sh->full, (uint32_t)(armed - 1) & 1u, abort_flag, P.status, false);
        mbar_wait(&sh->done, (uint32_t)(nchunk - 1) & 1u, abort_flag, P.status, false);
    }
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

}  // namespace dtc

// Scratch for one level of up to `cnt` problems of m, k <= mk and n <= nmax.
size_t dtc_scratch_bytes(int cnt, int mk, int nmax)
{
    const int KA = (mk + 63) / 64 * 64, RAq = (mk + 127) / 128 * 128;
    const size_t sa = (size_t)dtc::SLICES * cnt * RAq * KA * 2, sb = (size_t)dtc::SLICES * cnt * nmax * KA * 2;
    return round_up64((int64_t)sa, 256) + round_up64((int64_t)sb, 256) + sizeof(int) * (size_t)cnt * (RAq + nmax) +
           sizeof(dtc::Prob) * (size_t)cnt + 1024;
}

// C_q = alpha A_q B_q for the problems of one level (host list; offsets with leading dimension
// ld; all n_q equal to a multiple of 64).  tri: 1 = B lower triangular, 2 = A lower triangular.
int dgemm_tc_level(gpbo_ctx *ctx, cudaStream_t st, const double *A, const double *B, double *C, int ld,
                   const GemmProb *probs, int cnt, double alpha, int tri, void *scratch)
{
    if (cnt < 1) return GPBO_OK;
    int mk = 0, nmax = 0;
    for (int q = 0; q < cnt; ++q) {
        mk = std::max(mk, std::max(probs[q].m, probs[q].k));
        nmax = std::max(nmax, probs[q].n);
        if (probs[q].n % 64 != 0) return GPBO_EINVAL;
    }
    const int KA = (mk + 63) / 64 * 64, RAq = (mk + 127) / 128 * 128;
    const int RA = cnt * RAq, RB = cnt * nmax;
    unsigned char *w = (unsigned char *)scratch;
    const size_t sa_bytes = (size_t)dtc::SLICES * RA * KA * 2, sb_bytes = (size_t)dtc::SLICES * RB * KA * 2;
    __nv_bfloat16 *Sa = (__nv_bfloat16 *)w;
    __nv_bfloat16 *Sb = (__nv_bfloat16 *)(w + round_up64((int64_t)sa_bytes, 256));
    int *exa = (int *)((unsigned char *)Sb + round_up64((int64_t)sb_bytes, 256));
    int *exb = exa + RA;
    dtc::Prob *dp = (dtc::Prob *)(((uintptr_t)(exb + RB) + 255) & ~(uintptr_t)255);
    std::vector<dtc::Prob> hp(cnt);
    for (int q = 0; q < cnt; ++q) {
        hp[q].a_off = probs[q].a_off;
        hp[q].b_off = probs[q].b_off;
        hp[q].c_off = probs[q].c_off;
        hp[q].a_row0 = q * RAq;
        hp[q].b_row0 = q * nmax;
        hp[q].m = probs[q].m;
        hp[q].n = probs[q].n;
        hp[q].k = probs[q].k;
    }
    // from pageable memory the copy is staged before the call returns, so hp may go at return
    GPBO_CUDA_TRY(cudaMemcpyAsync(dp, hp.data(), sizeof(dtc::Prob) * cnt, cudaMemcpyHostToDevice, st));
    static bool attr = false;
    if (!attr) {
        GPBO_CUDA_TRY(cudaFuncSetAttribute(dtc::k_dtc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)dtc::SMEM_BYTES));
        attr = true;
    }
    dtc::k_dtc_split_rows<<<dim3((mk + 7) / 8, cnt), 256, 0, st>>>(A, ld, dp, KA, RA, Sa, exa);
    GPBO_LAUNCH_CHECK(ctx);
    dtc::k_dtc_exp_cols<<<dim3(nmax / 32, cnt), 256, 0, st>>>(B, ld, dp, exb);
    GPBO_LAUNCH_CHECK(ctx);
    dtc::k_dtc_split_cols<<<dim3(nmax / 32, KA / 32, cnt), 256, 0, st>>>(B, ld, dp, KA, RB, exb, Sb);
    GPBO_LAUNCH_CHECK(ctx);
    CUtensorMap ma, mb;
    GPBO_TRY(encode_2d_box(&ma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, Sa, (uint64_t)dtc::SLICES * RA, (uint64_t)KA, dtc::BM,
                           dtc::BK, CU_TENSOR_MAP_SWIZZLE_128B));
    GPBO_TRY(encode_2d_box(&mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, Sb, (uint64_t)dtc::SLICES * RB, (uint64_t)KA, dtc::BN,
                           dtc::BK, CU_TENSOR_MAP_SWIZZLE_128B));
    dtc::Params P;
    P.C = C;
    P.probs = dp;
    P.exa = exa;
    P.exb = exb;
    P.status = ctx->dev_status;
    P.ld = ld;
    P.RA = RA;
    P.RB = RB;
    P.tri = tri;
    P.alpha = alpha;
    P.idesc = tcx::idesc_f16(1u, dtc::BN, dtc::BM);
    dtc::k_dtc_gemm<<<dim3(nmax / dtc::BN, RAq / dtc::BM, cnt), dtc::THREADS, dtc::SMEM_BYTES, st>>>(ma, mb, P);
    GPBO_LAUNCH_CHECK(ctx);
    return GPBO_OK;
}

}  // namespace gpbo
