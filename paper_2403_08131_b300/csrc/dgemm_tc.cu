// Batched GEMMs on the tensor cores at FP64 or FP32 accuracy, for the large levels of the
// triangular inverse (L^-1 by recursive doubling: T = L21 X11, then X21 = -X22 T).
//
// C_q = alpha A_q B_q for each problem q of a level, A_q (m x k) and B_q (k x n) FP64 or FP32 with
// leading dimension ld.  The slice products of the tensor-core Cholesky update and of K^-1
// (Ozaki, Ogita, Oishi and Rump 2012): each row of A_q and each column of B_q is 2^(e - 7) times
// S integer slices of at most 8 bits (exact in BF16), e per row / per column over its k values,
// taken on the integer pipe from the bits of the values.  The slice pairs (1-based) with
// s + t <= LMAX accumulate per level s + t in FP32 (exact integers while a fold covers few enough
// of k), fold into int64 sums per element, and the result is built as a double on the integer
// pipe.  FP64 accuracy: S = 7, the 34 pairs with s + t <= 9 (left-out terms below 2^-56 of
// |A_r| |B_c| per product).  FP32 accuracy: S = 3, the 6 pairs with s + t <= 4 (below 2^-24).
// Triangular operands skip their zero parts: with B lower triangular (B_kj = 0 for k < j) a
// tile's k starts at its first column; with A lower triangular (A_ik = 0 for k > i) it ends
// after its last row.
//
//   k_dtc_split_rows  one warp per row of A_q: exponent, then the slices (zero past k)
//   k_dtc_max_cols    per column of B_q: largest magnitude (atomic max over k chunks)
//   k_dtc_split_cols  B_q's columns as slice rows, through a 32 x 32 shared-memory transpose
//   k_dtc_gemm        one CTA per 128 x 64 tile of C_q, k in chunks of 64, folds every FOLD chunks
// Every mbarrier wait is bounded; a timeout raises DEV_TIMEOUT and the CTA waits (bounded) for
// its copies and MMAs and frees TMEM.
#include "tc_common.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

namespace gpbo {

namespace dtc {

constexpr int BM = 128, BN = 64, BK = 64;
constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
constexpr int THREADS = 256;
constexpr int TRI_B_LOWER = 1, TRI_A_LOWER = 2;

// Per slice count: the last level kept, chunks per fold (every level's FP32 sum stays below 2^24:
// at most 7 pairs x 128 of k, or 3 pairs x 256 of k, times 2^14), TMEM columns, CTAs per SM.
template <int S> struct Cfg;
template <> struct Cfg<7> {
    static constexpr int LMAX = 9, FOLD = 2, TMEM_COLS = 512, MIN_CTAS = 1;
    static constexpr size_t SMEM_BYTES = (size_t)7 * (A_BYTES + B_BYTES) + 2048;
};
template <> struct Cfg<3> {
    static constexpr int LMAX = 4, FOLD = 4, TMEM_COLS = 256, MIN_CTAS = 2;
    // 72 KiB of tiles, padded so that at most two CTAs (the TMEM of an SM) share an SM
    static constexpr size_t SMEM_BYTES = (size_t)100 * 1024;
};
template <int S> __host__ __device__ constexpr int levels_hi() { return Cfg<S>::LMAX < 5 ? Cfg<S>::LMAX : 5; }

using namespace tcx;

struct Prob {
    int64_t a_off, b_off, c_off;  // element offsets of A_q, B_q, C_q (leading dimension ld)
    int a_row0, b_row0;           // first slice row of A_q / of B_q's columns
    int m, n, k;
};

// One warp per row r of A_q (blockIdx.y = q): e_r over the row's k values, then the slices
// for k' < KA (zero from k on).
template <typename T, int S>
__global__ void __launch_bounds__(256) k_dtc_split_rows(const T *__restrict__ A, int ld, const Prob *__restrict__ P,
                                                        int KA, int RA, uint16_t *__restrict__ Sl, int *__restrict__ ex)
{
    const Prob p = P[blockIdx.y];
    const int r = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (r >= p.m) return;
    const T *row = A + p.a_off + (int64_t)r * ld;
    unsigned long long mx = 0;
    for (int j = lane; j < p.k; j += 32) mx = max(mx, (unsigned long long)mag_bits(row[j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int e = exp_of_mag_t<T>(mx);
    if (lane == 0) ex[p.a_row0 + r] = e;
    for (int j = lane; j < KA; j += 32) {
        uint16_t d[S];
        split_digits<S>(j < p.k ? fixed_of(row[j], e, 8 * S - 1) : 0, d);
#pragma unroll
        for (int s = 0; s < S; ++s) Sl[((int64_t)s * RA + p.a_row0 + r) * KA + j] = d[s];
    }
}

// Largest |B_kj| per column j as magnitude bits: CTA (bx, by, q) covers columns 32 bx .. and
// k values 256 by .. (8 row groups), and combines into mx[j] (zeroed before) by an atomic max.
template <typename T>
__global__ void __launch_bounds__(256) k_dtc_max_cols(const T *__restrict__ B, int ld, const Prob *__restrict__ P,
                                                      unsigned long long *__restrict__ mxg)
{
    __shared__ unsigned long long mx[8][32];
    const Prob p = P[blockIdx.z];
    const int j = blockIdx.x * 32 + (threadIdx.x & 31), rg = threadIdx.x >> 5;
    const int k0 = blockIdx.y * 256, k1 = min(p.k, k0 + 256);
    unsigned long long m = 0;
    if (j < p.n)
        for (int kk = k0 + rg; kk < k1; kk += 8) m = max(m, (unsigned long long)mag_bits(B[p.b_off + (int64_t)kk * ld + j]));
    mx[rg][threadIdx.x & 31] = m;
    __syncthreads();
    if (threadIdx.x < 32 && j < p.n) {
        for (int g = 1; g < 8; ++g) m = max(m, mx[g][threadIdx.x]);
        if (m) atomicMax(mxg + p.b_row0 + j, m);
    }
}

// Slices of B_q's columns: CTA (bx, by, q) covers columns 32 bx .. and k values 32 by ..
// (k' < KA; zero from k on); e_j from the column maxima, written out by the CTAs with by = 0.
template <typename T, int S>
__global__ void __launch_bounds__(256) k_dtc_split_cols(const T *__restrict__ B, int ld, const Prob *__restrict__ P,
                                                        int KA, int RB, const unsigned long long *__restrict__ mxg,
                                                        int *__restrict__ ex, uint16_t *__restrict__ Sl)
{
    __shared__ T t[32][33];
    __shared__ int ec[32];
    const Prob p = P[blockIdx.z];
    const int j0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    if (j0 >= p.n) return;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    if (threadIdx.x < 32) {
        ec[tx] = j0 + tx < p.n ? exp_of_mag_t<T>(mxg[p.b_row0 + j0 + tx]) : 0;
        if (blockIdx.y == 0 && j0 + tx < p.n) ex[p.b_row0 + j0 + tx] = ec[tx];
    }
    for (int r = ty; r < 32; r += 8) {
        const int kk = k0 + r, j = j0 + tx;
        t[r][tx] = (kk < p.k && j < p.n) ? B[p.b_off + (int64_t)kk * ld + j] : T(0);  // t[k][j]
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int j = j0 + r;
        if (j >= p.n) continue;
        uint16_t d[S];
        split_digits<S>(fixed_of(t[tx][r], ec[r], 8 * S - 1), d);
#pragma unroll
        for (int s = 0; s < S; ++s) Sl[((int64_t)s * RB + p.b_row0 + j) * KA + k0 + tx] = d[s];
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

template <typename T> struct Params {
    T *C;
    const Prob *probs;
    const int *exa, *exb;
    unsigned *status;
    int ld, RA, RB, tri;
    double alpha;
    uint32_t idesc;
};

template <typename T, int S>
__global__ void __launch_bounds__(THREADS, Cfg<S>::MIN_CTAS)
    k_dtc_gemm(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b, Params<T> P)
{
    constexpr int LMAX = Cfg<S>::LMAX, FOLD = Cfg<S>::FOLD, TMEM_COLS = Cfg<S>::TMEM_COLS;
    constexpr int HL = levels_hi<S>();  // levels 2 .. HL fold into hi, HL + 1 .. LMAX into lo
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
                if (col0 + half * 32 + j < pr.n) P.C[pr.c_off + (int64_t)r * P.ld + col0 + half * 32 + j] = T(0);
        return;
    }
    extern __shared__ unsigned char smraw[];
    unsigned char *tiles = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char *sa = tiles, *sb = tiles + (size_t)S * A_BYTES;
    Shared *sh = (Shared *)(sb + (size_t)S * B_BYTES);
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
    long long hi[32], lo[HL < LMAX ? 32 : 1];
#pragma unroll
    for (int j = 0; j < 32; ++j) hi[j] = 0;
#pragma unroll
    for (int j = 0; j < (HL < LMAX ? 32 : 1); ++j) lo[j] = 0;

    auto load = [&](int c) {
        mbar_arrive_expect_tx(&sh->full, S * (A_BYTES + B_BYTES));
        const int k = kbeg + c * BK;
        for (int s = 0; s < S; ++s) {
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
        const bool fold_here = c % FOLD == FOLD - 1 || c + 1 == nchunk;
        if (threadIdx.x == 0 && ok) {
            if (!mbar_wait(&sh->full, (uint32_t)c & 1u, abort_flag, P.status)) {
                ok = false;
            } else {
                tc_fence_after();
                for (int l = 2; l <= LMAX; ++l) {
                    const uint32_t d = tmem + (uint32_t)((l - 2) * BN);
                    bool first = c % FOLD == 0;
                    for (int s = 1; s <= S; ++s) {
                        const int t = l - s;
                        if (t < 1 || t > S) continue;
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
            const bool got = mbar_wait_inl(&sh->fold, (uint32_t)(c / FOLD) & 1u, abort_flag, P.status);
            if (!__all_sync(0xffffffffu, got)) {
                ok = false;
                break;
            }
            tc_fence_after();
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                const int c0 = half * 32 + g * 16;
                long long h16[16];
                uint32_t v[16];
                tmem_ld16_nw(taddr + (uint32_t)c0, v);
                tmem_wait();
                pin16(v);
#pragma unroll
                for (int j = 0; j < 16; ++j) h16[j] = __float2int_rn(__uint_as_float(v[j]));
#pragma unroll 1
                for (int l = 3; l <= HL; ++l) {
                    tmem_ld16_nw(taddr + (uint32_t)((l - 2) * BN + c0), v);
                    tmem_wait();
                    pin16(v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) h16[j] = h16[j] * 256 + __float2int_rn(__uint_as_float(v[j]));
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) hi[g * 16 + j] += h16[j];
                if constexpr (HL < LMAX) {
                    long long l16[16];
                    tmem_ld16_nw(taddr + (uint32_t)((HL - 1) * BN + c0), v);
                    tmem_wait();
                    pin16(v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) l16[j] = __float2int_rn(__uint_as_float(v[j]));
#pragma unroll 1
                    for (int l = HL + 2; l <= LMAX; ++l) {
                        tmem_ld16_nw(taddr + (uint32_t)((l - 2) * BN + c0), v);
                        tmem_wait();
                        pin16(v);
#pragma unroll
                        for (int j = 0; j < 16; ++j) l16[j] = l16[j] * 256 + __float2int_rn(__uint_as_float(v[j]));
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j) lo[g * 16 + j] += l16[j];
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
            T *dst = P.C + pr.c_off + (int64_t)r * P.ld + col0 + half * 32;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (col0 + half * 32 + j >= pr.n) break;
                const int E = er + sh->ec[half * 32 + j];
                // level l weighs 2^(E - 14 - 8 (l - 2)): hi ends at level HL, lo at LMAX
                double v = scaled_to_double(hi[j], E - 14 - 8 * (HL - 2));
                if constexpr (HL < LMAX) v += scaled_to_double(lo[j], E - 14 - 8 * (LMAX - 2));
                dst[j] = (T)(P.alpha * v);
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

template <typename T, int S> static size_t scratch_bytes(int cnt, int mk, int nmax)
{
    const int KA = (mk + 63) / 64 * 64, RAq = (mk + 127) / 128 * 128;
    const size_t sa = (size_t)S * cnt * RAq * KA * 2, sb = (size_t)S * cnt * nmax * KA * 2;
    return round_up64((int64_t)sa, 256) + round_up64((int64_t)sb, 256) + sizeof(int) * (size_t)cnt * (RAq + nmax) +
           sizeof(unsigned long long) * (size_t)cnt * nmax + sizeof(dtc::Prob) * (size_t)cnt + 1024;
}

// C_q = alpha A_q B_q for the problems of one level (host list; offsets with leading dimension
// ld; all n_q equal to a multiple of 64).  tri: 1 = B lower triangular, 2 = A lower triangular.
template <typename T, int S>
static int gemm_level(gpbo_ctx *ctx, cudaStream_t st, const T *A, const T *B, T *C, int ld, const GemmProb *probs,
                      int cnt, double alpha, int tri, void *scratch)
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
    const size_t sa_bytes = (size_t)S * RA * KA * 2, sb_bytes = (size_t)S * RB * KA * 2;
    uint16_t *Sa = (uint16_t *)w;
    uint16_t *Sb = (uint16_t *)(w + round_up64((int64_t)sa_bytes, 256));
    int *exa = (int *)((unsigned char *)Sb + round_up64((int64_t)sb_bytes, 256));
    int *exb = exa + RA;
    unsigned long long *mxb = (unsigned long long *)(((uintptr_t)(exb + RB) + 255) & ~(uintptr_t)255);
    dtc::Prob *dp = (dtc::Prob *)(((uintptr_t)(mxb + RB) + 255) & ~(uintptr_t)255);
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
    GPBO_TRY(ensure_smem((const void *)dtc::k_dtc_gemm<T, S>, ctx->device, (int)dtc::Cfg<S>::SMEM_BYTES));
    dtc::k_dtc_split_rows<T, S><<<dim3((mk + 7) / 8, cnt), 256, 0, st>>>(A, ld, dp, KA, RA, Sa, exa);
    GPBO_LAUNCH_CHECK(ctx);
    GPBO_CUDA_TRY(cudaMemsetAsync(mxb, 0, sizeof(unsigned long long) * RB, st));
    dtc::k_dtc_max_cols<T><<<dim3(nmax / 32, (mk + 255) / 256, cnt), 256, 0, st>>>(B, ld, dp, mxb);
    GPBO_LAUNCH_CHECK(ctx);
    dtc::k_dtc_split_cols<T, S><<<dim3(nmax / 32, KA / 32, cnt), 256, 0, st>>>(B, ld, dp, KA, RB, mxb, exb, Sb);
    GPBO_LAUNCH_CHECK(ctx);
    CUtensorMap ma, mb;
    GPBO_TRY(encode_2d_box(&ma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, Sa, (uint64_t)S * RA, (uint64_t)KA, dtc::BM, dtc::BK,
                           CU_TENSOR_MAP_SWIZZLE_128B));
    GPBO_TRY(encode_2d_box(&mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, Sb, (uint64_t)S * RB, (uint64_t)KA, dtc::BN, dtc::BK,
                           CU_TENSOR_MAP_SWIZZLE_128B));
    dtc::Params<T> P;
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
    dtc::k_dtc_gemm<T, S><<<dim3(nmax / dtc::BN, RAq / dtc::BM, cnt), dtc::THREADS, dtc::Cfg<S>::SMEM_BYTES, st>>>(ma, mb,
                                                                                                                 P);
    GPBO_LAUNCH_CHECK(ctx);
    return GPBO_OK;
}

// FP64 accuracy (7 slices) on FP64 operands
size_t dtc_scratch_bytes(int cnt, int mk, int nmax) { return scratch_bytes<double, 7>(cnt, mk, nmax); }
int dgemm_tc_level(gpbo_ctx *ctx, cudaStream_t st, const double *A, const double *B, double *C, int ld,
                   const GemmProb *probs, int cnt, double alpha, int tri, void *scratch)
{
    return gemm_level<double, 7>(ctx, st, A, B, C, ld, probs, cnt, alpha, tri, scratch);
}
// FP32 accuracy (3 slices) on FP32 operands
size_t stc_scratch_bytes(int cnt, int mk, int nmax) { return scratch_bytes<float, 3>(cnt, mk, nmax); }
int sgemm_tc_level(gpbo_ctx *ctx, cudaStream_t st, const float *A, const float *B, float *C, int ld,
                   const GemmProb *probs, int cnt, double alpha, int tri, void *scratch)
{
    return gemm_level<float, 3>(ctx, st, A, B, C, ld, probs, cnt, alpha, tri, scratch);
}

}  // namespace gpbo
