// Cross-kernel and posterior mean on the tensor cores (16-bit scoring models, d <= 32).
//
//   K*_ci = s2 m(r_ci),  r_ci^2 = |z_c|^2 + |z_i|^2 - 2 z_c . z_i,  z = (x - 1/2) / l
//   mu_c  = sum_i K*_ci alpha_i   (FP32, before K* is rounded)
//
// The cross term z_c . z_i is a dense (candidates x d) by (d x observations) contraction.
// Each coordinate is split into FP16 hi = fp16(z) and lo = fp16(z - hi); with
// A' = -2 [hi | hi | lo | 1 1 0 ..] and B' = [hi | lo | hi | s_hi s_lo 0 ..] (32 columns each,
// K = 128), where s = |z_i|^2 split the same way and the -2 is exact, one kind::f16 MMA
// chain accumulates |z_i|^2 - 2 (hi.hi + hi.lo + lo.hi) in FP32 -- about 22 significant bits,
// the accuracy of an FP32 dot product -- so the epilogue only adds |z_c|^2.  Centring the
// coordinates at 1/2 keeps |z|^2 small, so r^2 = |z_c|^2 + |z_i|^2 - 2 z_c . z_i cancels little.
// The Matern evaluation, the mean and the 16-bit rounding of K* run in the epilogue, where
// each thread owns one candidate (one TMEM lane) and a quarter of a 256-observation chunk.
//
// Roles (one CTA per SM, persistent over 128-candidate tiles, 576 threads):
//   warp 0     TMA: B' chunk (256 observations x 128) per stage, 2 stages of 64 KiB
//   warp 1     TMEM (512 columns); one lane issues 8 MMAs (M=128, N=256, K=16) per chunk
//              into one of two 256-column accumulators
//   warps 2-17 epilogue: warp w reads TMEM lane quadrant w % 4 and column group (w-2) / 4
//              (64 of each chunk's 256 columns);
//              warps 2-5 also build A' for the next tile (two smem slots) and its |z_c|^2;
//              a slot is rebuilt only after its MMAs completed and all 8 warps read its |z_c|^2
// Every wait is bounded; on timeout the kernel raises DEV_TIMEOUT, drains and exits.
#include "tc_common.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

namespace gpbo {
namespace xtc {

using namespace tcx;

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int KB = 128;                    // split width: [hi|hi|lo|0] x 32 for A', [hi|lo|hi|0] for B'
constexpr int DMAX = 32;
constexpr int STAGES = 1;                  // B' copies are short next to a chunk's epilogue
constexpr int EPI_WARPS = 16;             // 4 lane quadrants x 4 column groups of 64
constexpr int GROUPS = EPI_WARPS / 4;
constexpr int THREADS = (2 + EPI_WARPS) * 32;
constexpr int TMEM_COLS = 512;
constexpr int A_TILE = BM * 128;           // bytes of one 64-column K tile of A'
constexpr int A_SLOT = 2 * A_TILE;         // A' = 2 K tiles
constexpr int B_TILE = BN * 128;
constexpr int B_STAGE = 2 * B_TILE;

struct alignas(16) Shared {
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint64_t a_full[2];
    uint64_t a_empty[2];
    uint64_t mu_ready[2];
    uint64_t mu_free[2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
    float na[2][BM];                 // |z_c|^2 per A' slot
    float mu_part[2][GROUPS - 1][BM]; // column groups 1..3: partial means per slot
};

// K* leaves through per-warp staging tiles of 32 rows x 32 values (2 KB), stored by TMA with
// 64-byte swizzle: the 16-byte chunk c of row r sits at chunk c ^ ((r >> 1) & 3), which also
// keeps the lanes' row-wise shared-memory writes free of bank conflicts.
constexpr int STAGE_BYTES = 32 * 64;

constexpr int ALPHA_SMEM_MAX = 4096;  // models up to this n_pad keep alpha in shared memory
inline size_t smem_bytes(bool alpha_smem)
{
    return (size_t)2 * A_SLOT + (size_t)STAGES * B_STAGE + (size_t)EPI_WARPS * STAGE_BYTES + 1024 + sizeof(Shared) +
           (alpha_smem ? sizeof(float) * ALPHA_SMEM_MAX : 0);
}

struct Params {
    int64_t C;            // candidates in this chunk
    int64_t c0;           // pool index of the first
    int n, n_pad, d;
    int num_tiles;
    float s2;
    uint64_t seed;
    const float *Xc;      // pool-indexed M x d, or null: drawn from seed
    float zs[DMAX];       // 1 / lengthscale
    const float *nb;      // n_pad: |z_i|^2
    const float *alpha;   // n_pad
    float *mu;            // pool-indexed
    unsigned *status;
    uint32_t idesc;
};

template <typename Out> struct Pack8;
template <> struct Pack8<__half> {
    __device__ static uint32_t two(float a, float b)
    {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
};
template <> struct Pack8<__nv_bfloat16> {
    __device__ static uint32_t two(float a, float b)
    {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
};

// s2 (1 + sqrt5 r + 5 r^2/3) exp(-sqrt5 r) with r = sqrt.approx(r2) (0 at 0) and
// exp via ex2.approx; c1 = s2 sqrt5, c2 = s2 5/3 are folded in by the caller.
__device__ __forceinline__ float matern_folded(float r2, float s2, float c1, float c2)
{
    float r, e;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(r2));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-3.2259460f * r));  // -sqrt5 / ln 2
    return fmaf(c2, r2, fmaf(c1, r, s2)) * e;
}
// The same for two squared distances, the FP32 arithmetic on paired lanes (each lane's result
// is the scalar form's, bit for bit).
__device__ __forceinline__ float2 matern_folded2(float2 r2, float s2, float c1, float c2)
{
    float2 r, e;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r.x) : "f"(r2.x));
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r.y) : "f"(r2.y));
    const float2 a = mul2(make_float2(-3.2259460f, -3.2259460f), r);  // -sqrt5 / ln 2
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e.x) : "f"(a.x));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e.y) : "f"(a.y));
    const float2 p = fma2(make_float2(c2, c2), r2, fma2(make_float2(c1, c1), r, make_float2(s2, s2)));
    return mul2(p, e);
}

// Build A' row `r` of tile `t` into slot base `a` (128B-swizzled K-major, two 64-column tiles).
__device__ __forceinline__ float build_row(unsigned char *a, int r, int64_t t, const Params &P)
{
    const int64_t cl = t * BM + r;
    const int64_t c = P.c0 + cl;
    float z[DMAX];
    float na = 0.0f;
#pragma unroll
    for (int k = 0; k < DMAX; ++k) {
        float x = 0.0f;
        if (k < P.d) {
            if (P.Xc) x = cl < P.C ? P.Xc[c * P.d + k] : 0.5f;
            else x = uniform24f(P.seed, 2, (uint64_t)(c * P.d + k));
            z[k] = (x - 0.5f) * P.zs[k];
        } else {
            z[k] = 0.0f;
        }
        na = fmaf(z[k], z[k], na);
    }
    uint32_t hi[DMAX / 2], lo[DMAX / 2];
#pragma unroll
    for (int k = 0; k < DMAX; k += 2) {
        const __half h0 = __float2half_rn(z[k]), h1 = __float2half_rn(z[k + 1]);
        const __half l0 = __float2half_rn(z[k] - __half2float(h0)), l1 = __float2half_rn(z[k + 1] - __half2float(h1));
        // -2 x (exact in FP16)
        __half2 hh = __hmul2(__halves2half2(h0, h1), __float2half2_rn(-2.0f));
        __half2 ll = __hmul2(__halves2half2(l0, l1), __float2half2_rn(-2.0f));
        hi[k / 2] = *reinterpret_cast<uint32_t *>(&hh);
        lo[k / 2] = *reinterpret_cast<uint32_t *>(&ll);
    }
    __half2 one2 = __float2half2_rn(1.0f);
    const uint32_t ones = *reinterpret_cast<uint32_t *>(&one2);
    // chunk j (16 bytes = 8 halves) of row r sits at r * 128 + ((j ^ (r & 7)) * 16)
    unsigned char *row0 = a + r * 128, *row1 = a + A_TILE + r * 128;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int sj = (j ^ (r & 7)) * 16;
        const int src = (j & 3) * 4;  // 4 uint32 = 8 halves
        uint4 v0 = make_uint4(hi[src], hi[src + 1], hi[src + 2], hi[src + 3]);  // [hi | hi]
        uint4 v1 = j < 4 ? make_uint4(lo[src], lo[src + 1], lo[src + 2], lo[src + 3])
                         : (j == 4 ? make_uint4(ones, 0, 0, 0) : make_uint4(0, 0, 0, 0));  // [lo | 1 1 0 ..]
        *reinterpret_cast<uint4 *>(row0 + sj) = v0;
        *reinterpret_cast<uint4 *>(row1 + sj) = v1;
    }
    return na;
}

template <typename Out, bool ALPHA_SMEM>
__global__ void __launch_bounds__(THREADS, 1) k_xkern_tc(const __grid_constant__ CUtensorMap map_b, const __grid_constant__ CUtensorMap map_k,
                                                    const Params P)
{
    extern __shared__ unsigned char smraw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char *aslot = base;                       // 2 x A_SLOT
    unsigned char *bst = base + 2 * A_SLOT;            // STAGES x B_STAGE
    unsigned char *stg = bst + (size_t)STAGES * B_STAGE;  // EPI_WARPS x STAGE_BYTES
    Shared *sh = (Shared *)(stg + (size_t)EPI_WARPS * STAGE_BYTES);
    float *alpha_s = (float *)(sh + 1);  // n_pad floats when ALPHA_SMEM
    if (ALPHA_SMEM)
        for (int i = threadIdx.x; i < P.n_pad; i += blockDim.x) alpha_s[i] = P.alpha[i];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int nq = P.n_pad / BN;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&sh->full[s], 1);
            mbar_init(&sh->empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&sh->acc_full[a], 1);
            mbar_init(&sh->acc_empty[a], EPI_WARPS);
            mbar_init(&sh->a_full[a], 4);
            mbar_init(&sh->a_empty[a], 1 + EPI_WARPS);  // MMA commit + every epilogue warp read |z_c|^2
            mbar_init(&sh->mu_ready[a], 4 * (GROUPS - 1));
            mbar_init(&sh->mu_free[a], 4);
        }
        mbar_init(&sh->drain, 1);
        sh->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
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
            // ---------------- TMA: B' chunks (the same sequence for every tile)
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&map_b) : "memory");
            int stage = 0;
            uint32_t phase = 0;
            int armed[STAGES];
            uint32_t armed_par[STAGES];
            for (int s = 0; s < STAGES; ++s) armed[s] = 0, armed_par[s] = 0;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < P.num_tiles; t += gridDim.x) {
                for (int q = 0; q < nq; ++q) {
                    if (!mbar_wait(&sh->empty[stage], phase ^ 1u, abort_flag, P.status)) { ok = false; break; }
                    unsigned char *b = bst + (size_t)stage * B_STAGE;
                    mbar_arrive_expect_tx(&sh->full[stage], B_STAGE);
                    armed[stage] = 1;
                    armed_par[stage] = phase;
                    tma_load_2d(b, &map_b, 0, q * BN, &sh->full[stage]);
                    tma_load_2d(b + B_TILE, &map_b, 64, q * BN, &sh->full[stage]);
                    if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                }
            }
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
            int k = 0;
            for (int t = blockIdx.x; ok && t < P.num_tiles; t += gridDim.x, ++k) {
                const int slot = k & 1;
                if (!mbar_wait(&sh->a_full[slot], (uint32_t)(k >> 1) & 1u, abort_flag, P.status)) break;
                tc_fence_after();
                const unsigned char *a = aslot + (size_t)slot * A_SLOT;
                for (int q = 0; q < nq; ++q) {
                    if (!mbar_wait(&sh->acc_empty[acc], acc_phase ^ 1u, abort_flag, P.status)) { ok = false; break; }
                    if (!mbar_wait(&sh->full[stage], phase, abort_flag, P.status)) { ok = false; break; }
                    tc_fence_after();
                    const unsigned char *b = bst + (size_t)stage * B_STAGE;
                    const uint32_t d_tmem = tmem + (uint32_t)(acc * BN);
#pragma unroll
                    for (int kt = 0; kt < 2; ++kt)
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            mma_f16(d_tmem, smem_desc(a + kt * A_TILE + kk * 32), smem_desc(b + kt * B_TILE + kk * 32),
                                    P.idesc, (kt | kk) ? 1u : 0u);
                    mma_commit(&sh->empty[stage]);
                    mma_commit(&sh->acc_full[acc]);
                    if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                    if (++acc == 2) { acc = 0; acc_phase ^= 1u; }
                }
                if (!ok) break;
                mma_commit(&sh->a_empty[slot]);  // A' slot free once this tile's MMAs complete
            }
            mma_commit(&sh->drain);
            mbar_wait(&sh->drain, 0, abort_flag, P.status, false);
        }
    } else {
        // ---------------- epilogue (+ A' builders in warps 2..5)
        const int ew = warp - 2;
        const int quad = warp & 3;
        const int grp = ew >> 2;                // column group: 64 of the chunk's 256 columns
        const int row = quad * 32 + lane;
        const bool builder = grp == 0;
        const float s2 = P.s2, c1 = P.s2 * 2.2360680f, c2 = P.s2 * 1.6666666f;
        const uint32_t lane_addr = (uint32_t)(quad * 32) << 16;
        uint4 *my_stage = reinterpret_cast<uint4 *>(stg + (size_t)ew * STAGE_BYTES);
        int acc = 0;
        uint32_t acc_phase = 0;
        bool ok = true;
        // A' for this CTA's first tile
        if (builder && (int)blockIdx.x < P.num_tiles) {
            sh->na[0][row] = build_row(aslot, row, blockIdx.x, P);
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh->a_full[0]);
        }
        int k = 0;
        for (int t = blockIdx.x; ok && t < P.num_tiles; t += gridDim.x, ++k) {
            const int slot = k & 1;
            // A' for the next tile into the other slot (its previous tile's MMAs are done)
            const int tn = t + gridDim.x;
            if (builder && tn < P.num_tiles) {
                const int ns = (k + 1) & 1;
                const bool g = mbar_wait_inl(&sh->a_empty[ns], ((uint32_t)((k + 1) >> 1) & 1u) ^ 1u, abort_flag, P.status);
                if (!__all_sync(0xffffffffu, g)) { ok = false; break; }
                sh->na[ns][row] = build_row(aslot + (size_t)ns * A_SLOT, row, tn, P);
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh->a_full[ns]);
            }
            // this tile's |z_c|^2
            const bool ga = mbar_wait_inl(&sh->a_full[slot], (uint32_t)(k >> 1) & 1u, abort_flag, P.status);
            if (!__all_sync(0xffffffffu, ga)) { ok = false; break; }
            const float na = sh->na[slot][row];
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh->a_empty[slot]);
            const int64_t cl = (int64_t)t * BM + row;
            const int64_t row0 = (int64_t)t * BM + quad * 32;  // the warp's first row
            float2 mu2 = make_float2(0.0f, 0.0f);  // mu as even- and odd-observation partial sums
            for (int q = 0; q < nq; ++q) {
                const bool g = mbar_wait_inl(&sh->acc_full[acc], acc_phase, abort_flag, P.status);
                if (!__all_sync(0xffffffffu, g)) { ok = false; break; }
                tc_fence_after();
#pragma unroll 1
                for (int cb = 0; cb < 2; ++cb) {
                    float v[32];
                    tmem_ld32(tmem + lane_addr + (uint32_t)(acc * BN + grp * 64 + cb * 32), v);
                    const int i0 = q * BN + grp * 64 + cb * 32;
                    uint32_t pk[16];
#pragma unroll
                    for (int j = 0; j < 32; j += 4) {
                        const float4 al = ALPHA_SMEM ? *reinterpret_cast<const float4 *>(alpha_s + i0 + j)
                                                     : *reinterpret_cast<const float4 *>(P.alpha + i0 + j);
                        // padded observations: alpha = 0 and the 16-bit L^-1 rows are zero there,
                        // so their (finite) K* values never reach mu or sigma
                        const float2 d01 = add2(make_float2(v[j], v[j + 1]), make_float2(na, na));
                        const float2 d23 = add2(make_float2(v[j + 2], v[j + 3]), make_float2(na, na));
                        const float2 k01 = matern_folded2(make_float2(fmaxf(d01.x, 0.0f), fmaxf(d01.y, 0.0f)), s2, c1, c2);
                        const float2 k23 = matern_folded2(make_float2(fmaxf(d23.x, 0.0f), fmaxf(d23.y, 0.0f)), s2, c1, c2);
                        mu2 = fma2(k01, make_float2(al.x, al.y), mu2);
                        mu2 = fma2(k23, make_float2(al.z, al.w), mu2);
                        pk[j / 2] = Pack8<Out>::two(k01.x, k01.y);
                        pk[j / 2 + 1] = Pack8<Out>::two(k23.x, k23.y);
                    }
                    // K* out: each lane writes its row's 64 bytes into the warp's staging tile
                    // (once the previous tile's TMA store has read it), one lane stores the
                    // 32 x 32 tile; rows past C are clipped by the tensor map
                    if (lane == 0) bulk_wait_read0();
                    __syncwarp();
                    const int sw = (lane >> 1) & 3;
#pragma unroll
                    for (int w4 = 0; w4 < 4; ++w4)
                        my_stage[lane * 4 + (w4 ^ sw)] =
                            make_uint4(pk[4 * w4], pk[4 * w4 + 1], pk[4 * w4 + 2], pk[4 * w4 + 3]);
                    fence_async_smem();
                    __syncwarp();
                    if (lane == 0 && row0 < P.C) {
                        tma_store_2d(&map_k, my_stage, i0, (int)row0);
                        bulk_commit();
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh->acc_empty[acc]);
                if (++acc == 2) { acc = 0; acc_phase ^= 1u; }
            }
            if (!ok) break;
            const float mu = mu2.x + mu2.y;
            // combine the column groups' partial means (group 0 writes the result)
            const uint32_t use = (uint32_t)(k >> 1) & 1u;
            if (!builder) {
                const bool g = mbar_wait_inl(&sh->mu_free[slot], use ^ 1u, abort_flag, P.status);
                if (!__all_sync(0xffffffffu, g)) { ok = false; break; }
                sh->mu_part[slot][grp - 1][row] = mu;
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh->mu_ready[slot]);
            } else {
                const bool g = mbar_wait_inl(&sh->mu_ready[slot], use, abort_flag, P.status);
                if (!__all_sync(0xffffffffu, g)) { ok = false; break; }
                float m = mu;
#pragma unroll
                for (int gg = 0; gg < GROUPS - 1; ++gg) m += sh->mu_part[slot][gg][row];
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh->mu_free[slot]);
                if (cl < P.C) P.mu[P.c0 + cl] = m;
            }
        }
        if (lane == 0) bulk_wait_all0();  // the last K* tiles are written before the CTA ends
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// Observation split B' = [hi | lo | hi | s_hi s_lo 0 ..] (n_pad x 128 FP16) with s = |z_i|^2,
// and s in FP32, from FP64 X.
__global__ void k_obs_split(const double *__restrict__ X, int n, int d, int n_pad, Lengthscales_inv ls,
                            __half *__restrict__ B, float *__restrict__ nb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pad) return;
    double s = 0.0;
    __half *row = B + (size_t)i * KB;
    for (int k = 0; k < DMAX; ++k) {
        const float z = (i < n && k < d) ? (float)((X[(size_t)i * d + k] - 0.5) * ls.inv[k]) : 0.0f;
        s += (double)z * (double)z;
        const __half h = __float2half_rn(z);
        const __half l = __float2half_rn(z - __half2float(h));
        row[k] = h;
        row[32 + k] = l;
        row[64 + k] = h;
        row[96 + k] = __float2half_rn(0.0f);
    }
    nb[i] = (float)s;
    const __half sh = __float2half_rn((float)s);
    row[96] = sh;
    row[97] = __float2half_rn((float)(s - (double)__half2float(sh)));
}

}  // namespace xtc

int xkern_tc_prepare(gpbo_ctx *ctx, gp_model *m)
{
    if (m->d > xtc::DMAX) return GPBO_OK;  // wider inputs use the CUDA-core cross-kernel
    Lengthscales_inv ls;
    for (int k = 0; k < m->d; ++k) ls.inv[k] = 1.0 / m->ls[k];
    xtc::k_obs_split<<<(m->n_pad + 127) / 128, 128, 0, ctx->stream>>>(m->X, m->n, m->d, m->n_pad, ls,
                                                                      (__half *)m->Zsplit, m->nb32);
    GPBO_LAUNCH_CHECK(ctx);
    return GPBO_OK;
}

bool xkern_tc_usable(const gp_model *m) { return m->Zsplit != nullptr && m->d <= xtc::DMAX; }

int xkern_tc(gpbo_ctx *ctx, const gp_model *m, const float *Xc, uint64_t seed, int64_t c0, int64_t C, void *Kst,
             float *mu)
{
    if (m->n_pad % xtc::BN != 0 || !Kst || ((uintptr_t)Kst & 15) || C <= 0 || C > 0x7fffffffll) return GPBO_EINVAL;
    CUtensorMap mb, mk;
    GPBO_TRY(encode_2d(&mb, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, m->Zsplit, (uint64_t)m->n_pad, (uint64_t)xtc::KB, xtc::BN));
    GPBO_TRY(encode_2d_box(&mk,
                           m->prec == GPBO_PREC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                           Kst, (uint64_t)C, (uint64_t)m->n_pad, 32, 32, CU_TENSOR_MAP_SWIZZLE_64B));
    xtc::Params P;
    P.C = C;
    P.c0 = c0;
    P.n = m->n;
    P.n_pad = m->n_pad;
    P.d = m->d;
    P.num_tiles = (int)cdiv64(C, xtc::BM);
    P.s2 = (float)m->s2;
    P.seed = seed;
    P.Xc = Xc;
    for (int k = 0; k < xtc::DMAX; ++k) P.zs[k] = k < m->d ? (float)(1.0 / m->ls[k]) : 0.0f;
    P.nb = m->nb32;
    P.alpha = m->alpha32;
    P.mu = mu;
    P.status = ctx->dev_status;
    P.idesc = tcx::idesc_f16(0u, xtc::BN, xtc::BM);
    const int grid = std::min(P.num_tiles, ctx->sm_count);
    const bool as = m->n_pad <= xtc::ALPHA_SMEM_MAX;
    const size_t smem = xtc::smem_bytes(as);
    auto launch = [&](auto kern) -> int {
        GPBO_TRY(ensure_smem((const void *)kern, ctx->device, (int)smem));
        kern<<<grid, xtc::THREADS, smem, ctx->stream>>>(mb, mk, P);
        return GPBO_OK;
    };
    if (m->prec == GPBO_PREC_BF16) {
        GPBO_TRY(as ? launch(xtc::k_xkern_tc<__nv_bfloat16, true>) : launch(xtc::k_xkern_tc<__nv_bfloat16, false>));
    } else {
        GPBO_TRY(as ? launch(xtc::k_xkern_tc<__half, true>) : launch(xtc::k_xkern_tc<__half, false>));
    }
    GPBO_LAUNCH_CHECK(ctx);
    return GPBO_OK;
}

}  // namespace gpbo
