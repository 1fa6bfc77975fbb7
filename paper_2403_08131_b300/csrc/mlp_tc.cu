// Ensemble pre-screen forward on the tensor cores (FP16 operands, FP32 accumulate), fused
// with the ensemble combine and the expected improvement of every candidate.
//
// For a tile of 128 candidates and each network e of the ensemble (d -> 256 -> 256 -> 2):
//   Z1 = [x | 1] [W1 ; b1]         tcgen05.mma, K = 32 (d <= 31 inputs, then the constant 1)
//   H1 = fp16(gelu(Z1))            epilogue; written to shared memory as the next A operand
//   Z2 = b2 + H1 W2                tcgen05.mma: the bias as [1 1] [b2_hi ; b2_lo] (one K = 16 step,
//                                  b2 = b2_hi + b2_lo to 2^-22 relative), then K = 256 in four
//                                  64-column K tiles
//   o  = gelu(Z2) W3 + b3          epilogue, FP32 on the CUDA cores (two outputs)
// then mu_e = o_0 sd_mu + mean_mu and sigma_e = exp(o_1 sd_ls + mean_ls); after the last
// network mu_bar = mean_e mu_e, sigma_bar^2 = mean_e sigma_e^2 + var_e mu_e and
// EI(mu_bar, sigma_bar) for minimisation.
// gelu is the tanh form of Hendrycks & Gimpel (2016) with the hardware tanh.approx.f32; it
// differs from z Phi(z) by < 5e-4 absolute.  Its factor 1/2 is folded into W2 and W3 (exact: a power of two), so the epilogues
// compute h' = z (1 + t) = 2 gelu(z) with one FMA.  FP16 rather than BF16 operands: the same
// tensor rate, 11 significant bits instead of 8.
//
// Roles (clusters of two CTAs, one CTA per SM, persistent over pairs of tiles; 608 threads):
//   warp 0      TMA: per network, [W1 ; b1 ; b2 split]^T (256 x 64, zero padded) then W2^T in
//               four 256 x 64 K chunks, through 3 stages of 32 KiB (the first chunk's stage is
//               held until layer 2's bias MMA).  Each CTA of a pair loads half of every chunk's
//               rows and multicasts it to both, and a stage is refilled once both CTAs' MMAs
//               are done with it, so L2 serves each chunk once per pair.  The packed ensemble
//               (8 networks, 1.3 MB) is read from L2 for every pair of tiles; W3 and b3 of
//               every network (E <= 8) stay in shared memory.
//   warp 1      TMEM (512 columns): network k keeps Z1 and then Z2 in region k mod 2 (256
//               columns each); one lane issues the MMAs
//   warps 2-17  epilogue: warp w reads TMEM lane quadrant w % 4 and column group (w-2) / 4;
//               warps 2-5 (group 0) also own the ensemble state of their rows (one thread =
//               one candidate)
//   warp 18     builds the x tiles (four rows a lane) into two buffers, up to one tile ahead:
//               the counter-RNG draws stay off the epilogue's path
// Per network k the epilogue writes H1 from Z1(k), then runs layer 2 of network k - 1: layer
// 2's MMAs of network k (into region k mod 2, once Z1(k) is read) run under that second part,
// and layer 1 of network k + 1 waits only for region (k + 1) mod 2, which Z2(k - 1) frees.
// Every wait is bounded (about 2 s of SM clock); on timeout the kernel raises DEV_TIMEOUT,
// every role leaves its loop, the producer waits (bounded) for its copies in flight, the MMA
// issuer drains, and the allocating warp frees TMEM.
#include "tc_common.cuh"

#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>

namespace gpbo {
namespace mtc {

using namespace tcx;

constexpr int BM = 128;                  // candidates per tile
constexpr int HID = 256;                 // hidden width (MMA N)
constexpr int KT = 64;                   // K elements per 128-byte swizzled row
constexpr int CHUNKS = 5;                // per network: [W1;b1]^T, then W2^T in 4 K chunks
constexpr int STAGES = 3;
constexpr int EPI_WARPS = 16;
constexpr int GROUPS = EPI_WARPS / 4;    // column groups
constexpr int BUILDER_WARP = 2 + EPI_WARPS;
constexpr int THREADS = (3 + EPI_WARPS) * 32;
constexpr int TMEM_COLS = 512;
constexpr int TILE_BYTES = BM * 128;     // one 128 x 64 BF16 K tile
constexpr int H1_BYTES = 4 * TILE_BYTES; // 128 x 256
constexpr int X_BYTES = TILE_BYTES;
constexpr int W_BYTES = HID * 128;       // one 256 x 64 FP16 chunk (a stage)
constexpr int W_HROWS = HID / 2;         // the half of a chunk's rows that each CTA of a pair loads
constexpr int W_HBYTES = W_BYTES / 2;
constexpr int AUX = 772;                 // per network FP32: b2 [256], W3 [256 x 2], b3 [2], pad 2
constexpr int EMAX = 8;                  // networks whose AUX rows stay in shared memory
constexpr int DMAX = 31;

struct alignas(16) Shared {
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    uint64_t z1_full;
    uint64_t h_full;           // the epilogue has read Z1 and written all of H1
    uint64_t z2_full[2], z2_empty[2];  // per TMEM region
    uint64_t x_full[2], x_empty[2];
    uint64_t part_ready[2], part_free[2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
    float2 part[2][GROUPS - 1][BM];      // layer-3 partial sums of column groups 1..3
};

inline size_t smem_bytes()
{
    return (size_t)H1_BYTES + 2 * X_BYTES + (size_t)STAGES * W_BYTES + 1024 + sizeof(Shared) + sizeof(float) * EMAX * AUX;
}

struct Params {
    int64_t C;          // candidates
    int64_t c0;         // pool index of the first
    int num_tiles;
    int num_ptiles;     // pair tiles: tiles 2 pt and 2 pt + 1 (the second past the end when num_tiles is odd)
    int E, d, nk1;      // networks, inputs, layer-1 MMA K steps (16 each)
    uint64_t seed;
    const float *Xc;    // pool-indexed rows of d, or null: drawn from seed (stream 2)
    const float *aux;   // E x AUX
    float n0, n1, n2, n3;
    float tau, xi;
    float *ei, *mu, *sigma;  // pool-indexed; mu and sigma may be null
    unsigned *status;
    uint32_t idesc;
};

// 2 gelu(z) in the tanh form: z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))).
// 2 gelu(z) of two elements: z (1 + tanh(z (c0 + c1 z^2))), c0 = sqrt(2/pi), c1 = 0.044715 c0
__device__ __forceinline__ float2 gelu2_tanh_x2(float2 z)
{
    const float2 u = mul2(z, fma2(mul2(z, z), make_float2(0.0356774081f, 0.0356774081f),
                                  make_float2(0.7978845608f, 0.7978845608f)));
    float2 t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t.x) : "f"(u.x));
    asm("tanh.approx.f32 %0, %1;" : "=f"(t.y) : "f"(u.y));
    return fma2(z, t, z);
}

__device__ __forceinline__ uint32_t pack_f16(float a, float b)
{
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

// Row r of the x tile of tile t: [x_0 .. x_{d-1}, 1, 0 ... | 1, 1, 0 ...] in FP16 (the second part
// from K column 32: the A operand of layer 2's bias), 128-byte swizzled
// (16-byte chunk j of row r at r * 128 + ((j ^ (r & 7)) * 16)).
// The fields come by value: a reference to the kernel's parameters would copy them to local memory.
__device__ __noinline__ void build_x(unsigned char *xs, int r, int64_t t, int64_t C, int64_t c0, int d,
                                     const float *Xc, uint64_t seed)
{
    const int64_t cl = t * BM + r;
    const int64_t c = c0 + cl;
    uint32_t w[16];
#pragma unroll
    for (int k = 0; k < 32; k += 2) {
        float v[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int kk = k + u;
            float x = 0.0f;
            if (kk < d) {
                if (Xc) x = cl < C ? Xc[c * d + kk] : 0.5f;
                else x = uniform24f(seed, 2, (uint64_t)(c * d + kk));
            } else if (kk == d) {
                x = 1.0f;
            }
            v[u] = x;
        }
        w[k / 2] = pack_f16(v[0], v[1]);
    }
    unsigned char *row = xs + r * 128;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint4 val = j < 4 ? make_uint4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3])
                                : make_uint4(j == 4 ? pack_f16(1.0f, 1.0f) : 0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4 *>(row + ((j ^ (r & 7)) * 16)) = val;
    }
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(THREADS, 1)
    k_mlp_screen_tc(const __grid_constant__ CUtensorMap map_w, const Params P)
{
    extern __shared__ unsigned char smraw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char *h1 = base;                       // 4 K tiles
    unsigned char *xs = base + H1_BYTES;            // 2 x tiles (tile ti in buffer ti & 1)
    unsigned char *wst = xs + 2 * X_BYTES;          // STAGES x W_BYTES
    Shared *sh = (Shared *)(wst + (size_t)STAGES * W_BYTES);
    float *aux_s = (float *)(sh + 1);               // E x AUX (16-byte aligned: Shared is)
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t rank = cluster_rank();
    const int pair = (int)(blockIdx.x >> 1), npairs = (int)(gridDim.x >> 1);
    for (int i = threadIdx.x; i < P.E * AUX; i += blockDim.x) aux_s[i] = P.aux[i];

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&sh->full[s], 1);
            mbar_init(&sh->empty[s], 2);  // both CTAs' MMAs are done with the stage
        }
        mbar_init(&sh->z1_full, 1);
        mbar_init(&sh->h_full, EPI_WARPS);
        for (int r = 0; r < 2; ++r) {
            mbar_init(&sh->z2_full[r], 1);
            mbar_init(&sh->z2_empty[r], EPI_WARPS);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sh->x_full[b], 1);
            mbar_init(&sh->x_empty[b], 1);
        }
        for (int p = 0; p < 2; ++p) {
            mbar_init(&sh->part_ready[p], 4 * (GROUPS - 1));
            mbar_init(&sh->part_free[p], 4);
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
    cluster_sync();  // both CTAs' barriers are initialised before either signals the other
    tc_fence_after();
    const uint32_t tmem = sh->tmem_base;
    volatile int *abort_flag = &sh->abort;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer: the same chunk sequence for every tile.  The CTAs of
            // a pair run the same sequence; each loads half of every chunk's rows and multicasts
            // it to both, so L2 serves each chunk once per pair
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&map_w) : "memory");
            int stage = 0;
            uint32_t phase = 0;
            uint32_t armed = 0, armed_par = 0;  // bit s: stage s has a copy issued, and its phase
            bool ok = true;
            for (int pt = pair; ok && pt < P.num_ptiles; pt += npairs)
                for (int e = 0; ok && e < P.E; ++e)
                    for (int c = 0; c < CHUNKS; ++c) {
                        if (!mbar_wait_fast(&sh->empty[stage], phase ^ 1u, abort_flag, P.status)) { ok = false; break; }
                        mbar_arrive_expect_tx(&sh->full[stage], W_BYTES);
                        armed |= 1u << stage;
                        armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
                        tma_load_2d_mc(wst + (size_t)stage * W_BYTES + (size_t)rank * W_HBYTES, &map_w, 0,
                                       (e * CHUNKS + c) * HID + (int)rank * W_HROWS, &sh->full[stage], 3);
                        if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                    }
            for (int s = 0; s < STAGES; ++s)
                if ((armed >> s) & 1u) mbar_wait(&sh->full[s], (armed_par >> s) & 1u, abort_flag, P.status, false);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer
            int stage = 0;
            uint32_t phase = 0;
            uint32_t k = 0, ti = 0;
            bool ok = true;
            for (int pt = pair; ok && pt < P.num_ptiles; pt += npairs, ++ti) {
                for (int e = 0; ok && e < P.E; ++e, ++k) {
                    // Network k holds Z1 and then Z2 in TMEM region k & 1 (256 columns each): layer
                    // 1 waits until the epilogue has read Z2 of network k - 2 from that region
                    const uint32_t r = k & 1u;
                    const uint32_t rk = tmem + r * (uint32_t)HID;
                    const int xb = (int)(ti & 1u);
                    const unsigned char *xt = xs + xb * X_BYTES;
                    if (e == 0 && !mbar_wait_fast(&sh->x_full[xb], (ti >> 1) & 1u, abort_flag, P.status)) { ok = false; break; }
                    if (k >= 2 && !mbar_wait_fast(&sh->z2_empty[r], ((k >> 1) & 1u) ^ 1u, abort_flag, P.status)) { ok = false; break; }
                    if (!mbar_wait_fast(&sh->full[stage], phase, abort_flag, P.status)) { ok = false; break; }
                    tc_fence_after();
                    const unsigned char *w0 = wst + (size_t)stage * W_BYTES;
                    for (int kk = 0; kk < P.nk1; ++kk)
                        mma_f16(rk, smem_desc(xt + kk * 32), smem_desc(w0 + kk * 32), P.idesc, kk ? 1u : 0u);
                    mma_commit(&sh->z1_full);
                    // layer 2 into the same region once the epilogue has read all of Z1 and written
                    // H1: first the bias, Z2 = [1 1] [b2_hi ; b2_lo] (K columns 32..47 of the x tile
                    // and of chunk 0), then H1 W2 K tile by K tile.  These MMAs run while the
                    // epilogue works on layer 2 of network k - 1.
                    if (!mbar_wait_fast(&sh->h_full, k & 1u, abort_flag, P.status)) { ok = false; break; }
                    tc_fence_after();
                    mma_f16(rk, smem_desc(xt + 64), smem_desc(w0 + 64), P.idesc, 0u);
                    mma_commit_mc(&sh->empty[stage], 3);
                    if (e == P.E - 1) mma_commit(&sh->x_empty[xb]);  // the tile's last read of its x tile
                    if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                    for (int q = 0; q < 4; ++q) {
                        if (!mbar_wait_fast(&sh->full[stage], phase, abort_flag, P.status)) { ok = false; break; }
                        tc_fence_after();
                        const unsigned char *w = wst + (size_t)stage * W_BYTES;
                        const unsigned char *a = h1 + q * TILE_BYTES;
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            mma_f16(rk, smem_desc(a + kk * 32), smem_desc(w + kk * 32), P.idesc, 1u);
                        mma_commit_mc(&sh->empty[stage], 3);
                        if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                    }
                    if (!ok) break;
                    mma_commit(&sh->z2_full[r]);
                }
            }
            mma_commit(&sh->drain);
            mbar_wait(&sh->drain, 0, abort_flag, P.status, false);
        }
    } else if (warp == BUILDER_WARP) {
        // ---------------- x tiles, up to one tile ahead of the MMAs (two buffers)
        uint32_t ti = 0;
        for (int pt = pair; pt < P.num_ptiles; pt += npairs, ++ti) {
            const int64_t t = 2 * (int64_t)pt + rank;
            const int b = (int)(ti & 1u);
            const bool g = mbar_wait_inl(&sh->x_empty[b], ((ti >> 1) & 1u) ^ 1u, abort_flag, P.status);
            if (!__all_sync(0xffffffffu, g)) break;
            for (int r = lane; r < BM; r += 32) build_x(xs + b * X_BYTES, r, t, P.C, P.c0, P.d, P.Xc, P.seed);
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh->x_full[b]);
        }
    } else {
        // ---------------- epilogue
        // Per network k: the layer-1 epilogue of k, then the layer-2 epilogue of k - 1 (whose
        // MMAs ran under the first).
        const int ew = warp - 2;
        const int quad = warp & 3;
        const int grp = ew >> 2;
        const int row = quad * 32 + lane;
        const bool owner = grp == 0;  // owns its rows' ensemble state
        const uint32_t lane_addr = (uint32_t)(quad * 32) << 16;
        const float invE = 1.0f / (float)P.E;
        float mu_shift = 0.f, sm = 0.f, sm2 = 0.f, sv = 0.f;  // ensemble state (group 0)
        // layer-2 epilogue, layer 3 and the column-group combine of network kk (network ee of
        // its tile; ccl: this thread's candidate)
        auto layer2 = [&](uint32_t kk, int ee, int64_t ccl) -> bool {
            const uint32_t r = kk & 1u;
            const bool got = mbar_wait_inl(&sh->z2_full[r], (kk >> 1) & 1u, abort_flag, P.status);
            if (!__all_sync(0xffffffffu, got)) return false;
            tc_fence_after();
            const float *aux = aux_s + ee * AUX;
            const uint32_t zc = tmem + lane_addr + r * (uint32_t)HID + (uint32_t)(grp * 64);
            // layer 3 on pairs of hidden units: a0 = (even, odd) partial sums of output 0, a1 of output 1
            float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
            {
                uint32_t va[16], vb[16];
                tmem_ld16_nw(zc, va);
                tmem_wait();
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint32_t *cur = (q & 1) ? vb : va;
                    uint32_t *nxt = (q & 1) ? va : vb;
                    if (q < 3) tmem_ld16_nw(zc + (uint32_t)((q + 1) * 16), nxt);
                    pin16(cur);
                    const int j0 = grp * 64 + q * 16;
#pragma unroll
                    for (int j = 0; j < 16; j += 2) {
                        // W3 rows j, j+1 as (w[j][0], w[j+1][0], w[j][1], w[j+1][1])
                        const float4 wv = *reinterpret_cast<const float4 *>(aux + HID + 2 * (j0 + j));
                        const float2 h = gelu2_tanh_x2(make_float2(__uint_as_float(cur[j]), __uint_as_float(cur[j + 1])));
                        a0 = fma2(h, make_float2(wv.x, wv.y), a0);
                        a1 = fma2(h, make_float2(wv.z, wv.w), a1);
                    }
                    if (q < 3) tmem_wait();
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh->z2_empty[r]);
            float o0 = a0.x + a0.y, o1 = a1.x + a1.y;
            // groups 1..3 hand their sums to group 0, which updates the ensemble state
            const int par = kk & 1;
            const uint32_t use = (kk >> 1) & 1u;
            if (!owner) {
                const bool g = mbar_wait_inl(&sh->part_free[par], use ^ 1u, abort_flag, P.status);
                if (!__all_sync(0xffffffffu, g)) return false;
                sh->part[par][grp - 1][row] = make_float2(o0, o1);
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh->part_ready[par]);
                return true;
            }
            const bool g = mbar_wait_inl(&sh->part_ready[par], use, abort_flag, P.status);
            if (!__all_sync(0xffffffffu, g)) return false;
#pragma unroll
            for (int gg = 0; gg < GROUPS - 1; ++gg) {
                const float2 v = sh->part[par][gg][row];
                o0 += v.x;
                o1 += v.y;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh->part_free[par]);
            const float m = (o0 + aux[3 * HID]) * P.n1 + P.n0;
            const float s = expf((o1 + aux[3 * HID + 1]) * P.n3 + P.n2);
            if (ee == 0) {
                mu_shift = m;
                sm = sm2 = sv = 0.f;
            }
            const float dm = m - mu_shift;
            sm += dm;
            sm2 = fmaf(dm, dm, sm2);
            sv = fmaf(s, s, sv);
            if (ee == P.E - 1 && ccl < P.C) {
                const float mm = sm * invE;
                const float mbar = mu_shift + mm;
                const float sbar = sqrtf(sv * invE + fmaxf(sm2 * invE - mm * mm, 0.f));
                const int64_t c = P.c0 + ccl;
                P.ei[c] = ei_minf(mbar, sbar, P.tau, P.xi);
                if (P.mu) P.mu[c] = mbar;
                if (P.sigma) P.sigma[c] = sbar;
            }
            return true;
        };
        uint32_t k = 0;
        bool ok = true;
        bool has_prev = false;  // network k - 1 waits for its layer-2 epilogue
        int prev_e = 0;
        int64_t prev_cl = 0;
        for (int pt = pair; ok && pt < P.num_ptiles; pt += npairs) {
            const int64_t cl = (2 * (int64_t)pt + rank) * BM + row;
            for (int e = 0; e < P.E; ++e, ++k) {
                // ---- layer-1 epilogue: H1 = fp16(2 gelu(Z1)), K tile by K tile
                const bool g = mbar_wait_inl(&sh->z1_full, k & 1u, abort_flag, P.status);
                if (!__all_sync(0xffffffffu, g)) { ok = false; break; }
                tc_fence_after();
                const uint32_t z1c = tmem + lane_addr + (k & 1u) * (uint32_t)HID + (uint32_t)(grp * 16);
                // K tile q's 16 columns are processed while tile q+1's load is in flight
                uint32_t va[16], vb[16];
                tmem_ld16_nw(z1c, va);
                tmem_wait();
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint32_t *cur = (q & 1) ? vb : va;
                    uint32_t *nxt = (q & 1) ? va : vb;
                    if (q < 3) tmem_ld16_nw(z1c + (uint32_t)((q + 1) * KT), nxt);
                    pin16(cur);
                    uint32_t w[8];
#pragma unroll
                    for (int j = 0; j < 16; j += 2) {
                        const float2 h = gelu2_tanh_x2(make_float2(__uint_as_float(cur[j]), __uint_as_float(cur[j + 1])));
                        w[j / 2] = pack_f16(h.x, h.y);
                    }
                    unsigned char *dst = h1 + q * TILE_BYTES + row * 128;
                    const int j0 = 2 * grp, j1 = 2 * grp + 1;
                    *reinterpret_cast<uint4 *>(dst + ((j0 ^ (row & 7)) * 16)) = make_uint4(w[0], w[1], w[2], w[3]);
                    *reinterpret_cast<uint4 *>(dst + ((j1 ^ (row & 7)) * 16)) = make_uint4(w[4], w[5], w[6], w[7]);
                    if (q < 3) tmem_wait();
                }
                // all of Z1 read (the region takes Z2 next) and all of H1 written
                fence_async_smem();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh->h_full);
                // ---- layer 2 of the previous network, whose MMAs ran under this epilogue
                if (has_prev && !layer2(k - 1, prev_e, prev_cl)) { ok = false; break; }
                has_prev = true;
                prev_e = e;
                prev_cl = cl;
            }
        }
        if (ok && has_prev) layer2(k - 1, prev_e, prev_cl);
    }
    tc_fence_before();
    __syncthreads();
    // neither CTA leaves while the other may still write its stages or signal its barriers
    cluster_sync();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// Pack one network's FP32 parameters (layout W1 [d x H], b1, W2 [H x H], b2, W3 [H x 2], b3)
// into the kernel's operands: wt = E x 5 chunks of 256 x 64 FP16, K-major
//   chunk 0: row j = [W1[0][j] .. W1[d-1][j], b1[j], 0 ... | b2_hi[j], b2_lo[j], 0 ...] (the second
//            part from K column 32: b2_hi = fp16(b2[j]), b2_lo = fp16(b2[j] - b2_hi))
//   chunk c = 1..4: row j = W2[64(c-1) .. 64c-1][j] / 2
// and aux = E x AUX FP32: b2 [256] (not read by the forward, which takes b2 from chunk 0),
// W3 [256 x 2] / 2 in pairs of rows (w[2p][0], w[2p+1][0], w[2p][1], w[2p+1][1]), b3 [2], zeros.
// The halves absorb gelu's factor 1/2 (the epilogues produce 2 gelu).
__global__ void k_pack(const float *__restrict__ theta, int E, int d, int64_t P, int64_t oW1, int64_t ob1,
                       int64_t oW2, int64_t ob2, int64_t oW3, int64_t ob3, __half *__restrict__ wt,
                       float *__restrict__ aux)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)CHUNKS * HID * KT;
    if (t < E * per) {
        const int e = (int)(t / per);
        const int64_t r = t - e * per;
        const int c = (int)(r / (HID * KT));
        const int j = (int)((r / KT) % HID);
        const int kk = (int)(r % KT);
        const float *th = theta + e * P;
        float v;
        __half hv;
        if (c == 0) {
            const float b2 = th[ob2 + j];
            const __half b2_hi = __float2half_rn(b2);
            if (kk == 32) hv = b2_hi;
            else if (kk == 33) hv = __float2half_rn(b2 - __half2float(b2_hi));
            else hv = __float2half_rn(kk < d ? th[oW1 + (int64_t)kk * HID + j] : (kk == d ? th[ob1 + j] : 0.0f));
        } else {
            hv = __float2half_rn(0.5f * th[oW2 + (int64_t)(64 * (c - 1) + kk) * HID + j]);
        }
        wt[t] = hv;
    }
    if (t < (int64_t)E * AUX) {
        const int e = (int)(t / AUX);
        const int i = (int)(t % AUX);
        const float *th = theta + e * P;
        float v = 0.0f;
        if (i < HID) v = th[ob2 + i];
        else if (i < 3 * HID) {
            // rows 2p and 2p+1 of W3 as (w[2p][0], w[2p+1][0], w[2p][1], w[2p+1][1])
            const int r = i - HID, pr = r / 4, o = (r / 2) & 1, sub = r & 1;
            v = 0.5f * th[oW3 + (int64_t)(2 * pr + sub) * 2 + o];
        }
        else if (i < 3 * HID + 2) v = th[ob3 + (i - 3 * HID)];
        aux[t] = v;
    }
}

}  // namespace mtc

bool mlp_tc_usable(int d, int H, int E) { return H == mtc::HID && d >= 1 && d <= mtc::DMAX && E >= 1 && E <= mtc::EMAX; }

size_t mlp_tc_weight_bytes(int E) { return (size_t)E * mtc::CHUNKS * mtc::W_BYTES; }
size_t mlp_tc_aux_floats(int E) { return (size_t)E * mtc::AUX; }

int mlp_tc_pack(gpbo_ctx *ctx, const float *theta, int E, int d, int64_t P, const int64_t off[6], void *wt, float *aux)
{
    const int64_t total = std::max<int64_t>((int64_t)E * mtc::CHUNKS * mtc::HID * mtc::KT, (int64_t)E * mtc::AUX);
    mtc::k_pack<<<(unsigned)cdiv64(total, 256), 256, 0, ctx->stream>>>(theta, E, d, P, off[0], off[1], off[2], off[3],
                                                                       off[4], off[5], (__half *)wt, aux);
    GPBO_LAUNCH_CHECK(ctx);
    return GPBO_OK;
}

int mlp_tc_score(gpbo_ctx *ctx, const void *wt, const float *aux, int E, int d, const double norm[4], const float *Xc,
                 uint64_t seed, int64_t c0, int64_t C, double tau, double xi, float *ei, float *mu, float *sigma)
{
    if (!mlp_tc_usable(d, mtc::HID, E) || C < 1 || !ei || ((uintptr_t)wt & 15) || ((uintptr_t)aux & 15))
        return GPBO_EINVAL;
    if (cdiv64(C, mtc::BM) > 0x7fffffffll) return GPBO_EINVAL;
    CUtensorMap mw;
    GPBO_TRY(encode_2d(&mw, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, wt, (uint64_t)E * mtc::CHUNKS * mtc::HID, mtc::KT,
                       mtc::W_HROWS));
    mtc::Params P;
    P.C = C;
    P.c0 = c0;
    P.num_tiles = (int)cdiv64(C, mtc::BM);
    P.num_ptiles = (P.num_tiles + 1) / 2;
    P.E = E;
    P.d = d;
    P.nk1 = (d + 1 + 15) / 16;
    P.seed = seed;
    P.Xc = Xc;
    P.aux = aux;
    P.n0 = (float)norm[0];
    P.n1 = (float)norm[1];
    P.n2 = (float)norm[2];
    P.n3 = (float)norm[3];
    P.tau = (float)tau;
    P.xi = (float)xi;
    P.ei = ei;
    P.mu = mu;
    P.sigma = sigma;
    P.status = ctx->dev_status;
    P.idesc = tcx::idesc_f16(0u, mtc::HID, mtc::BM);  // FP16 A and B
    const size_t smem = mtc::smem_bytes();
    GPBO_TRY(ensure_smem((const void *)mtc::k_mlp_screen_tc, ctx->device, (int)smem));
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
            cfg.blockDim = dim3(mtc::THREADS);
            cfg.dynamicSmemBytes = smem;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = 2;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            GPBO_CUDA_TRY(cudaOccupancyMaxActiveClusters(&pairs, (const void *)mtc::k_mlp_screen_tc, &cfg));
            if (pairs < 1) return GPBO_ENOTSUP;
            if (ctx->device >= 0 && ctx->device < 64) cached[ctx->device] = pairs;
        }
    }
    const int grid = 2 * std::min(P.num_ptiles, pairs);
    mtc::k_mlp_screen_tc<<<grid, mtc::THREADS, smem, ctx->stream>>>(mw, P);
    GPBO_LAUNCH_CHECK(ctx);
    return GPBO_OK;
}

}  // namespace gpbo
