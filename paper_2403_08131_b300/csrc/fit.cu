// Surrogate fit on the GPU (§III-A: the surrogate is retrained on every evaluated
// configuration; §IV-D: GP training costs O(N^3)).  Everything here is FP64 except the
// triangular inverse used by the FP32 and tensor-core scoring paths, which is formed in
// FP32 from the FP64 factor.
//
//   K      = s2 m(r) + sn2 I            k_kmat            (Matern-5/2 ARD)
//   K      = L L^T                      k_chol_*          (blocked, right-looking, NB = 64,
//                                                          lookahead of one block column)
//   alpha  = L^-T L^-1 y, refined once  k_fwd_wave/k_bwd_wave/k_residual (one launch per substitution)
//   L^-1                                k_gemm_batched, k_gemm128, tensor-core slice products
//                                       (level-by-level block recursion; for large models the
//                                       leading half under the factorisation's last steps)
//
// Padding: n is padded to n_pad (a multiple of 64, or of 256 for tensor-core models).
// Padded rows/columns of K are the identity, so L and L^-1 are the identity there, the
// padded right-hand side is zero, and alpha is zero there.  No kernel needs a ragged tail.
#include "fit_kernels.cuh"
#include "tc_common.cuh"
#include "int_math.cuh"

#include <utility>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>
#include <vector>

namespace gpbo {

// Single-problem kernels: thin wrappers over the bodies in fit_kernels.cuh.
__global__ void k_scale_x(const double *__restrict__ X, int n, int d, int n_pad, Lengthscales_inv ls,
                          double *__restrict__ Xs64, float *__restrict__ Xs32)
{
    k_scale_x_body(X, n, d, n_pad, ls, Xs64, Xs32, blockIdx.x, blockIdx.y);
}

__global__ void k_kmat(const double *__restrict__ Xs, int n, int d, int n_pad, double s2, double sn2,
                       double *__restrict__ K)
{
    k_kmat_body(Xs, n, d, n_pad, s2, sn2, K, blockIdx.x, blockIdx.y);
}

// Kernel matrix with the distances in exact integer arithmetic (models with the tensor-core
// updates): each coordinate x / l as the integer q = round(x / l 2^(58 - e)) (|x / l| < 2^e
// over the model, from k_xs_max; |q| <= 2^58), so every difference q_i - q_j and the sum of
// its d squares (below 2^125) are exact in 128 bits, rounded once to FP64 and scaled by
// 2^(2 (e - 58)).  Against the FP64 loop (one rounding per subtraction and per FMA) the
// distance is exact up to the inputs' quantisation (2^-59 of the largest |x / l|), and the
// 2 d FP64 operations per pair move to the integer pipe.  The Matern factor stays FP64 but for
// its square root and exponential (rsqrt_int, exp_neg_int in int_math.cuh).

// The Matern-5/2 factor with r = r2 rsqrt(r2) (within about 1 ulp of sqrt(r2)) and exp_neg_int.
__device__ __forceinline__ double matern52_r2_int(double r2)
{
    const double r = r2 > 0.0 ? r2 * rsqrt_int(r2) : 0.0;
    const double t = SQRT5 * r;
    return (1.0 + t + (5.0 / 3.0) * r2) * exp_neg_int(t);
}

__global__ void k_xs_max(const double *__restrict__ Xs, int64_t count, unsigned long long *__restrict__ xmax)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned long long m = t < count ? (unsigned long long)tcx::mag_bits(Xs[t]) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(xmax, m);
}

__global__ void k_kmat_fixed(const double *__restrict__ Xs, const unsigned long long *__restrict__ xmax, int n,
                             int d, int n_pad, double s2, double sn2, double *__restrict__ K, double *__restrict__ L)
{
    constexpr int P = 58;
    const int tj = blockIdx.x, ti = blockIdx.y;
    if (tj > ti) return;
    __shared__ long long qi[GPBO_MAX_D][32], qj[GPBO_MAX_D][32];
    __shared__ double tile[32][33];
    // a NaN or infinite coordinate makes the FP64 loop's K NaN (and the factorisation report
    // it); the fixed-point form would hide it, so it writes NaN entries instead
    const bool finite = *xmax < 0x7ff0000000000000ull;
    const int e = finite ? tcx::exp_of_mag(*xmax) : 0;
    for (int idx = threadIdx.y * 32 + threadIdx.x; idx < d * 32; idx += 32 * blockDim.y) {
        const int k = idx / 32, c = idx % 32;
        qi[k][c] = tcx::fixed_of(Xs[(int64_t)k * n_pad + ti * 32 + c], e, P);
        qj[k][c] = tcx::fixed_of(Xs[(int64_t)k * n_pad + tj * 32 + c], e, P);
    }
    __syncthreads();
    const int sh = 2 * (e - P);
    const bool fast = sh > -1000 && sh < 1000;
    const double scale = fast ? ldexp(1.0, sh) : 0.0;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = ti * 32 + r, j = tj * 32 + threadIdx.x;
        double v;
        if (i < n && j < n) {
            unsigned long long lo = 0, hi = 0;
            for (int k = 0; k < d; ++k) {
                const long long t = qi[k][r] - qj[k][threadIdx.x];
                const unsigned long long a = (unsigned long long)(t < 0 ? -t : t);
                const unsigned long long pl = a * a;
                lo += pl;
                hi += __umul64hi(a, a) + (lo < pl ? 1ull : 0ull);
            }
            const double S = (double)hi * 18446744073709551616.0 + (double)lo;  // hi 2^64 + lo
            const double r2 = fast ? S * scale : ldexp(S, sh);
            v = finite ? s2 * matern52_r2_int(r2) + (i == j ? sn2 : 0.0) : __longlong_as_double(0x7ff8000000000000ll);
        } else {
            v = i == j ? 1.0 : 0.0;
        }
        K[(int64_t)i * n_pad + j] = v;
        L[(int64_t)i * n_pad + j] = v;  // the factorisation's working copy (its lower triangle)
        tile[r][threadIdx.x] = v;
    }
    if (ti == tj) return;
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int j = tj * 32 + r, i = ti * 32 + threadIdx.x;
        K[(int64_t)j * n_pad + i] = tile[threadIdx.x][r];
    }
}

// Diagonal factor: warp 0 takes the pivots, 31 warps share each column's updates (the
// arithmetic per element does not depend on the count).
constexpr int DIAG_THREADS = 1024;
// Trailing updates of fewer than SLAB_BELOW x SMs whole 64 x 64 tiles (two waves at three
// CTAs per SM) run as 16-row slabs.  Slabs for every launch measured the same (22.3 ms per
// step): the update is FP64-bound, not wave-bound.
constexpr int SLAB_BELOW = 6;
constexpr int SLAB_ROWS = 4;
// Warps per CTA of the diagonal-block inverse (one column per warp, NB / INV_WARPS CTAs).  Two
// measured best at n = 4096 (Cholesky 8.54 ms against 8.68 with four and 9.04 with one): the
// inverse overlaps the tensor-core updates of the main stream, and narrower CTAs share fewer SMs'
// FP64 units with them; with one warp the load of the block dominates.
constexpr int INV_WARPS = 2;
// Programmatic dependent launch along the factorisation's chain (next-column update -> diagonal
// factor -> inverse -> panel, one stream): each kernel lets the next one be scheduled as soon as
// all of its own CTAs are running, and each waits (griddepcontrol.wait: the previous kernel has
// completed and its writes are visible) before it reads anything, so the launch latency of a
// dependent kernel overlaps the kernel before it.  Without the launch attribute both
// instructions do nothing.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
static int launch_pdl(gpbo_ctx *ctx, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                      Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    GPBO_CUDA_TRY(cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...));
    GPBO_LAUNCH_CHECK(ctx);
    return GPBO_OK;
}

__global__ void __launch_bounds__(DIAG_THREADS) k_chol_diag(double *__restrict__ A, int n_pad, int kb,
                                                   double *__restrict__ Dinv, unsigned *status)
{
    pdl_wait();
    pdl_trigger();
    k_chol_diag_body(A, n_pad, kb, Dinv, status, blockIdx.x, blockIdx.y);
}

__global__ void __launch_bounds__(128) k_chol_inv(const double *__restrict__ A, int n_pad, int kb,
                                                  double *__restrict__ Dinv)
{
    pdl_wait();
    pdl_trigger();
    k_chol_inv_body(A, n_pad, kb, Dinv, blockIdx.x);
}

__global__ void __launch_bounds__(128) k_chol_panel(double *__restrict__ A, int n_pad, int kb,
                                                    const double *__restrict__ Dinv, int boff)
{
    pdl_wait();
    k_chol_panel_body(A, n_pad, kb, Dinv, blockIdx.x, blockIdx.y, boff);
}

__global__ void __launch_bounds__(128) k_chol_panel_subst(double *__restrict__ A, int n_pad, int kb,
                                                          const double *__restrict__ Dinv)
{
    pdl_wait();
    pdl_trigger();
    k_chol_panel_subst_body(A, n_pad, kb, Dinv, blockIdx.x);
}

__global__ void __launch_bounds__(128) k_chol_panel_row(double *__restrict__ A, int n_pad, int kb,
                                                        const double *__restrict__ Dinv, int boff)
{
    pdl_wait();
    pdl_trigger();
    k_chol_panel_row_body(A, n_pad, kb, Dinv, boff, blockIdx.x);
}

__global__ void __launch_bounds__(128) k_chol_update_diagblk(double *__restrict__ A, int n_pad, int kb)
{
    pdl_wait();
    pdl_trigger();
    k_chol_update_diagblk_body(A, n_pad, kb, blockIdx.x);
}

__global__ void __launch_bounds__(256) k_chol_update(double *__restrict__ A, int n_pad, int kb, int nblk, int part)
{
    k_chol_update_body(A, n_pad, kb, nblk, blockIdx.x, blockIdx.y, part);
}

__global__ void __launch_bounds__(256) k_chol_update_slab(double *__restrict__ A, int n_pad, int kb, int part,
                                                          int t0)
{
    pdl_trigger();
    k_chol_update_slab_body<SLAB_ROWS>(A, n_pad, kb, blockIdx.x, part, t0);
}

__global__ void k_zero_upper_blocks(double *__restrict__ A, int n_pad)
{
    k_zero_upper_blocks_body(A, n_pad, blockIdx.x, blockIdx.y);
}

__global__ void k_residual(const double *__restrict__ K, const double *__restrict__ alpha,
                           const double *__restrict__ y, int n_pad, double *__restrict__ r)
{
    k_residual_body(K, alpha, y, n_pad, r, blockIdx.x, blockIdx.y);
}

// Refinement correction through L^-1 (bodies in fit_kernels.cuh).
template <typename T>
__global__ void __launch_bounds__(256) k_trmv(const T *__restrict__ X, int n_pad, const double *__restrict__ r,
                                              double *__restrict__ u)
{
    k_trmv_body(X, n_pad, r, u, blockIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(256) k_trmv_t_part(const T *__restrict__ X, int n_pad, const double *__restrict__ u,
                                                     double *__restrict__ part)
{
    k_trmv_t_part_body(X, n_pad, u, part, blockIdx.x, blockIdx.y);
}

__global__ void k_trmv_t_sum(const double *__restrict__ part, int n_pad, int chunks, double *__restrict__ a,
                             float *__restrict__ a32)
{
    k_trmv_t_sum_body(part, n_pad, chunks, a, a32, blockIdx.x);
}

__global__ void k_pad_copy(const double *__restrict__ y, int n, int n_pad, double *__restrict__ out)
{
    k_pad_copy_body(y, n, n_pad, out, blockIdx.x, blockIdx.y);
}

template <typename T>
__global__ void __launch_bounds__(256) k_gemm_batched(const T *__restrict__ Abase, const T *__restrict__ Bbase,
                                                      T *__restrict__ Cbase, int lda, int ldb, int ldc,
                                                      const GemmProb *__restrict__ probs, T alpha, int tri_a,
                                                      int tri_b)
{
    k_gemm_batched_body<T>(Abase, Bbase, Cbase, lda, ldb, ldc, probs, alpha, tri_a, tri_b, blockIdx.x, blockIdx.y);
}

__global__ void __launch_bounds__(256) k_fwd_wave(const double *__restrict__ L, const double *__restrict__ Dinv,
                                                  int n_pad, const double *__restrict__ w, double *z, int *flags,
                                                  int *ticket, unsigned *status)
{
    k_fwd_wave_body(L, Dinv, n_pad, w, z, flags, ticket, status);
}

__global__ void __launch_bounds__(256) k_bwd_wave(const double *__restrict__ L, const double *__restrict__ Dinv,
                                                  int n_pad, const double *__restrict__ w, double *x, int *flags,
                                                  int *ticket, unsigned *status)
{
    k_bwd_wave_body(L, Dinv, n_pad, w, x, flags, ticket, status);
}

__global__ void __launch_bounds__(256) k_gemm128(const float *__restrict__ A, const float *__restrict__ B,
                                                 float *__restrict__ C, const GemmProb *__restrict__ probs, float alpha,
                                                 int tri_a, int tri_b)
{
    k_gemm128_body(A, B, C, probs, alpha, tri_a, tri_b, blockIdx.x, blockIdx.y, blockIdx.z);
}

template <typename T>
__global__ void k_linv_init(const double *__restrict__ Dinv, int n_pad, T *__restrict__ Linv)
{
    k_linv_init_body<T>(Dinv, n_pad, Linv, blockIdx.x, blockIdx.y);
}

template <typename Tin, typename Tout>
__global__ void k_cast(const Tin *__restrict__ in, int64_t count, Tout *__restrict__ out)
{
    k_cast_body<Tin, Tout>(in, count, out, blockIdx.x, blockIdx.y);
}

// The column band [c0, c1) of a block lower triangular n_pad x n_pad matrix in another type,
// with the blocks above the block diagonal written as zeros (they are not read).
template <typename Tin, typename Tout>
__global__ void k_cast_cols(const Tin *__restrict__ in, int n_pad, int c0, int c1, Tout *__restrict__ out)
{
    const int w = c1 - c0;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)n_pad * w) return;
    const int i = (int)(t / w), j = c0 + (int)(t % w);
    const int64_t o = (int64_t)i * n_pad + j;
    out[o] = j / NB > i / NB ? Tout(0) : convert_to<Tout>((double)in[o]);
}

// Linv's start for the inverse in two halves: part 1 writes every element except the diagonal
// blocks from b_split on (zeros, and the inverses of blocks 0 .. b_split - 1 from Dinv); part 2
// writes those remaining diagonal blocks.
template <typename T>
__global__ void k_linv_init_part(const double *__restrict__ Dinv, int n_pad, T *__restrict__ Linv, int b_split, int part)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (part == 2) {
        const int64_t per = (int64_t)NB * NB;
        if (t >= (int64_t)(n_pad / NB - b_split) * per) return;
        const int b = b_split + (int)(t / per), r = (int)(t % per / NB), c = (int)(t % NB);
        Linv[(int64_t)(b * NB + r) * n_pad + b * NB + c] = (T)Dinv[b * per + r * NB + c];
        return;
    }
    if (t >= (int64_t)n_pad * n_pad) return;
    const int i = (int)(t / n_pad), j = (int)(t % n_pad), b = i / NB;
    if (b == j / NB) {
        if (b >= b_split) return;
        Linv[t] = (T)Dinv[(int64_t)b * NB * NB + (i % NB) * NB + (j % NB)];
    } else {
        Linv[t] = T(0);
    }
}

__global__ void k_split_bf16(const float *__restrict__ in, int64_t count, __nv_bfloat16 *__restrict__ hi,
                             __nv_bfloat16 *__restrict__ lo)
{
    k_split_bf16_body(in, count, hi, lo, blockIdx.x, blockIdx.y);
}

__global__ void k_zero_pad_rows(uint16_t *__restrict__ A, int n, int n_pad)
{
    k_zero_pad_rows_body(A, n, n_pad, blockIdx.x, blockIdx.y);
}

__global__ void __launch_bounds__(1024) k_standardize(const double *__restrict__ y, int n, double *__restrict__ ys,
                                                      double *__restrict__ tau)
{
    k_standardize_body(y, n, ys, tau, blockIdx.x, blockIdx.y);
}

// Bottom-up block recursion: at level l the runs of 2^l diagonal blocks are inverted; runs
// 2j and 2j+1 merge by X21 = -X22 (L21 X11).  Ls is L in the working type T.  Every level's
// problem list goes to the device in one copy up front, so no host sync sits between levels.
static void trtri_plan(int n_pad, std::vector<GemmProb> &probs, std::vector<int> &level_first,
                       std::vector<int> &level_count, std::vector<int2> &level_maxmn)
{
    const int nblk = n_pad / NB;
    probs.clear();
    level_first.clear();
    level_count.clear();
    level_maxmn.clear();
    for (int run = 1; run < nblk; run *= 2) {
        const int first = (int)probs.size();
        int maxm = 0, maxn = 0;
        for (int b0 = 0; b0 + run < nblk; b0 += 2 * run) {
            const int r0 = (b0 + run) * NB;
            const int sl = run * NB;
            const int sr = std::min(run, nblk - b0 - run) * NB;
            GemmProb p;                                           // T = L21 X11
            p.a_off = (int64_t)r0 * n_pad + (int64_t)b0 * NB;
            p.b_off = (int64_t)b0 * NB * n_pad + (int64_t)b0 * NB;
            p.c_off = (int64_t)r0 * n_pad + (int64_t)b0 * NB;
            p.m = sr;
            p.n = sl;
            p.k = sl;
            p.ld = n_pad;
            probs.push_back(p);
            maxm = std::max(maxm, sr);
            maxn = std::max(maxn, sl);
        }
        const int cnt = (int)probs.size() - first;
        for (int q = 0; q < cnt; ++q) {                           // X21 = -X22 T
            GemmProb p = probs[first + q];
            const int64_t r0 = p.a_off / n_pad;
            p.b_off = p.c_off;
            p.a_off = r0 * n_pad + r0;
            p.k = p.m;
            probs.push_back(p);
        }
        level_first.push_back(first);
        level_count.push_back(cnt);
        level_maxmn.push_back(make_int2(maxm, maxn));
    }
}

// Levels of at least TRTRI_TC_MIN columns run on the tensor cores: slice products at FP64
// accuracy for the FP64 inverse (7 slices), at FP32 accuracy for the FP32 one (3 slices); the
// small levels on the FP64 / FP32 pipes.  128 measured 0.2 ms faster than 256 for the FP64
// inverse at n = 4096 and the same for the FP32 one.
constexpr int TRTRI_TC_MIN = 128;
// The FP32 inverse takes the tensor-core levels only in models that also take the tensor-core
// Cholesky updates (n_pad >= CHOL_TC_MIN_NPAD): below that size this path runs the batched
// path's CUDA-core arithmetic throughout, and the two agree bit for bit.
static int trtri_tc_min(int n_pad, bool f64)
{
    return f64 || n_pad >= CHOL_TC_MIN_NPAD ? TRTRI_TC_MIN : 1 << 30;
}

// Scratch of the tensor-core levels (the largest level's).
static size_t trtri_tc_scratch(int n_pad, bool f64)
{
    std::vector<GemmProb> probs;
    std::vector<int> first, count;
    std::vector<int2> mm;
    trtri_plan(n_pad, probs, first, count, mm);
    size_t b = 0;
    for (size_t l = 0; l < first.size(); ++l)
        if (mm[l].y >= trtri_tc_min(n_pad, f64)) {
            const int mk = std::max(mm[l].x, mm[l].y);
            b = std::max(b, f64 ? dtc_scratch_bytes(count[l], mk, mm[l].y) : stc_scratch_bytes(count[l], mk, mm[l].y));
        }
    return b;
}

// part 0: every level on stream s.  With n_pad / NB a power of two, part 1 takes the pairs
// inside the leading half (rows < n_pad / 2) and the top level's T = L21 X11, which need only
// the leading half of L (final once block column n_pad / (2 NB) - 1 is), and part 2 the rest:
// the trailing half's pairs and the top level's X21 = -X22 T.  The parts write disjoint
// regions of tmp and Linv, and each problem gets the arithmetic it gets in part 0.
template <typename T>
static int trtri_levels(gpbo_ctx *ctx, cudaStream_t s, const T *Ls, T *Linv, T *tmp, int n_pad, GemmProb *probs_dev,
                        void *tc_scratch = nullptr, int part = 0)
{
    std::vector<GemmProb> plan;
    std::vector<int> first0, count0;
    std::vector<int2> mm;
    trtri_plan(n_pad, plan, first0, count0, mm);
    if (plan.empty()) return GPBO_OK;
    // each level's problems for this part: its T = L21 X11 products, then its X21 = -X22 T
    const int64_t half = n_pad / 2;
    std::vector<GemmProb> probs;
    std::vector<int> first(first0.size()), count(first0.size()), count2(first0.size());
    for (size_t l = 0; l < first0.size(); ++l) {
        std::vector<GemmProb> g1, g2;
        for (int q = 0; q < count0[l]; ++q) {
            const GemmProb &p1 = plan[first0[l] + q], &p2 = plan[first0[l] + count0[l] + q];
            const int64_t r0 = p1.c_off / n_pad;                // first row of the pair's lower block
            const bool lead = r0 + p1.m <= half;                // the pair lies in the leading half
            const bool top = r0 == half && p1.c_off % n_pad == 0 && (int64_t)p1.n == half;
            if (part == 0 || (part == 1) == (lead || top)) g1.push_back(p1);
            if (part == 0 || (part == 1) == lead) g2.push_back(p2);
        }
        first[l] = (int)probs.size();
        count[l] = (int)g1.size();
        count2[l] = (int)g2.size();
        probs.insert(probs.end(), g1.begin(), g1.end());
        probs.insert(probs.end(), g2.begin(), g2.end());
    }
    if (probs.empty()) return GPBO_OK;
    // the host vector dies at return: copy synchronously with respect to it (pageable memory)
    GPBO_CUDA_TRY(cudaMemcpyAsync(probs_dev, probs.data(), sizeof(GemmProb) * probs.size(), cudaMemcpyHostToDevice, s));
    for (size_t l = 0; l < first.size(); ++l) {
        const int c1 = count[l], c2 = count2[l];
        const int f1 = first[l], f2 = first[l] + c1;
        if (std::is_same<T, double>::value && tc_scratch && mm[l].y >= TRTRI_TC_MIN) {
            // T = L21 X11 (X11 lower), then X21 = -X22 T (X22 lower)
            GPBO_TRY(dgemm_tc_level(ctx, s, (const double *)Ls, (const double *)Linv, (double *)tmp, n_pad,
                                    probs.data() + f1, c1, 1.0, 1, tc_scratch));
            GPBO_TRY(dgemm_tc_level(ctx, s, (const double *)Linv, (const double *)tmp, (double *)Linv, n_pad,
                                    probs.data() + f2, c2, -1.0, 2, tc_scratch));
            continue;
        }
        if (std::is_same<T, float>::value && tc_scratch && mm[l].y >= trtri_tc_min(n_pad, false)) {
            // FP32 accuracy from three slices: T = L21 X11 (X11 lower), then X21 = -X22 T
            GPBO_TRY(sgemm_tc_level(ctx, s, (const float *)Ls, (const float *)Linv, (float *)tmp, n_pad,
                                    probs.data() + f1, c1, 1.0, 1, tc_scratch));
            GPBO_TRY(sgemm_tc_level(ctx, s, (const float *)Linv, (const float *)tmp, (float *)Linv, n_pad,
                                    probs.data() + f2, c2, -1.0, 2, tc_scratch));
            continue;
        }
        if (std::is_same<T, float>::value && mm[l].y >= 128) {
            // large FP32 levels: 128 x 128 tiles (the batched step uses the same rule per level)
            if (c1) {
                dim3 grid((mm[l].y + 127) / 128, (mm[l].x + 127) / 128, c1);
                k_gemm128<<<grid, 256, 0, s>>>((const float *)Ls, (const float *)Linv, (float *)tmp, probs_dev + f1, 1.0f,
                                               0, 1);
                GPBO_LAUNCH_CHECK(ctx);
            }
            if (c2) {
                dim3 grid((mm[l].y + 127) / 128, (mm[l].x + 127) / 128, c2);
                k_gemm128<<<grid, 256, 0, s>>>((const float *)Linv, (const float *)tmp, (float *)Linv, probs_dev + f2,
                                               -1.0f, 1, 0);
                GPBO_LAUNCH_CHECK(ctx);
            }
            continue;
        }
        if (c1) {
            dim3 grid((mm[l].y + 63) / 64, (mm[l].x + 63) / 64, c1);
            k_gemm_batched<T><<<grid, 256, 0, s>>>(Ls, Linv, tmp, n_pad, n_pad, n_pad, probs_dev + f1, T(1), 0, 1);
            GPBO_LAUNCH_CHECK(ctx);
        }
        if (c2) {
            dim3 grid((mm[l].y + 63) / 64, (mm[l].x + 63) / 64, c2);
            k_gemm_batched<T><<<grid, 256, 0, s>>>(Linv, tmp, Linv, n_pad, n_pad, n_pad, probs_dev + f2, T(-1), 1, 0);
            GPBO_LAUNCH_CHECK(ctx);
        }
    }
    return GPBO_OK;
}

static unsigned blocks_for(int64_t count, int threads = 256) { return (unsigned)((count + threads - 1) / threads); }

// Solve K x = rhs with the factor: L z = rhs, then L^T x = z, each as one wavefront launch.
// sync: 2 nblk + 2 ints of scratch (flags and tickets of the two launches).
static int alpha_solve(gpbo_ctx *ctx, cudaStream_t st, const gp_model *m, const double *rhs, double *work,
                       double *out, int *sync)
{
    const int n_pad = m->n_pad, nblk = n_pad / NB;
    double *z = work + n_pad;
    GPBO_CUDA_TRY(cudaMemsetAsync(sync, 0, sizeof(int) * (2 * nblk + 2), st));
    k_fwd_wave<<<nblk, 256, 0, st>>>(m->L, m->Dinv, n_pad, rhs, z, sync, sync + 2 * nblk, ctx->dev_status);
    GPBO_LAUNCH_CHECK(ctx);
    k_bwd_wave<<<nblk, 256, 0, st>>>(m->L, m->Dinv, n_pad, z, out, sync + nblk, sync + 2 * nblk + 1,
                                     ctx->dev_status);
    GPBO_LAUNCH_CHECK(ctx);
    return GPBO_OK;
}

static int fit_model_on(gpbo_ctx *ctx, gp_model *m, const double *X_dev, const double *y_dev);

// The fit runs its main-stream work on an internal stream forked from the context's and joined
// back: its priority, between the factorisation chain's and that of the leading-half inverse
// (fit_model_on), lets the factorisation's own kernels take SMs ahead of the inverse's (FP64 fit
// at n = 4096: 8.77 -> 8.57 ms; at one priority the inverse's CTAs held SMs the updates waited
// for).  Everything inside enqueues on ctx->stream, which names that stream meanwhile.
int fit_model(gpbo_ctx *ctx, gp_model *m, const double *X_dev, const double *y_dev)
{
    cudaStream_t side = nullptr;
    GPBO_TRY(side_stream(ctx, &side));
    cudaStream_t user = ctx->stream;
    GPBO_CUDA_TRY(cudaEventRecord(ctx->side_ev[10], user));
    GPBO_CUDA_TRY(cudaStreamWaitEvent(ctx->mainf, ctx->side_ev[10], 0));
    ctx->stream = ctx->mainf;
    const int st = fit_model_on(ctx, m, X_dev, y_dev);
    ctx->stream = user;
    GPBO_CUDA_TRY(cudaEventRecord(ctx->side_ev[11], ctx->mainf));
    GPBO_CUDA_TRY(cudaStreamWaitEvent(user, ctx->side_ev[11], 0));
    return st;
}

static int fit_model_on(gpbo_ctx *ctx, gp_model *m, const double *X_dev, const double *y_dev)
{
    const int n = m->n, d = m->d, n_pad = m->n_pad, nblk = n_pad / NB;
    cudaStream_t st = ctx->stream;
    Lengthscales_inv ls;
    for (int k = 0; k < d; ++k) ls.inv[k] = 1.0 / m->ls[k];
    GPBO_TRY(trace_begin(ctx, PH_FACTOR, (double)n * n * n / 3.0));
    GPBO_CUDA_TRY(cudaMemcpyAsync(m->X, X_dev, sizeof(double) * n * d, cudaMemcpyDeviceToDevice, st));
    k_scale_x<<<blocks_for((int64_t)d * n_pad), 256, 0, st>>>(m->X, n, d, n_pad, ls, m->Xs64, m->Xs32);
    GPBO_LAUNCH_CHECK(ctx);
    if (m->Zsplit) GPBO_TRY(xkern_tc_prepare(ctx, m));
    {
        dim3 grid(n_pad / 32, n_pad / 32);
        if (m->xmax) {
            GPBO_CUDA_TRY(cudaMemsetAsync(m->xmax, 0, sizeof(unsigned long long), st));
            k_xs_max<<<blocks_for((int64_t)d * n_pad), 256, 0, st>>>(m->Xs64, (int64_t)d * n_pad, m->xmax);
            GPBO_LAUNCH_CHECK(ctx);
            k_kmat_fixed<<<grid, dim3(32, 8), 0, st>>>(m->Xs64, m->xmax, n, d, n_pad, m->s2, m->sn2, m->K, m->L);
        } else {
            k_kmat<<<grid, dim3(32, 8), 0, st>>>(m->Xs64, n, d, n_pad, m->s2, m->sn2, m->K);
        }
        GPBO_LAUNCH_CHECK(ctx);
    }
    // the factorisation works in L (k_kmat_fixed writes its lower triangle with K)
    if (!m->xmax) GPBO_CUDA_TRY(cudaMemcpyAsync(m->L, m->K, sizeof(double) * n_pad * n_pad, cudaMemcpyDeviceToDevice, st));
    const size_t smem2 = sizeof(double) * 2 * NB * (NB + 1), smem1 = sizeof(double) * NB * (NB + 1);
    // One workspace reservation, before any launch on the side streams, for the solve and the
    // inverse (they run concurrently).
    const int max_probs = 2 * nblk + 2;
    const int64_t sq = (int64_t)n_pad * n_pad;
    const size_t vec = sizeof(double) * n_pad;
    const bool f64 = m->prec == GPBO_PREC_F64;
    const size_t tc_bytes = n_pad >= 2 * trtri_tc_min(n_pad, f64) ? trtri_tc_scratch(n_pad, f64) : 0;
    const size_t inv_bytes = (m->prec == GPBO_PREC_F64 ? sizeof(double) * sq : sizeof(float) * 2 * sq) +
                             sizeof(GemmProb) * 2 * max_probs + tc_bytes + 256;
    const size_t sync_bytes = round_up64(sizeof(int) * (2 * (int64_t)nblk + 2), 256);
    const int chunks = (n_pad + TRMV_ROWS - 1) / TRMV_ROWS;
    void *wsp = nullptr;
    GPBO_TRY(ws_reserve(ctx, vec * (6 + chunks) + sync_bytes + inv_bytes, &wsp));
    double *ypad = (double *)wsp, *work = ypad + n_pad, *r = work + 2 * n_pad, *u = r + n_pad;
    double *part = ypad + 6 * (int64_t)n_pad;
    int *sync = (int *)((char *)wsp + vec * (6 + chunks));
    void *w2 = (void *)((char *)wsp + vec * (6 + chunks) + sync_bytes);

    // Right-looking blocked factorisation with a lookahead of one block column.  The chain that
    // every step waits on runs on the high-priority side stream and holds only 64 x 64 blocks:
    // the panel's first block row L_{kb+1,kb}, the update of diagonal block kb+1 by it, the
    // factorisation of that block and its inverse.  The main stream takes the rest of each
    // step: the panel's other block rows, the update of the rest of block column kb+1 (which
    // the next step's first panel row waits for), then the trailing update of block columns
    // kb+2 .. .  Each element gets the same arithmetic, in the same order, as in one launch per
    // part; the streams only reorder independent tiles.
    // Models of n_pad >= CHOL_TC_MIN_NPAD take latency-shaped kernels (smaller ones keep the
    // batched step's arithmetic, bit for bit): the first panel row by substitution against the
    // diagonal factor, so the chain no longer waits for the block's inverse, which runs on a
    // second side stream for the main stream's rows of the panel.
    const bool large = n_pad >= CHOL_TC_MIN_NPAD;
    cudaStream_t side = nullptr;
    GPBO_TRY(side_stream(ctx, &side));
    cudaStream_t side2 = ctx->side2;
    cudaEvent_t ev_fork = ctx->side_ev[0], ev_pf = ctx->side_ev[1], ev_rest = ctx->side_ev[2],
                ev_join = ctx->side_ev[3], ev_col = ctx->side_ev[5], ev_d = ctx->side_ev[6], ev_inv = ctx->side_ev[7];
    GPBO_CUDA_TRY(cudaEventRecord(ev_fork, st));
    GPBO_CUDA_TRY(cudaStreamWaitEvent(side, ev_fork, 0));
    k_chol_diag<<<1, DIAG_THREADS, smem1, side>>>(m->L, n_pad, 0, m->Dinv, ctx->dev_status);
    GPBO_LAUNCH_CHECK(ctx);
    auto inverse_on_side2 = [&](int jb) -> int {
        GPBO_CUDA_TRY(cudaEventRecord(ev_d, side));
        GPBO_CUDA_TRY(cudaStreamWaitEvent(side2, ev_d, 0));
        k_chol_inv<<<NB / INV_WARPS, 32 * INV_WARPS, 0, side2>>>(m->L, n_pad, jb, m->Dinv);
        GPBO_LAUNCH_CHECK(ctx);
        GPBO_CUDA_TRY(cudaEventRecord(ev_inv, side2));
        return GPBO_OK;
    };
    // The inverse L^-1 in two halves where n_pad / NB is a power of two (at least 4): once
    // block column nblk / 2 - 1 is final, the leading half of L is, and a third stream takes
    // the inverse's work that needs nothing else (the leading half's doubling levels and the
    // top level's T = L21 X11) under the factorisation's remaining steps.  Its kernels share
    // the SMs with the factorisation's (stream priority does not preempt), so they start where
    // that cost least as measured (fit times at n = 2048, 4096, 8192): the FP64 inverse, and the
    // FP32 one below 64 blocks, right after block column nblk / 2 - 1; the FP32 one from 64
    // blocks with an eighth of the factorisation left, where its steps leave most SMs idle.
    const bool split_inv = large && nblk >= 4 && (nblk & (nblk - 1)) == 0;
    const int lead_kb = !f64 && nblk >= 64 ? 7 * nblk / 8 - 1 : nblk / 2 - 1;
    cudaEvent_t ev_half = ctx->side_ev[8], ev_lead = ctx->side_ev[9];
    GemmProb *probs = nullptr;
    void *tcs = nullptr;
    double *tmp64 = nullptr;
    float *L32 = nullptr, *tmp32 = nullptr;
    if (f64) {
        tmp64 = (double *)w2;
        probs = (GemmProb *)(tmp64 + sq);
    } else {
        L32 = (float *)w2;
        tmp32 = L32 + sq;
        probs = (GemmProb *)(tmp32 + sq);
    }
    if (tc_bytes) tcs = (void *)(((uintptr_t)(probs + 2 * max_probs) + 255) & ~(uintptr_t)255);
    auto inverse_lead = [&]() -> int {
        cudaStream_t s3 = ctx->side3;
        const int hb = nblk / 2;
        GPBO_CUDA_TRY(cudaEventRecord(ev_half, st));
        GPBO_CUDA_TRY(cudaStreamWaitEvent(s3, ev_half, 0));
        if (f64) {
            k_linv_init_part<double><<<blocks_for(sq), 256, 0, s3>>>(m->Dinv, n_pad, m->Linv64, hb, 1);
            GPBO_LAUNCH_CHECK(ctx);
            GPBO_TRY(trtri_levels<double>(ctx, s3, m->L, m->Linv64, tmp64, n_pad, probs, tcs, 1));
        } else {
            k_cast_cols<double, float><<<blocks_for((int64_t)n_pad * hb * NB), 256, 0, s3>>>(m->L, n_pad, 0, hb * NB,
                                                                                             L32);
            GPBO_LAUNCH_CHECK(ctx);
            k_linv_init_part<float><<<blocks_for(sq), 256, 0, s3>>>(m->Dinv, n_pad, m->Linv32, hb, 1);
            GPBO_LAUNCH_CHECK(ctx);
            GPBO_TRY(trtri_levels<float>(ctx, s3, L32, m->Linv32, tmp32, n_pad, probs, tcs, 1));
        }
        GPBO_CUDA_TRY(cudaEventRecord(ev_lead, s3));
        return GPBO_OK;
    };
    if (large) GPBO_TRY(inverse_on_side2(0));
    else
        GPBO_TRY(launch_pdl(ctx, k_chol_inv, dim3(NB / INV_WARPS), dim3(32 * INV_WARPS), 0, side, m->L, n_pad, 0,
                            m->Dinv));
    // tensor-core trailing updates (FP64 accuracy by exact slice products) for large models
    alignas(64) unsigned char tc_maps[2][128];
    const bool tc = chol_tc_enabled(m);
    if (tc) GPBO_TRY(chol_tc_maps(m, tc_maps[0], tc_maps[1]));
    for (int kb = 0; kb + 1 < nblk; ++kb) {
        const int T = nblk - kb - 1;  // block rows below block kb
        // side: L_{kb+1,kb} (needs block column kb final: the main stream's step kb-1), then
        // diagonal block kb+1 (needs the main stream's trailing update of step kb-1)
        // (where the step before updated block column kb+1 on the tensor cores, ev_col and
        // ev_rest mark the same point: one wait, so the next two launches chain without a gap)
        const bool one_wait = kb > 0 && tc && n_pad >= CHOL_TC_MIN_NPAD && chol_tc_step(n_pad, nblk, kb - 1);
        if (kb > 0) GPBO_CUDA_TRY(cudaStreamWaitEvent(side, one_wait ? ev_rest : ev_col, 0));
        if (large)
            GPBO_TRY(launch_pdl(ctx, k_chol_panel_subst, dim3(NB / 4), dim3(128), 0, side, m->L, n_pad, kb, m->Dinv));
        else
            GPBO_TRY(launch_pdl(ctx, k_chol_panel, dim3(NB / 4), dim3(128), 0, side, m->L, n_pad, kb, m->Dinv, 0));
        GPBO_CUDA_TRY(cudaEventRecord(ev_pf, side));
        if (kb > 0 && !one_wait) GPBO_CUDA_TRY(cudaStreamWaitEvent(side, ev_rest, 0));
        if (large) {
            GPBO_TRY(launch_pdl(ctx, k_chol_update_diagblk, dim3(NB), dim3(128), 0, side, m->L, n_pad, kb));
        } else {
            k_chol_update_slab<<<NB / SLAB_ROWS, 256, 0, side>>>(m->L, n_pad, kb, 1, 0);
            GPBO_LAUNCH_CHECK(ctx);
        }
        GPBO_TRY(launch_pdl(ctx, k_chol_diag, dim3(1), dim3(DIAG_THREADS), smem1, side, m->L, n_pad, kb + 1, m->Dinv,
                            ctx->dev_status));
        if (!large)
            GPBO_TRY(launch_pdl(ctx, k_chol_inv, dim3(NB / INV_WARPS), dim3(32 * INV_WARPS), 0, side, m->L, n_pad,
                                kb + 1, m->Dinv));
        // main: the rest of panel kb and of block column kb+1, then block columns kb+2 ..; large
        // models take block column kb+1 into the tensor-core update of the step
        GPBO_CUDA_TRY(cudaStreamWaitEvent(st, ev_pf, 0));
        if (large) GPBO_CUDA_TRY(cudaStreamWaitEvent(st, ev_inv, 0));  // the inverse of block kb
        const bool tc_step = tc && chol_tc_step(n_pad, nblk, kb);
        const bool tc_col = tc_step && n_pad >= CHOL_TC_MIN_NPAD;
        if (T > 1) {
            if (large)
                k_chol_panel_row<<<(T - 1) * NB, 128, 0, st>>>(m->L, n_pad, kb, m->Dinv, 1);
            else
                k_chol_panel<<<(T - 1) * (NB / 4), 128, 0, st>>>(m->L, n_pad, kb, m->Dinv, 1);
            GPBO_LAUNCH_CHECK(ctx);
            if (split_inv && kb == lead_kb) GPBO_TRY(inverse_lead());  // block columns 0 .. nblk / 2 - 1 are final
            if (!tc_col) {
                k_chol_update_slab<<<(T - 1) * (NB / SLAB_ROWS), 256, 0, st>>>(m->L, n_pad, kb, 1, 1);
                GPBO_LAUNCH_CHECK(ctx);
            }
        }
        if (!tc_col) GPBO_CUDA_TRY(cudaEventRecord(ev_col, st));
        if (T > 1) {
            const int64_t tiles = (int64_t)T * (T - 1) / 2;
            GPBO_TRY(trace_begin(ctx, PH_CHOL_UPDATE, (double)tiles * 2.0 * NB * NB * NB));
            if (tc_step) {
                GPBO_TRY(chol_tc_update(ctx, m, kb, tc_col ? kb + 1 : kb + 2, st, tc_maps[0], tc_maps[1]));
            } else {
                if (tiles >= SLAB_BELOW * (int64_t)ctx->sm_count)
                    k_chol_update<<<(unsigned)tiles, 256, smem2, st>>>(m->L, n_pad, kb, nblk, 2);
                else
                    k_chol_update_slab<<<(unsigned)(tiles * (NB / SLAB_ROWS)), 256, 0, st>>>(m->L, n_pad, kb, 2, 0);
                GPBO_LAUNCH_CHECK(ctx);
            }
            GPBO_TRY(trace_end(ctx));
        }
        if (tc_col) GPBO_CUDA_TRY(cudaEventRecord(ev_col, st));
        GPBO_CUDA_TRY(cudaEventRecord(ev_rest, st));
        if (large) GPBO_TRY(inverse_on_side2(kb + 1));  // after the main stream's wait for block kb's
    }
    GPBO_CUDA_TRY(cudaEventRecord(ev_join, side));
    GPBO_CUDA_TRY(cudaStreamWaitEvent(st, ev_join, 0));
    if (large) GPBO_CUDA_TRY(cudaStreamWaitEvent(st, ev_inv, 0));
    k_zero_upper_blocks<<<blocks_for((int64_t)n_pad * n_pad), 256, 0, st>>>(m->L, n_pad);
    GPBO_LAUNCH_CHECK(ctx);
    GPBO_TRY(trace_end(ctx));
    GPBO_TRY(trace_begin(ctx, PH_INVERSE, (double)n * n * n / 3.0));
    // A pivot that was not positive is reported by the status check at the end (the factor
    // carries on with 1 in its place, so what follows stays finite): no host round trip here.


    // alpha = K^-1 y with one step of iterative refinement, on the side stream: the FP64 solve
    // (latency-bound substitutions, beside the L^-1 products on the main stream) and the FP64
    // residual r = y - K alpha; the correction K^-1 r = X^T (X r) then goes through X = L^-1
    // once it is ready (FP64 for FP64 models, FP32-accurate otherwise: mixed-precision
    // refinement, whose correction only needs the precision of the correction itself).
    GPBO_CUDA_TRY(cudaEventRecord(ev_fork, st));
    GPBO_CUDA_TRY(cudaStreamWaitEvent(side, ev_fork, 0));
    k_pad_copy<<<blocks_for(n_pad), 256, 0, side>>>(y_dev, n, n_pad, ypad);
    GPBO_LAUNCH_CHECK(ctx);
    GPBO_TRY(alpha_solve(ctx, side, m, ypad, work, m->alpha64, sync));
    k_residual<<<(n_pad + 7) / 8, 256, 0, side>>>(m->K, m->alpha64, ypad, n_pad, r);
    GPBO_LAUNCH_CHECK(ctx);
    cudaEvent_t ev_linv = ctx->side_ev[4];
    auto correction = [&](auto *X) -> int {
        using T = std::remove_const_t<std::remove_pointer_t<decltype(X)>>;
        GPBO_CUDA_TRY(cudaEventRecord(ev_linv, st));
        GPBO_CUDA_TRY(cudaStreamWaitEvent(side, ev_linv, 0));
        k_trmv<T><<<(n_pad + 7) / 8, 256, 0, side>>>(X, n_pad, r, u);
        GPBO_LAUNCH_CHECK(ctx);
        k_trmv_t_part<T><<<dim3(n_pad / 32, chunks), 256, 0, side>>>(X, n_pad, u, part);
        GPBO_LAUNCH_CHECK(ctx);
        k_trmv_t_sum<<<blocks_for(n_pad), 256, 0, side>>>(part, n_pad, chunks, m->alpha64, m->alpha32);
        GPBO_LAUNCH_CHECK(ctx);
        GPBO_CUDA_TRY(cudaEventRecord(ev_join, side));
        return GPBO_OK;
    };

    // L^-1 for scoring (the trailing half where the leading one ran under the factorisation:
    // its own problem list, so the two never share one)
    const int hb = nblk / 2;
    if (split_inv) GPBO_CUDA_TRY(cudaStreamWaitEvent(st, ev_lead, 0));
    if (m->prec == GPBO_PREC_F64) {
        if (split_inv) {
            k_linv_init_part<double><<<blocks_for((int64_t)(nblk - hb) * NB * NB), 256, 0, st>>>(m->Dinv, n_pad,
                                                                                                m->Linv64, hb, 2);
            GPBO_LAUNCH_CHECK(ctx);
            GPBO_TRY(trtri_levels<double>(ctx, st, m->L, m->Linv64, tmp64, n_pad, probs + max_probs, tcs, 2));
        } else {
            k_linv_init<double><<<blocks_for(sq), 256, 0, st>>>(m->Dinv, n_pad, m->Linv64);
            GPBO_LAUNCH_CHECK(ctx);
            GPBO_TRY(trtri_levels<double>(ctx, st, m->L, m->Linv64, tmp64, n_pad, probs, tcs));
        }
        GPBO_TRY(correction(m->Linv64));
    } else {
        if (split_inv) {
            k_cast_cols<double, float><<<blocks_for((int64_t)n_pad * (n_pad - hb * NB)), 256, 0, st>>>(
                m->L, n_pad, hb * NB, n_pad, L32);
            GPBO_LAUNCH_CHECK(ctx);
            k_linv_init_part<float><<<blocks_for((int64_t)(nblk - hb) * NB * NB), 256, 0, st>>>(m->Dinv, n_pad,
                                                                                               m->Linv32, hb, 2);
            GPBO_LAUNCH_CHECK(ctx);
            GPBO_TRY(trtri_levels<float>(ctx, st, L32, m->Linv32, tmp32, n_pad, probs + max_probs, tcs, 2));
        } else {
            k_cast<double, float><<<blocks_for(sq), 256, 0, st>>>(m->L, sq, L32);
            GPBO_LAUNCH_CHECK(ctx);
            k_linv_init<float><<<blocks_for(sq), 256, 0, st>>>(m->Dinv, n_pad, m->Linv32);
            GPBO_LAUNCH_CHECK(ctx);
            GPBO_TRY(trtri_levels<float>(ctx, st, L32, m->Linv32, tmp32, n_pad, probs, tcs));
        }
        GPBO_TRY(correction(m->Linv32));
        if (m->prec == GPBO_PREC_BF16) {
            __nv_bfloat16 *hi = (__nv_bfloat16 *)m->Linv16;
            k_split_bf16<<<blocks_for(sq), 256, 0, st>>>(m->Linv32, sq, hi, hi + sq);
            GPBO_LAUNCH_CHECK(ctx);
            if (n_pad > n) {
                for (int part = 0; part < 2; ++part) {
                    k_zero_pad_rows<<<blocks_for((int64_t)(n_pad - n) * n_pad), 256, 0, st>>>(
                        (uint16_t *)(hi + part * sq), n, n_pad);
                    GPBO_LAUNCH_CHECK(ctx);
                }
            }
        } else if (m->prec == GPBO_PREC_F16) {
            k_cast<float, __half><<<blocks_for(sq), 256, 0, st>>>(m->Linv32, sq, (__half *)m->Linv16);
            GPBO_LAUNCH_CHECK(ctx);
            if (n_pad > n) {
                k_zero_pad_rows<<<blocks_for((int64_t)(n_pad - n) * n_pad), 256, 0, st>>>((uint16_t *)m->Linv16, n,
                                                                                          n_pad);
                GPBO_LAUNCH_CHECK(ctx);
            }
        }
    }
    GPBO_CUDA_TRY(cudaStreamWaitEvent(st, ev_join, 0));
    GPBO_TRY(trace_end(ctx));
    unsigned bits = 0;
    GPBO_TRY(take_device_status(ctx, &bits));
    if (bits & DEV_NOTSPD) return GPBO_ENOTSPD;
    if (bits & DEV_TIMEOUT) return GPBO_ETIMEOUT;
    return GPBO_OK;
}

int standardize_dev(gpbo_ctx *ctx, const double *y, int n, double *ys, double *tau_dev)
{
    k_standardize<<<1, 1024, 0, ctx->stream>>>(y, n, ys, tau_dev);
    GPBO_LAUNCH_CHECK(ctx);
    return GPBO_OK;
}

void fit_set_smem_limits()
{
    const int smem2 = (int)(sizeof(double) * 2 * NB * (NB + 1));
    cudaFuncSetAttribute(k_chol_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, smem2);
    cudaFuncSetAttribute(k_chol_update, cudaFuncAttributeMaxDynamicSharedMemorySize, smem2);
}

// ------------------------------------------------------------------ FMA throughput probe
// Each thread runs 8 independent FMA chains; one store per thread keeps the work alive.
template <typename T>
__global__ void k_fma_probe(T *out, int iters, T a, T b)
{
    T x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = (T)(threadIdx.x + j);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
    T s = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

int probe_fma(gpbo_ctx *ctx, int kind, double *tflops)
{
    const int blocks = ctx->sm_count * 8, threads = 256;
    const int64_t n = (int64_t)blocks * threads;
    const int iters = kind == 0 ? 2000 : 40000;
    void *w = nullptr;
    GPBO_TRY(ws_reserve(ctx, sizeof(double) * n, &w));
    cudaEvent_t a, b;
    GPBO_CUDA_TRY(cudaEventCreate(&a));
    GPBO_CUDA_TRY(cudaEventCreate(&b));
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        GPBO_CUDA_TRY(cudaEventRecord(a, ctx->stream));
        if (kind == 0) k_fma_probe<double><<<blocks, threads, 0, ctx->stream>>>((double *)w, iters, 0.999, 1e-3);
        else k_fma_probe<float><<<blocks, threads, 0, ctx->stream>>>((float *)w, iters, 0.999f, 1e-3f);
        GPBO_LAUNCH_CHECK(ctx);
        GPBO_CUDA_TRY(cudaEventRecord(b, ctx->stream));
        GPBO_CUDA_TRY(cudaEventSynchronize(b));
        float ms = 0.f;
        GPBO_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
        if (ms < best) best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *tflops = 2.0 * 8.0 * iters * (double)n / (best * 1e-3) / 1e12;
    return GPBO_OK;
}

}  // namespace gpbo

