// Surrogate fit on the GPU (§III-A: the surrogate is retrained on every evaluated
// configuration; §IV-D: GP training costs O(N^3)).  Everything here is FP64 except the
// triangular inverse used by the FP32 and tensor-core scoring paths, which is formed in
// FP32 from the FP64 factor.
//
//   K      = s2 m(r) + sn2 I            k_kmat            (Matern-5/2 ARD)
//   K      = L L^T                      k_chol_*          (blocked, right-looking, NB = 64)
//   alpha  = L^-T L^-1 y, refined once  k_fwd_step/k_bwd_step/k_residual
//   L^-1                                k_gemm_batched    (level-by-level block recursion)
//
// Padding: n is padded to n_pad (a multiple of 64, or of 256 for tensor-core models).
// Padded rows/columns of K are the identity, so L and L^-1 are the identity there, the
// padded right-hand side is zero, and alpha is zero there.  No kernel needs a ragged tail.
#include "gpbo_internal.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <vector>

namespace gpbo {

// ------------------------------------------------------------------ inputs
// Xs64[k][i] = X[i][k] / l_k for i < n, 0 for padding; Xs32 is its FP32 rounding.
__global__ void k_scale_x(const double *__restrict__ X, int n, int d, int n_pad, Lengthscales_inv ls,
                          double *__restrict__ Xs64, float *__restrict__ Xs32)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)d * n_pad) return;
    int k = (int)(t / n_pad), i = (int)(t % n_pad);
    double v = i < n ? X[(int64_t)i * d + k] * ls.inv[k] : 0.0;
    Xs64[t] = v;
    if (Xs32) Xs32[t] = (float)v;
}

// K_ij = s2 m(r_ij) + sn2 [i == j] over the real block, identity on the padding.  Each
// thread of the lower half (i >= j, by 32 x 32 tiles) writes K_ij and its mirror K_ji.
__global__ void k_kmat(const double *__restrict__ Xs, int n, int d, int n_pad, double s2, double sn2,
                       double *__restrict__ K)
{
    const int tj = blockIdx.x, ti = blockIdx.y;
    if (tj > ti) return;
    __shared__ double tile[32][33];
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = ti * 32 + r, j = tj * 32 + threadIdx.x;
        double v;
        if (i < n && j < n) {
            double r2 = 0.0;
            for (int k = 0; k < d; ++k) {
                double t = Xs[(int64_t)k * n_pad + i] - Xs[(int64_t)k * n_pad + j];
                r2 = fma(t, t, r2);
            }
            v = s2 * matern52_r2(r2) + (i == j ? sn2 : 0.0);
        } else {
            v = i == j ? 1.0 : 0.0;
        }
        K[(int64_t)i * n_pad + j] = v;
        tile[r][threadIdx.x] = v;
    }
    if (ti == tj) return;
    __syncthreads();
    // mirror: K[j][i] for the transposed tile, coalesced along i
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int j = tj * 32 + r, i = ti * 32 + threadIdx.x;
        K[(int64_t)j * n_pad + i] = tile[threadIdx.x][r];
    }
}

// ------------------------------------------------------------------ Cholesky
// Diagonal block k: unblocked right-looking factorisation in shared memory, then the
// inverse of the factor (column j solves L x = e_j).  Writes L_kk (zeros above) and Dinv_k.
// Pivots use one reciprocal square root: L_jj = p * rsqrt(p), 1/L_jj = rsqrt(p), so the
// column scaling and the inverse multiply instead of divide.  The inverse gives each
// column four threads (a lane quad) that split every dot product and combine by shuffles.
__global__ void __launch_bounds__(256) k_chol_diag(double *__restrict__ A, int n_pad, int kb,
                                                   double *__restrict__ Dinv, unsigned *status)
{
    extern __shared__ double sm[];
    double(*a)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(sm);
    double(*inv)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(sm + NB * (NB + 1));
    __shared__ double rdiag[NB];
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)kb * NB * n_pad + (int64_t)kb * NB;
    for (int e = tid; e < NB * NB; e += blockDim.x) a[e / NB][e % NB] = A[base + (int64_t)(e / NB) * n_pad + e % NB];
    for (int j = 0; j < NB; ++j) {
        __syncthreads();
        if (tid == 0) {
            double p = a[j][j];
            if (!(p > 0.0)) {
                atomicOr(status, DEV_NOTSPD);
                p = 1.0;
            }
            const double r = rsqrt(p);
            a[j][j] = p * r;
            rdiag[j] = r;
        }
        __syncthreads();
        const double r = rdiag[j];
        for (int i = j + 1 + tid; i < NB; i += blockDim.x) a[i][j] *= r;
        __syncthreads();
        const int cnt = NB - 1 - j;
        for (int e = tid; e < cnt * cnt; e += blockDim.x) {
            int i = j + 1 + e / cnt, c = j + 1 + e % cnt;
            if (c <= i) a[i][c] = fma(-a[i][j], a[c][j], a[i][c]);
        }
    }
    __syncthreads();
    {
        const int j = tid >> 2, sub = tid & 3;
        const unsigned mask = 0xFu << (threadIdx.x & 28);
        for (int i = sub; i < j; i += 4) inv[i][j] = 0.0;
        if (sub == 0) inv[j][j] = rdiag[j];
        __syncwarp(mask);
        for (int i = j + 1; i < NB; ++i) {
            double s = 0.0;
            for (int t = j + sub; t < i; t += 4) s = fma(a[i][t], inv[t][j], s);
            s += __shfl_xor_sync(mask, s, 1);
            s += __shfl_xor_sync(mask, s, 2);
            if (sub == 0) inv[i][j] = -s * rdiag[i];
            __syncwarp(mask);
        }
    }
    __syncthreads();
    double *D = Dinv + (int64_t)kb * NB * NB;
    for (int e = tid; e < NB * NB; e += blockDim.x) {
        int i = e / NB, c = e % NB;
        A[base + (int64_t)i * n_pad + c] = c <= i ? a[i][c] : 0.0;
        D[e] = inv[i][c];
    }
}

// Panel: L_ik = A_ik L_kk^-T for the block rows i > k, one CTA per 16-row slab so that
// the short panels at the end of the factorisation still spread over many SMs.
__global__ void __launch_bounds__(256) k_chol_panel(double *__restrict__ A, int n_pad, int kb,
                                                    const double *__restrict__ Dinv)
{
    __shared__ double a[16][NB + 1];
    __shared__ double dv[NB][NB + 1];
    const int64_t row0 = (int64_t)(kb + 1) * NB + (int64_t)blockIdx.x * 16;
    const int tid = threadIdx.x, tx = tid % 64, ty = tid / 64;
    const double *D = Dinv + (int64_t)kb * NB * NB;
    for (int e = tid; e < 16 * NB; e += blockDim.x)
        a[e / NB][e % NB] = A[(row0 + e / NB) * n_pad + (int64_t)kb * NB + e % NB];
    for (int e = tid; e < NB * NB; e += blockDim.x) dv[e / NB][e % NB] = D[e];
    __syncthreads();
    // thread (ty, tx): rows ty, ty+4, ty+8, ty+12; column tx; L_kk^-T is lower, so t <= tx
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int t = 0; t <= tx; ++t) {
        const double y = dv[tx][t];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = fma(a[ty + 4 * u][t], y, acc[u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) A[(row0 + ty + 4 * u) * n_pad + (int64_t)kb * NB + tx] = acc[u];
}

// Trailing update of the lower tiles: A_ij -= L_ik L_jk^T for k < j <= i.
__global__ void __launch_bounds__(256) k_chol_update(double *__restrict__ A, int n_pad, int kb, int nblk)
{
    extern __shared__ double sm[];
    double(*li)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(sm);
    double(*lj)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(sm + NB * (NB + 1));
    const int64_t p = blockIdx.x;
    int ii = (int)((sqrt(8.0 * (double)p + 1.0) - 1.0) * 0.5);
    while ((int64_t)(ii + 1) * (ii + 2) / 2 <= p) ++ii;
    while ((int64_t)ii * (ii + 1) / 2 > p) --ii;
    const int jj = (int)(p - (int64_t)ii * (ii + 1) / 2);
    const int ib = kb + 1 + ii, jb = kb + 1 + jj;
    if (ib >= nblk || jb > ib) return;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int64_t bi = (int64_t)ib * NB * n_pad + (int64_t)kb * NB;
    const int64_t bj = (int64_t)jb * NB * n_pad + (int64_t)kb * NB;
    for (int e = tid; e < NB * NB; e += blockDim.x) {
        int r = e / NB, c = e % NB;
        li[r][c] = A[bi + (int64_t)r * n_pad + c];
        lj[r][c] = A[bj + (int64_t)r * n_pad + c];
    }
    __syncthreads();
    double acc[4][4] = {};
    for (int t = 0; t < NB; ++t) {
        double x[4], y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) { x[u] = li[ty + 16 * u][t]; y[u] = lj[tx + 16 * u][t]; }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fma(x[u], y[v], acc[u][v]);
    }
    const int64_t bo = (int64_t)ib * NB * n_pad + (int64_t)jb * NB;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) A[bo + (int64_t)(ty + 16 * u) * n_pad + tx + 16 * v] -= acc[u][v];
}

// Zero the strictly upper blocks (they still hold K after the in-place factorisation).
__global__ void k_zero_upper_blocks(double *__restrict__ A, int n_pad)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)n_pad * n_pad) return;
    int i = (int)(t / n_pad), j = (int)(t % n_pad);
    if (j / NB > i / NB) A[t] = 0.0;
}

// ------------------------------------------------------------------ triangular solves
// Forward step b of L z = w: z_b = Dinv_b w_b (every CTA recomputes it), CTA 0 stores it,
// and each CTA updates one later block of w: w_r -= L_rb z_b.
__global__ void __launch_bounds__(256) k_fwd_step(const double *__restrict__ L, const double *__restrict__ Dinv,
                                                  int n_pad, int b, double *__restrict__ w, double *__restrict__ z)
{
    __shared__ double wb[NB], zb[NB];
    __shared__ double D[NB][NB + 1];
    const int tid = threadIdx.x;
    const double *Db = Dinv + (int64_t)b * NB * NB;
    for (int e = tid; e < NB * NB; e += blockDim.x) D[e / NB][e % NB] = Db[e];
    if (tid < NB) wb[tid] = w[b * NB + tid];
    __syncthreads();
    {   // z_b = Dinv_b w_b: four threads per row
        const int r = tid >> 2, sub = tid & 3;
        double s = 0.0;
        for (int t = sub; t <= r; t += 4) s = fma(D[r][t], wb[t], s);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        if (sub == 0) {
            zb[r] = s;
            if (blockIdx.x == 0) z[b * NB + r] = s;
        }
    }
    __syncthreads();
    const int rb = b + 1 + blockIdx.x;
    if (rb * NB >= n_pad) return;
    const int row = rb * NB + (tid >> 2), part = tid & 3;
    const double *Lr = L + (int64_t)row * n_pad + (int64_t)b * NB + part * 16;
    double s = 0.0;
#pragma unroll
    for (int t = 0; t < 16; ++t) s = fma(Lr[t], zb[part * 16 + t], s);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    if (part == 0) w[row] -= s;
}

// Backward step b of L^T x = w: x_b = Dinv_b^T w_b; each CTA c < b updates w_c -= L_bc^T x_b.
__global__ void __launch_bounds__(256) k_bwd_step(const double *__restrict__ L, const double *__restrict__ Dinv,
                                                  int n_pad, int b, double *__restrict__ w, double *__restrict__ x)
{
    __shared__ double wb[NB], xb[NB], red[4][NB];
    __shared__ double D[NB][NB + 1];
    const int tid = threadIdx.x;
    const double *Db = Dinv + (int64_t)b * NB * NB;
    for (int e = tid; e < NB * NB; e += blockDim.x) D[e / NB][e % NB] = Db[e];
    if (tid < NB) wb[tid] = w[b * NB + tid];
    __syncthreads();
    {   // x_b = Dinv_b^T w_b: four threads per output
        const int r = tid >> 2, sub = tid & 3;
        double s = 0.0;
        for (int t = r + sub; t < NB; t += 4) s = fma(D[t][r], wb[t], s);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        if (sub == 0) {
            xb[r] = s;
            if (blockIdx.x == 0) x[b * NB + r] = s;
        }
    }
    __syncthreads();
    const int cb = blockIdx.x;
    if (cb >= b) return;
    const int col = tid & 63, part = tid >> 6;
    const double *Lb = L + (int64_t)(b * NB + part * 16) * n_pad + (int64_t)cb * NB + col;
    double s = 0.0;
#pragma unroll
    for (int t = 0; t < 16; ++t) s = fma(Lb[(int64_t)t * n_pad], xb[part * 16 + t], s);
    red[part][col] = s;
    __syncthreads();
    if (tid < NB) w[cb * NB + tid] -= red[0][tid] + red[1][tid] + red[2][tid] + red[3][tid];
}

// r = y - K alpha (one warp per row).
__global__ void k_residual(const double *__restrict__ K, const double *__restrict__ alpha,
                           const double *__restrict__ y, int n_pad, double *__restrict__ r)
{
    const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
    if (row >= n_pad) return;
    const double *Kr = K + (int64_t)row * n_pad;
    double s = 0.0;
    for (int j = lane; j < n_pad; j += 32) s = fma(Kr[j], alpha[j], s);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) r[row] = y[row] - s;
}

__global__ void k_axpy_cast(double *__restrict__ a, const double *__restrict__ dlt, int n, float *__restrict__ a32)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = dlt ? a[i] + dlt[i] : a[i];
    a[i] = v;
    if (a32) a32[i] = (float)v;
}

__global__ void k_pad_copy(const double *__restrict__ y, int n, int n_pad, double *__restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_pad) out[i] = i < n ? y[i] : 0.0;
}

// ------------------------------------------------------------------ triangular inverse
// Batched SIMT GEMM C = alpha * A * B on row-major tiles; each problem in `probs` has its own
// operand offsets and shape.  tri_a: A is lower triangular (skip k > row block end);
// tri_b: B is lower triangular (skip k < column block start).
struct GemmProb {
    int64_t a_off, b_off, c_off;
    int m, n, k;
};

template <typename T>
__global__ void __launch_bounds__(256) k_gemm_batched(const T *__restrict__ Abase, const T *__restrict__ Bbase,
                                                      T *__restrict__ Cbase, int lda, int ldb, int ldc,
                                                      const GemmProb *__restrict__ probs, T alpha, int tri_a,
                                                      int tri_b)
{
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    const GemmProb pr = probs[blockIdx.z];
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    if (m0 >= pr.m || n0 >= pr.n) return;
    const T *A = Abase + pr.a_off;
    const T *B = Bbase + pr.b_off;
    T *C = Cbase + pr.c_off;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    int kbeg = 0, kend = pr.k;
    if (tri_a) kend = min(kend, m0 + BM);
    if (tri_b) kbeg = (n0 / BK) * BK;
    T acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        for (int e = tid; e < BM * BK; e += 256) {
            int r = e / BK, c = e % BK;
            int gr = m0 + r, gc = k0 + c;
            As[c][r] = (gr < pr.m && gc < pr.k) ? A[(int64_t)gr * lda + gc] : T(0);
        }
        for (int e = tid; e < BK * BN; e += 256) {
            int r = e / BN, c = e % BN;
            int gr = k0 + r, gc = n0 + c;
            Bs[r][c] = (gr < pr.k && gc < pr.n) ? B[(int64_t)gr * ldb + gc] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < BK; ++t) {
            T x[4], y[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) { x[u] = As[t][ty + 16 * u]; y[u] = Bs[t][tx + 16 * u]; }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += x[u] * y[v];
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            int gr = m0 + ty + 16 * u, gc = n0 + tx + 16 * v;
            if (gr < pr.m && gc < pr.n) C[(int64_t)gr * ldc + gc] = alpha * acc[u][v];
        }
}

// Linv's diagonal blocks from Dinv (rounded to T); everything else zero.
template <typename T>
__global__ void k_linv_init(const double *__restrict__ Dinv, int n_pad, T *__restrict__ Linv)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)n_pad * n_pad) return;
    int i = (int)(t / n_pad), j = (int)(t % n_pad);
    T v = T(0);
    if (i / NB == j / NB) {
        int b = i / NB;
        v = (T)Dinv[(int64_t)b * NB * NB + (i % NB) * NB + (j % NB)];
    }
    Linv[t] = v;
}

template <typename T> __device__ __forceinline__ T convert_to(double v) { return (T)v; }
template <> __device__ __forceinline__ __nv_bfloat16 convert_to<__nv_bfloat16>(double v) { return __float2bfloat16_rn((float)v); }
template <> __device__ __forceinline__ __half convert_to<__half>(double v) { return __float2half_rn((float)v); }

template <typename Tin, typename Tout>
__global__ void k_cast(const Tin *__restrict__ in, int64_t count, Tout *__restrict__ out)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < count) out[t] = convert_to<Tout>((double)in[t]);
}

// BF16 operands with a compensated inverse: hi = bf16(L^-1), lo = bf16(L^-1 - hi).
__global__ void k_split_bf16(const float *__restrict__ in, int64_t count, __nv_bfloat16 *__restrict__ hi,
                             __nv_bfloat16 *__restrict__ lo)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= count) return;
    const float v = in[t];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[t] = h;
    lo[t] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// Zero rows n..n_pad-1 of a 16-bit L^-1 (count rows of width n_pad), so that the cross-kernel
// values of padded observations never reach the variance.
__global__ void k_zero_pad_rows(uint16_t *__restrict__ A, int n, int n_pad)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t cnt = (int64_t)(n_pad - n) * n_pad;
    if (t < cnt) A[(int64_t)n * n_pad + t] = 0;
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

template <typename T>
static int trtri_levels(gpbo_ctx *ctx, const T *Ls, T *Linv, T *tmp, int n_pad, GemmProb *probs_dev)
{
    std::vector<GemmProb> probs;
    std::vector<int> first, count;
    std::vector<int2> mm;
    trtri_plan(n_pad, probs, first, count, mm);
    if (probs.empty()) return GPBO_OK;
    // the host vector dies at return: copy synchronously with respect to it (pageable memory)
    GPBO_CUDA_TRY(cudaMemcpyAsync(probs_dev, probs.data(), sizeof(GemmProb) * probs.size(), cudaMemcpyHostToDevice,
                                  ctx->stream));
    for (size_t l = 0; l < first.size(); ++l) {
        dim3 grid((mm[l].y + 63) / 64, (mm[l].x + 63) / 64, count[l]);
        k_gemm_batched<T><<<grid, 256, 0, ctx->stream>>>(Ls, Linv, tmp, n_pad, n_pad, n_pad, probs_dev + first[l],
                                                         T(1), 0, 1);
        GPBO_LAUNCH_CHECK(ctx);
        k_gemm_batched<T><<<grid, 256, 0, ctx->stream>>>(Linv, tmp, Linv, n_pad, n_pad, n_pad,
                                                         probs_dev + first[l] + count[l], T(-1), 1, 0);
        GPBO_LAUNCH_CHECK(ctx);
    }
    return GPBO_OK;
}

static unsigned blocks_for(int64_t count, int threads = 256) { return (unsigned)((count + threads - 1) / threads); }

static int alpha_solve(gpbo_ctx *ctx, const gp_model *m, const double *rhs, double *work, double *out)
{
    const int n_pad = m->n_pad, nblk = n_pad / NB;
    GPBO_CUDA_TRY(cudaMemcpyAsync(work, rhs, sizeof(double) * n_pad, cudaMemcpyDeviceToDevice, ctx->stream));
    double *z = work + n_pad;
    for (int b = 0; b < nblk; ++b) {
        k_fwd_step<<<std::max(1, nblk - b - 1), 256, 0, ctx->stream>>>(m->L, m->Dinv, n_pad, b, work, z);
        GPBO_LAUNCH_CHECK(ctx);
    }
    for (int b = nblk - 1; b >= 0; --b) {
        k_bwd_step<<<std::max(1, b), 256, 0, ctx->stream>>>(m->L, m->Dinv, n_pad, b, z, out);
        GPBO_LAUNCH_CHECK(ctx);
    }
    return GPBO_OK;
}

int fit_model(gpbo_ctx *ctx, gp_model *m, const double *X_dev, const double *y_dev)
{
    const int n = m->n, d = m->d, n_pad = m->n_pad, nblk = n_pad / NB;
    cudaStream_t st = ctx->stream;
    Lengthscales_inv ls;
    for (int k = 0; k < d; ++k) ls.inv[k] = 1.0 / m->ls[k];
    GPBO_CUDA_TRY(cudaMemcpyAsync(m->X, X_dev, sizeof(double) * n * d, cudaMemcpyDeviceToDevice, st));
    k_scale_x<<<blocks_for((int64_t)d * n_pad), 256, 0, st>>>(m->X, n, d, n_pad, ls, m->Xs64, m->Xs32);
    GPBO_LAUNCH_CHECK(ctx);
    if (m->Zsplit) GPBO_TRY(xkern_tc_prepare(ctx, m));
    {
        dim3 grid(n_pad / 32, n_pad / 32);
        k_kmat<<<grid, dim3(32, 8), 0, st>>>(m->Xs64, n, d, n_pad, m->s2, m->sn2, m->K);
        GPBO_LAUNCH_CHECK(ctx);
    }
    GPBO_CUDA_TRY(cudaMemcpyAsync(m->L, m->K, sizeof(double) * n_pad * n_pad, cudaMemcpyDeviceToDevice, st));
    const size_t smem2 = sizeof(double) * 2 * NB * (NB + 1);
    for (int kb = 0; kb < nblk; ++kb) {
        k_chol_diag<<<1, 256, smem2, st>>>(m->L, n_pad, kb, m->Dinv, ctx->dev_status);
        GPBO_LAUNCH_CHECK(ctx);
        const int T = nblk - kb - 1;
        if (T > 0) {
            k_chol_panel<<<T * (NB / 16), 256, 0, st>>>(m->L, n_pad, kb, m->Dinv);
            GPBO_LAUNCH_CHECK(ctx);
            const int64_t tiles = (int64_t)T * (T + 1) / 2;
            GPBO_TRY(trace_begin(ctx, PH_CHOL_UPDATE, (double)tiles * 2.0 * NB * NB * NB));
            k_chol_update<<<(unsigned)tiles, 256, smem2, st>>>(m->L, n_pad, kb, nblk);
            GPBO_LAUNCH_CHECK(ctx);
            GPBO_TRY(trace_end(ctx));
        }
    }
    k_zero_upper_blocks<<<blocks_for((int64_t)n_pad * n_pad), 256, 0, st>>>(m->L, n_pad);
    GPBO_LAUNCH_CHECK(ctx);
    unsigned bits = 0;
    GPBO_TRY(take_device_status(ctx, &bits));
    if (bits & DEV_NOTSPD) return GPBO_ENOTSPD;

    // alpha = K^-1 y with one refinement step (FP64 throughout)
    void *wsp = nullptr;
    const size_t vec = sizeof(double) * n_pad;
    GPBO_TRY(ws_reserve(ctx, vec * 6, &wsp));
    double *ypad = (double *)wsp, *work = ypad + n_pad, *r = work + 2 * n_pad, *dlt = r + n_pad;
    k_pad_copy<<<blocks_for(n_pad), 256, 0, st>>>(y_dev, n, n_pad, ypad);
    GPBO_LAUNCH_CHECK(ctx);
    GPBO_TRY(alpha_solve(ctx, m, ypad, work, m->alpha64));
    k_residual<<<(n_pad + 7) / 8, 256, 0, st>>>(m->K, m->alpha64, ypad, n_pad, r);
    GPBO_LAUNCH_CHECK(ctx);
    GPBO_TRY(alpha_solve(ctx, m, r, work, dlt));
    k_axpy_cast<<<blocks_for(n_pad), 256, 0, st>>>(m->alpha64, dlt, n_pad, m->alpha32);
    GPBO_LAUNCH_CHECK(ctx);

    // L^-1 for scoring
    const int max_probs = 2 * nblk + 2;
    GemmProb *probs = nullptr;
    const int64_t sq = (int64_t)n_pad * n_pad;
    if (m->prec == GPBO_PREC_F64) {
        void *w2 = nullptr;
        GPBO_TRY(ws_reserve(ctx, sizeof(double) * sq + sizeof(GemmProb) * 2 * max_probs, &w2));
        double *tmp = (double *)w2;
        probs = (GemmProb *)(tmp + sq);
        k_linv_init<double><<<blocks_for(sq), 256, 0, st>>>(m->Dinv, n_pad, m->Linv64);
        GPBO_LAUNCH_CHECK(ctx);
        GPBO_TRY(trtri_levels<double>(ctx, m->L, m->Linv64, tmp, n_pad, probs));
    } else {
        void *w2 = nullptr;
        GPBO_TRY(ws_reserve(ctx, sizeof(float) * 2 * sq + sizeof(GemmProb) * 2 * max_probs, &w2));
        float *L32 = (float *)w2, *tmp = L32 + sq;
        probs = (GemmProb *)(tmp + sq);
        k_cast<double, float><<<blocks_for(sq), 256, 0, st>>>(m->L, sq, L32);
        GPBO_LAUNCH_CHECK(ctx);
        k_linv_init<float><<<blocks_for(sq), 256, 0, st>>>(m->Dinv, n_pad, m->Linv32);
        GPBO_LAUNCH_CHECK(ctx);
        GPBO_TRY(trtri_levels<float>(ctx, L32, m->Linv32, tmp, n_pad, probs));
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
    GPBO_TRY(take_device_status(ctx, &bits));
    if (bits & DEV_NOTSPD) return GPBO_ENOTSPD;
    return GPBO_OK;
}

// ------------------------------------------------------------------ standardisation
// ys = (y - mean) / std (population std; 1 when zero), tau = min ys.  One CTA.
__global__ void __launch_bounds__(1024) k_standardize(const double *__restrict__ y, int n, double *__restrict__ ys,
                                                      double *__restrict__ tau)
{
    __shared__ double red[32];
    __shared__ double bc;
    const int tid = threadIdx.x, lane = tid % 32, wid = tid / 32;
    auto block_sum = [&](double v) {
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[wid] = v;
        __syncthreads();
        if (wid == 0) {
            v = lane < (int)(blockDim.x / 32) ? red[lane] : 0.0;
            for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) bc = v;
        }
        __syncthreads();
        double r = bc;
        __syncthreads();
        return r;
    };
    double s = 0.0;
    for (int i = tid; i < n; i += blockDim.x) s += y[i];
    const double mean = block_sum(s) / n;
    double v = 0.0;
    for (int i = tid; i < n; i += blockDim.x) v += (y[i] - mean) * (y[i] - mean);
    double sd = sqrt(block_sum(v) / n);
    if (!(sd > 0.0)) sd = 1.0;
    double mn = INFINITY;
    for (int i = tid; i < n; i += blockDim.x) {
        double t = (y[i] - mean) / sd;
        ys[i] = t;
        mn = fmin(mn, t);
    }
    for (int o = 16; o; o >>= 1) mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    if (lane == 0) red[wid] = mn;
    __syncthreads();
    if (tid == 0) {
        double m = red[0];
        for (int w = 1; w < (int)(blockDim.x / 32); ++w) m = fmin(m, red[w]);
        *tau = m;
    }
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

