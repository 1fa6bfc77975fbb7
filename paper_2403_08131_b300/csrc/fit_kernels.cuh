// Device bodies of the fit kernels, shared by the single-problem kernels (fit.cu) and the
// batched kernels (batched.cu) so that both run identical arithmetic.  Each body takes its
// block coordinates as arguments instead of reading blockIdx.
#pragma once

#include "gpbo_internal.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace gpbo {


// ------------------------------------------------------------------ inputs
// Xs64[k][i] = X[i][k] / l_k for i < n, 0 for padding; Xs32 is its FP32 rounding.
__device__ __forceinline__ void k_scale_x_body(const double *__restrict__ X, int n, int d, int n_pad, Lengthscales_inv ls,
                          double *__restrict__ Xs64, float *__restrict__ Xs32, const int bx, const int by)
{
    int64_t t = bx * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)d * n_pad) return;
    int k = (int)(t / n_pad), i = (int)(t % n_pad);
    double v = i < n ? X[(int64_t)i * d + k] * ls.inv[k] : 0.0;
    Xs64[t] = v;
    if (Xs32) Xs32[t] = (float)v;
}

// K_ij = s2 m(r_ij) + sn2 [i == j] over the real block, identity on the padding.  Each
// thread of the lower half (i >= j, by 32 x 32 tiles) writes K_ij and its mirror K_ji.
__device__ __forceinline__ void k_kmat_body(const double *__restrict__ Xs, int n, int d, int n_pad, double s2, double sn2,
                       double *__restrict__ K, const int bx, const int by)
{
    const int tj = bx, ti = by;
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
// Diagonal block kb: factor the 64x64 block in place, right-looking, column by column.
// Pass j applies the rank-1 update with column j of L (already scaled by 1 / L_jj) to the
// trailing lower triangle of the block, a_ic -= l_ij l_cj (j < c <= i), enumerated from a
// column-major table so that every lane of the worker warps has an element.  Warp 0 meanwhile
// finishes a_{j+1,j+1} and takes the next pivot, L_{j+1,j+1} = p rsqrt(p) with
// 1 / L_{j+1,j+1} = rsqrt(p), and publishes it through a shared flag: the pivot chain (on this
// part an FP64 rsqrt alone takes about 440 cycles) runs beside the updates instead of after
// them.  The elements of column j+1 come last in the range: their owners wait (bounded) for
// the flag and store them scaled, so one barrier per column suffices.  The factor's arithmetic
// per element is that of a plain right-looking loop.  The reciprocal pivots go to the diagonal
// of Dinv_kb; k_chol_inv builds the rest of the inverse for the panel.
constexpr int DIAG_TRI = NB * (NB + 1) / 2;

// The factorisation of one 64 x 64 diagonal block held in shared memory (a: the block, rows of
// NB + 1 doubles; tab: DIAG_TRI entries of scratch; rdiag: NB doubles; ready: one int), by the
// CTA's threads (a multiple of 128).  On return (after a barrier) a holds L_kk in its lower
// triangle and rdiag the reciprocal pivots.
__device__ __forceinline__ void chol_diag_factor_smem(double (*a)[NB + 1], uint16_t *tab, double *rdiag, int *ready_p,
                                                      unsigned *status)
{
    constexpr int TRI = DIAG_TRI;
    int &ready = *ready_p;         // highest column whose pivot is published
    const int tid = threadIdx.x;
    auto coff = [](int c) { return c * NB - c * (c - 1) / 2; };  // first entry of column c
    for (int e = tid; e < TRI; e += blockDim.x) {
        // column c: the largest with coff(c) <= e (closed form, then exact integer fix-up)
        int c = (int)((129.0f - sqrtf(16641.0f - 8.0f * (float)e)) * 0.5f);
        c = max(0, min(NB - 1, c));
        while (c > 0 && coff(c) > e) --c;
        while (c < NB - 1 && coff(c + 1) <= e) ++c;
        tab[e] = (uint16_t)((c + (e - coff(c))) | (c << 8));
    }
    __syncthreads();
    if (tid == 0) {
        double p = a[0][0];
        if (!(p > 0.0)) {
            atomicOr(status, DEV_NOTSPD);
            p = 1.0;
        }
        const double r = rsqrt(p);
        a[0][0] = p * r;
        rdiag[0] = r;
        ready = 0;
    }
    __syncthreads();
    if (tid > 0 && tid < NB) a[tid][0] *= rdiag[0];
    __syncthreads();
    volatile int *vready = &ready;
    volatile double *vrdiag = rdiag;
    for (int j = 0; j + 1 < NB; ++j) {
        const int m = NB - 1 - j;           // rows below j
        const int nF = TRI - coff(j + 2);   // triangle, columns >= j+2
        if (tid == 0) {
            double p = fma(-a[j + 1][j], a[j + 1][j], a[j + 1][j + 1]);
            if (!(p > 0.0)) {
                atomicOr(status, DEV_NOTSPD);
                p = 1.0;
            }
            const double rr = rsqrt(p);
            a[j + 1][j + 1] = p * rr;
            vrdiag[j + 1] = rr;
            __threadfence_block();
            *vready = j + 1;
        }
        // workers: the warps on schedulers 1-3, so that the pivot's FP64 instructions have
        // scheduler 0's FP64 unit to themselves (each FP64 warp instruction holds it 64 cycles)
        // Each worker thread takes at most one element of column j+1 below its diagonal (final
        // after this pass: updated now, stored scaled once the pivot is published) and elements
        // e, e + W, ... of the trailing triangle, four independent ones per pass so that the
        // shared-memory loads and FMAs of a warp overlap (each FP64 warp instruction holds its
        // scheduler's FP64 unit 64 cycles: the passes keep that unit, not latency, the limit).
        const int warp = tid >> 5, nw = (int)(blockDim.x >> 5), workers = nw - (nw + 3) / 4;
        const int wid = warp - warp / 4 - 1;
        if ((warp & 3) != 0) {
            const int W = workers * 32, w0 = wid * 32 + (tid & 31);
            const uint16_t *tj = tab + coff(j + 2);
            const bool has_col = w0 < m - 1;
            double vcol = 0.0;
            if (has_col) vcol = fma(-a[j + 2 + w0][j], a[j + 1][j], a[j + 2 + w0][j + 1]);
            int e = w0;
            for (; e + 3 * W < nF; e += 4 * W) {
                int ii[4], cc[4];
                double v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int t = tj[e + u * W];
                    ii[u] = t & 255;
                    cc[u] = t >> 8;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = fma(-a[ii[u]][j], a[cc[u]][j], a[ii[u]][cc[u]]);
#pragma unroll
                for (int u = 0; u < 4; ++u) a[ii[u]][cc[u]] = v[u];
            }
            for (; e < nF; e += W) {
                const int t = tj[e], i = t & 255, c = t >> 8;
                a[i][c] = fma(-a[i][j], a[c][j], a[i][c]);
            }
            if (has_col) {
                for (int it = 0; *vready < j + 1; ++it) {
                    if (it == (1 << 24)) {  // cannot happen: warp 0 publishes unconditionally
                        atomicOr(status, DEV_TIMEOUT);
                        break;
                    }
                }
                __threadfence_block();
                a[j + 2 + w0][j + 1] = vcol * vrdiag[j + 1];
            }
        }
        __syncthreads();
    }
}

// Diagonal block kb of A (global): load, factor (chol_diag_factor_smem), store L_kk with zeros
// above its diagonal and the reciprocal pivots on Dinv_kb's diagonal.
__device__ __forceinline__ void k_chol_diag_body(double *__restrict__ A, int n_pad, int kb,
                                                   double *__restrict__ Dinv, unsigned *status, const int bx, const int by)
{
    extern __shared__ double sm[];
    double(*a)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(sm);
    __shared__ double rdiag[NB];
    __shared__ uint16_t tab[DIAG_TRI];  // lower triangle, column-major: row | col << 8
    __shared__ int ready;
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)kb * NB * n_pad + (int64_t)kb * NB;
    for (int e = tid; e < NB * NB; e += blockDim.x) {
        const int r = e / NB, c = e % NB;
        a[r][c] = A[base + (int64_t)r * n_pad + c];
    }
    chol_diag_factor_smem(a, tab, rdiag, &ready, status);
    double *D = Dinv + (int64_t)kb * NB * NB;
    for (int e = tid; e < NB * NB; e += blockDim.x) {
        const int i = e / NB, c = e % NB;
        A[base + (int64_t)i * n_pad + c] = c <= i ? a[i][c] : 0.0;
    }
    if (tid < NB) D[tid * NB + tid] = rdiag[tid];
}

// Inverse X = L_kk^-1 of diagonal block kb (after k_chol_diag_body), by forward substitution of
// the unit columns, one warp per column (CTA bx: columns W bx .. W bx + W - 1 for W warps), lanes
// owning rows lane and lane + 32.  With rd_t = 1 / L_tt (the pivot's rsqrt, from Dinv's diagonal) and the
// scaled columns l'_it = l_it rd_t, the unscaled solution x~ takes x~_ic -= l'_it x~_tc for
// t = c .. i - 1, and X_ic = rd_i x~_ic: one shuffle and one or two FP64 FMAs per step (on this
// part every FP64 warp instruction holds its SMSP's FP64 unit for 64 cycles, so the step count
// of this chain is what the factorisation waits on).  Launch: 64 / W CTAs of 32 W threads.
// Column c of the inverse, by one warp, from the scaled block l (l_it rd_t below the diagonal,
// zero elsewhere) and the reciprocal pivots rd in shared memory; written to D (row-major 64 x 64).
__device__ __forceinline__ void chol_inv_column(const double (*l)[NB + 1], const double *rd, int c, int lane,
                                                double *__restrict__ D)
{
    double x0 = lane == c ? 1.0 : 0.0, x1 = lane + 32 == c ? 1.0 : 0.0;
    for (int t = c; t < NB; ++t) {
        const double v = __shfl_sync(0xffffffffu, t < 32 ? x0 : x1, t & 31);
        if (t < 31 && lane > t) x0 = fma(-l[lane][t], v, x0);
        if (lane + 32 > t) x1 = fma(-l[lane + 32][t], v, x1);
    }
    D[lane * NB + c] = x0 * rd[lane];   // zero above the diagonal (rows < c never change)
    D[(lane + 32) * NB + c] = x1 * rd[lane + 32];
}

__device__ __forceinline__ void k_chol_inv_body(const double *__restrict__ A, int n_pad, int kb,
                                                  double *__restrict__ Dinv, const int bx)
{
    __shared__ double l[NB][NB + 1];
    __shared__ double rd[NB];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = (int64_t)kb * NB * n_pad + (int64_t)kb * NB;
    double *D = Dinv + (int64_t)kb * NB * NB;
    for (int e = tid; e < NB; e += blockDim.x) rd[e] = D[e * NB + e];
    __syncthreads();
    for (int e = tid; e < NB * NB; e += blockDim.x) {
        const int i = e / NB, t = e % NB;
        l[i][t] = t < i ? A[base + (int64_t)i * n_pad + t] * rd[t] : 0.0;
    }
    __syncthreads();
    const int c = bx * (int)(blockDim.x >> 5) + warp;
    chol_inv_column(l, rd, c, lane, D);
}

// First block row of panel kb by substitution against L_kk (models of n_pad >= CHOL_TC_MIN_NPAD):
// row i of L_{kb+1,kb} solves x L_kk^T = A_{kb+1,kb}[i], by forward substitution with the
// column-scaled block (l'_it = l_it / l_tt, the inverse column's steps above: one shuffle and one
// or two FP64 FMAs per step), then x_t = x~_t / l_tt.  It needs only the factor of block kb, not
// its inverse, so the inverse leaves the factorisation's chain.  One warp per row; launch
// NB / W CTAs of 32 W threads.
__device__ __forceinline__ void k_chol_panel_subst_body(double *__restrict__ A, int n_pad, int kb,
                                                        const double *__restrict__ Dinv, const int bx)
{
    __shared__ double l[NB][NB + 1];
    __shared__ double rd[NB];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = (int64_t)kb * NB * n_pad + (int64_t)kb * NB;
    const double *D = Dinv + (int64_t)kb * NB * NB;
    for (int e = tid; e < NB; e += blockDim.x) rd[e] = D[e * NB + e];
    __syncthreads();
    for (int e = tid; e < NB * NB; e += blockDim.x) {
        const int i = e / NB, t = e % NB;
        l[i][t] = t < i ? A[base + (int64_t)i * n_pad + t] * rd[t] : 0.0;
    }
    __syncthreads();
    const int i = bx * (int)(blockDim.x >> 5) + warp;
    double *row = A + ((int64_t)(kb + 1) * NB + i) * n_pad + (int64_t)kb * NB;
    double x0 = row[lane], x1 = row[lane + 32];
    for (int t = 0; t < NB; ++t) {
        const double v = __shfl_sync(0xffffffffu, t < 32 ? x0 : x1, t & 31);
        if (lane > t) x0 = fma(-l[lane][t], v, x0);
        if (lane + 32 > t) x1 = fma(-l[lane + 32][t], v, x1);
    }
    row[lane] = x0 * rd[lane];
    row[lane + 32] = x1 * rd[lane + 32];
}

// Trailing update in slabs of SR rows (64 / SR CTAs per 64x64 tile), for launches too small to
// fill the GPU with whole tiles: on this part a CTA's FP64 work sets its latency, so short
// slabs keep the late, small updates short.  part 1: block column kb+1 from tile t0 on (CTA bx
// updates rows SR (bx % (64 / SR)) .. of block row kb+1+t0+bx/(64/SR)); part 2: block columns
// kb+2 .. (the tiles of k_chol_update part 2, in the same order).  Same per-element arithmetic
// as the full-tile update.
template <int SR>
__device__ __forceinline__ void k_chol_update_slab_body(double *__restrict__ A, int n_pad, int kb, const int bx,
                                                          int part = 1, int t0 = 0)
{
    constexpr int PER = NB / SR;
    __shared__ double li[SR][NB + 1];
    __shared__ double lj[NB][NB + 1];
    int ii = t0 + bx / PER, jj = 0;
    if (part == 2) {
        const int64_t p = bx / PER;
        ii = (int)((sqrt(8.0 * (double)p + 1.0) - 1.0) * 0.5);
        while ((int64_t)(ii + 1) * (ii + 2) / 2 <= p) ++ii;
        while ((int64_t)ii * (ii + 1) / 2 > p) --ii;
        jj = (int)(p - (int64_t)ii * (ii + 1) / 2);
        ++ii;
        ++jj;
    }
    const int ib = kb + 1 + ii, jb = kb + 1 + jj;
    const int64_t r0 = (int64_t)ib * NB + (bx % PER) * SR;
    const int tid = threadIdx.x, tx = tid % 64, ty = tid / 64;
    for (int e = tid; e < SR * NB; e += blockDim.x)
        li[e / NB][e % NB] = A[(r0 + e / NB) * n_pad + (int64_t)kb * NB + e % NB];
    for (int e = tid; e < NB * NB; e += blockDim.x)
        lj[e / NB][e % NB] = A[((int64_t)jb * NB + e / NB) * n_pad + (int64_t)kb * NB + e % NB];
    __syncthreads();
    double acc[SR / 4];
#pragma unroll
    for (int u = 0; u < SR / 4; ++u) acc[u] = 0.0;
    for (int t = 0; t < NB; ++t) {
        const double y = lj[tx][t];
#pragma unroll
        for (int u = 0; u < SR / 4; ++u) acc[u] = fma(li[ty + 4 * u][t], y, acc[u]);
    }
#pragma unroll
    for (int u = 0; u < SR / 4; ++u) A[(r0 + ty + 4 * u) * n_pad + (int64_t)jb * NB + tx] -= acc[u];
}

// Panel: L_ik = A_ik L_kk^-T for the block rows i > k, four rows per CTA of 128 threads, so that
// short panels still spread over many SMs.  Output column c is the triangular dot product
// sum_{t <= c} a_t Dinv[c][t] (L_kk^-T is lower); thread (row ty, lane tx) takes columns tx and
// 63 - tx in one loop of 65 steps -- every lane issues one FMA per step (a warp issues 65 FP64
// instructions per row instead of 96 when a lane takes one column) -- and each column keeps
// its t = 0 .. c accumulation order.  CTA bx takes rows 4 bx .. of block rows kb + 1 + boff ..
// (the factorisation launches the first block row, boff = 0, on its critical path and the
// rest, boff = 1, beside it).
// Output columns tx and 63 - tx of one panel row a (shared, NB values) times L_kk^-T, from the
// inverse dv (shared, rows of NB + 1), each column summed over t = 0 .. c in order.
__device__ __forceinline__ void chol_panel_pair(const double *a, const double (*dv)[NB + 1], int tx, double &out1,
                                                double &out2)
{
    const int c1 = tx, c2 = NB - 1 - tx;
    double acc = 0.0;
    out1 = 0.0;
    for (int s = 0; s <= NB; ++s) {
        const bool first = s <= c1;
        const int t = first ? s : s - c1 - 1, c = first ? c1 : c2;
        acc = fma(a[t], dv[c][t], acc);
        if (s == c1) {
            out1 = acc;
            acc = 0.0;
        }
    }
    out2 = acc;
}

__device__ __forceinline__ void k_chol_panel_body(double *__restrict__ A, int n_pad, int kb,
                                                    const double *__restrict__ Dinv, const int bx, const int by,
                                                    int boff = 0)
{
    __shared__ double a[4][NB + 1];
    __shared__ double dv[NB][NB + 1];
    const int64_t row0 = (int64_t)(kb + 1 + boff) * NB + (int64_t)bx * 4;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const double *D = Dinv + (int64_t)kb * NB * NB;
    for (int e = tid; e < 4 * NB; e += blockDim.x) a[e / NB][e % NB] = A[(row0 + e / NB) * n_pad + (int64_t)kb * NB + e % NB];
    for (int e = tid; e < NB * NB; e += blockDim.x) dv[e / NB][e % NB] = D[e];
    __syncthreads();
    double out1, out2;
    chol_panel_pair(a[ty], dv, tx, out1, out2);
    A[(row0 + ty) * n_pad + (int64_t)kb * NB + tx] = out1;
    A[(row0 + ty) * n_pad + (int64_t)kb * NB + NB - 1 - tx] = out2;
}

// The same two products for models with n_pad >= CHOL_TC_MIN_NPAD, shaped for latency: one CTA
// of 4 warps per output row, warp w summing t in [16 w, 16 w + 16) for two columns a lane, and the
// four partial sums added in a fixed order.  On this part every dependent FP64 operation costs
// a warp about 64 cycles, so the 64- and 65-term chains of the kernels above, not their FP64
// work, set the latency of the factorisation's 64 x 64 steps; here each chain is 16 terms and
// each row's work has an SM to itself.
// Panel row: L_{r,kb} = A_{r,kb} L_kk^-T (L_kk^-T from Dinv_kb, lower), row r = 64 (kb + 1 + boff) + blockIdx.x.
__device__ __forceinline__ void k_chol_panel_row_body(double *__restrict__ A, int n_pad, int kb,
                                                      const double *__restrict__ Dinv, int boff, const int bx)
{
    __shared__ double part[4][NB];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *ar = A + ((int64_t)(kb + 1 + boff) * NB + bx) * n_pad + (int64_t)kb * NB;
    const double *D = Dinv + (int64_t)kb * NB * NB;
    double x[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = ar[16 * w + k];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int c = lane + 32 * h;
        const double *dc = D + (int64_t)c * NB + 16 * w;
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (16 * w + k <= c) acc = fma(x[k], dc[k], acc);
        part[w][c] = acc;
    }
    __syncthreads();
    if (threadIdx.x < NB) {
        const int c = threadIdx.x;
        ar[c] = ((part[0][c] + part[1][c]) + part[2][c]) + part[3][c];
    }
}
// Diagonal block kb+1, lower triangle: A_{kb+1,kb+1} -= L_{kb+1,kb} L_{kb+1,kb}^T, row blockIdx.x.
__device__ __forceinline__ void k_chol_update_diagblk_body(double *__restrict__ A, int n_pad, int kb, const int r)
{
    __shared__ double part[4][NB];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t rowb = (int64_t)(kb + 1) * NB;
    const double *Pn = A + rowb * n_pad + (int64_t)kb * NB;  // panel rows of block kb+1
    double x[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = Pn[(int64_t)r * n_pad + 16 * w + k];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int c = lane + 32 * h;
        double acc = 0.0;
        if (c <= r) {
            const double *pc = Pn + (int64_t)c * n_pad + 16 * w;
#pragma unroll
            for (int k = 0; k < 16; ++k) acc = fma(x[k], pc[k], acc);
        }
        part[w][c] = acc;
    }
    __syncthreads();
    if (threadIdx.x <= r) {
        const int c = threadIdx.x;
        A[(rowb + r) * n_pad + rowb + c] -= ((part[0][c] + part[1][c]) + part[2][c]) + part[3][c];
    }
}

// Trailing update of the lower tiles: A_ij -= L_ik L_jk^T for k < j <= i.
// part 0: every tile of the trailing lower triangle (T(T+1)/2 CTAs, T = nblk - kb - 1);
// part 1: block column kb+1 only (T CTAs); part 2: block columns kb+2 .. (T(T-1)/2 CTAs).
__device__ __forceinline__ void k_chol_update_body(double *__restrict__ A, int n_pad, int kb, int nblk, const int bx, const int by,
                                                   int part = 0)
{
    extern __shared__ double sm[];
    double(*li)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(sm);
    double(*lj)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(sm + NB * (NB + 1));
    int ii = bx, jj = 0;
    if (part != 1) {
        const int64_t p = bx;
        ii = (int)((sqrt(8.0 * (double)p + 1.0) - 1.0) * 0.5);
        while ((int64_t)(ii + 1) * (ii + 2) / 2 <= p) ++ii;
        while ((int64_t)ii * (ii + 1) / 2 > p) --ii;
        jj = (int)(p - (int64_t)ii * (ii + 1) / 2);
        if (part == 2) { ++ii; ++jj; }
    }
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
__device__ __forceinline__ void k_zero_upper_blocks_body(double *__restrict__ A, int n_pad, const int bx, const int by)
{
    int64_t t = bx * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)n_pad * n_pad) return;
    int i = (int)(t / n_pad), j = (int)(t % n_pad);
    if (j / NB > i / NB) A[t] = 0.0;
}

// ------------------------------------------------------------------ triangular solves
// Forward step b of L z = w: z_b = Dinv_b w_b (every CTA recomputes it), CTA 0 stores it,
// and each CTA updates one later block of w: w_r -= L_rb z_b.
__device__ __forceinline__ void k_fwd_step_body(const double *__restrict__ L, const double *__restrict__ Dinv,
                                                  int n_pad, int b, double *__restrict__ w, double *__restrict__ z, const int bx, const int by)
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
            if (bx == 0) z[b * NB + r] = s;
        }
    }
    __syncthreads();
    const int rb = b + 1 + bx;
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
__device__ __forceinline__ void k_bwd_step_body(const double *__restrict__ L, const double *__restrict__ Dinv,
                                                  int n_pad, int b, double *__restrict__ w, double *__restrict__ x, const int bx, const int by)
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
            if (bx == 0) x[b * NB + r] = s;
        }
    }
    __syncthreads();
    const int cb = bx;
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

// Wavefront forms of the two substitutions: one launch each, one CTA per 64-row block, with
// the same arithmetic per element as the step kernels above (so the results are identical).
// A CTA takes its block from an atomic ticket in the order CTAs start, and only waits for
// blocks with smaller tickets, which have all started: no wait can depend on a CTA that is not
// running.  A finished block publishes its solution and then sets flags[block] = 1 (release:
// the solution's stores are fenced before the flag); a waiter spins on the flag (bounded),
// fences, and reads the solution past L1.  flags (nblk) and ticket must be zero at launch.
__device__ __forceinline__ bool wave_wait(const int *flag, unsigned *status)
{
    const long long t0 = clock64(), limit = wait_limit(status);
    for (long it = 0; *(volatile const int *)flag == 0; ++it)
        if ((it & 255) == 255 && clock64() - t0 > limit) {  // set the error and give up rather than hang
            atomicOr(status, DEV_TIMEOUT);
            return false;
        }
    __threadfence();
    return true;
}

// Forward: L z = w.  Ticket q handles block b = q; w is read once, z written.
__device__ __forceinline__ void k_fwd_wave_body(const double *__restrict__ L, const double *__restrict__ Dinv,
                                                int n_pad, const double *__restrict__ w, double *z, int *flags,
                                                int *ticket, unsigned *status)
{
    __shared__ double zp[NB], wb[NB];
    __shared__ double D[NB][NB + 1];
    __shared__ int sb;
    const int tid = threadIdx.x;
    if (tid == 0) sb = atomicAdd(ticket, 1);
    __syncthreads();
    const int b = sb;
    const double *Db = Dinv + (int64_t)b * NB * NB;
    for (int e = tid; e < NB * NB; e += blockDim.x) D[e / NB][e % NB] = Db[e];
    const int r = tid >> 2, part = tid & 3;
    const int64_t row = (int64_t)b * NB + r;
    double acc = w[row];
    for (int p = 0; p < b; ++p) {
        double lv[16];
        const double *Lr = L + row * n_pad + (int64_t)p * NB + part * 16;
#pragma unroll
        for (int t = 0; t < 16; ++t) lv[t] = Lr[t];
        if (tid == 0) wave_wait(flags + p, status);
        __syncthreads();
        if (tid < NB) zp[tid] = __ldcg(z + (int64_t)p * NB + tid);
        __syncthreads();
        double s = 0.0;
#pragma unroll
        for (int t = 0; t < 16; ++t) s = fma(lv[t], zp[part * 16 + t], s);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        acc -= s;
    }
    if (part == 0) wb[r] = acc;
    __syncthreads();
    double s = 0.0;
    for (int t = part; t <= r; t += 4) s = fma(D[r][t], wb[t], s);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    if (part == 0) {
        z[row] = s;
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) *(volatile int *)(flags + b) = 1;
}

// Backward: L^T x = w.  Ticket q handles block c = nblk - 1 - q.
__device__ __forceinline__ void k_bwd_wave_body(const double *__restrict__ L, const double *__restrict__ Dinv,
                                                int n_pad, const double *__restrict__ w, double *x, int *flags,
                                                int *ticket, unsigned *status)
{
    __shared__ double xp[NB], wb[NB], red[4][NB];
    __shared__ double D[NB][NB + 1];
    __shared__ int sb;
    const int tid = threadIdx.x, nblk = n_pad / NB;
    if (tid == 0) sb = atomicAdd(ticket, 1);
    __syncthreads();
    const int c = nblk - 1 - sb;
    const double *Dc = Dinv + (int64_t)c * NB * NB;
    for (int e = tid; e < NB * NB; e += blockDim.x) D[e / NB][e % NB] = Dc[e];
    const int col = tid & 63, part = tid >> 6;
    double acc = tid < NB ? w[(int64_t)c * NB + tid] : 0.0;
    for (int b = nblk - 1; b > c; --b) {
        double lv[16];
        const double *Lb = L + (int64_t)(b * NB + part * 16) * n_pad + (int64_t)c * NB + col;
#pragma unroll
        for (int t = 0; t < 16; ++t) lv[t] = Lb[(int64_t)t * n_pad];
        if (tid == 0) wave_wait(flags + b, status);
        __syncthreads();
        if (tid < NB) xp[tid] = __ldcg(x + (int64_t)b * NB + tid);
        __syncthreads();
        double s = 0.0;
#pragma unroll
        for (int t = 0; t < 16; ++t) s = fma(lv[t], xp[part * 16 + t], s);
        red[part][col] = s;
        __syncthreads();
        if (tid < NB) acc -= red[0][tid] + red[1][tid] + red[2][tid] + red[3][tid];
    }
    if (tid < NB) wb[tid] = acc;
    __syncthreads();
    const int rr = tid >> 2, sub = tid & 3;
    double s = 0.0;
    for (int t = rr + sub; t < NB; t += 4) s = fma(D[t][rr], wb[t], s);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    if (sub == 0) {
        x[(int64_t)c * NB + rr] = s;
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) *(volatile int *)(flags + c) = 1;
}

// r = y - K alpha (one warp per row).
__device__ __forceinline__ void k_residual_body(const double *__restrict__ K, const double *__restrict__ alpha,
                           const double *__restrict__ y, int n_pad, double *__restrict__ r, const int bx, const int by)
{
    const int row = bx * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
    if (row >= n_pad) return;
    const double *Kr = K + (int64_t)row * n_pad;
    double s = 0.0;
    for (int j = lane; j < n_pad; j += 32) s = fma(Kr[j], alpha[j], s);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) r[row] = y[row] - s;
}

// Refinement correction through X = L^-1 (lower triangular, row-major; FP64 or FP32), shared by
// the single-problem and batched paths.  u = X r: one warp per row (row bx * 8 + warp).
template <typename T>
__device__ __forceinline__ void k_trmv_body(const T *__restrict__ X, int n_pad, const double *__restrict__ r,
                                            double *__restrict__ u, const int bx)
{
    const int i = bx * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (i >= n_pad) return;
    const T *row = X + (int64_t)i * n_pad;
    T s = T(0);
    for (int j = lane; j <= i; j += 32) s = fma(row[j], (T)r[j], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) u[i] = (double)s;
}

// d = X^T u in two deterministic passes: CTA (bx, by) of 256 threads sums rows
// TRMV_ROWS by .. of columns 32 bx .. into part[by][j] (zero above the diagonal); then
// k_trmv_t_sum_body adds the row chunks in order and applies a += d (with the FP32 copy of a).
constexpr int TRMV_ROWS = 256;
template <typename T>
__device__ __forceinline__ void k_trmv_t_part_body(const T *__restrict__ X, int n_pad, const double *__restrict__ u,
                                                   double *__restrict__ part, const int bx, const int by)
{
    __shared__ T red[8][32];
    const int j = bx * 32 + (threadIdx.x & 31), w = threadIdx.x >> 5;
    const int i0 = by * TRMV_ROWS + w * (TRMV_ROWS / 8), i1 = min(i0 + TRMV_ROWS / 8, n_pad);
    T s = T(0);
    for (int i = max(i0, j); i < i1; ++i) s = fma(X[(int64_t)i * n_pad + j], (T)u[i], s);
    red[w][threadIdx.x & 31] = s;
    __syncthreads();
    if (w == 0) {
        for (int g = 1; g < 8; ++g) s += red[g][threadIdx.x];
        part[(int64_t)by * n_pad + j] = (double)s;
    }
}

__device__ __forceinline__ void k_trmv_t_sum_body(const double *__restrict__ part, int n_pad, int chunks,
                                                  double *__restrict__ a, float *__restrict__ a32, const int bx)
{
    const int j = bx * blockDim.x + threadIdx.x;
    if (j >= n_pad) return;
    double d = 0.0;
    for (int c = j / TRMV_ROWS; c < chunks; ++c) d += part[(int64_t)c * n_pad + j];
    const double v = a[j] + d;
    a[j] = v;
    a32[j] = (float)v;
}

__device__ __forceinline__ void k_axpy_cast_body(double *__restrict__ a, const double *__restrict__ dlt, int n, float *__restrict__ a32, const int bx, const int by)
{
    int i = bx * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = dlt ? a[i] + dlt[i] : a[i];
    a[i] = v;
    if (a32) a32[i] = (float)v;
}

__device__ __forceinline__ void k_pad_copy_body(const double *__restrict__ y, int n, int n_pad, double *__restrict__ out, const int bx, const int by)
{
    int i = bx * blockDim.x + threadIdx.x;
    if (i < n_pad) out[i] = i < n ? y[i] : 0.0;
}

// ------------------------------------------------------------------ triangular inverse
// Batched SIMT GEMM C = alpha * A * B on row-major tiles; each problem in `probs` has its own
// operand offsets and shape.  tri_a: A is lower triangular (skip k > row block end);
// tri_b: B is lower triangular (skip k < column block start).

template <typename T>
__device__ __forceinline__ void k_gemm_batched_body(const T *__restrict__ Abase, const T *__restrict__ Bbase,
                                                      T *__restrict__ Cbase, int lda, int ldb, int ldc,
                                                      const GemmProb *__restrict__ probs, T alpha, int tri_a,
                                                      int tri_b, const int bx, const int by)
{
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    const GemmProb pr = probs[blockIdx.z];
    const int m0 = by * BM, n0 = bx * BN;
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
            As[c][r] = (gr < pr.m && gc < pr.k) ? A[(int64_t)gr * pr.ld + gc] : T(0);
        }
        for (int e = tid; e < BK * BN; e += 256) {
            int r = e / BN, c = e % BN;
            int gr = k0 + r, gc = n0 + c;
            Bs[r][c] = (gr < pr.k && gc < pr.n) ? B[(int64_t)gr * pr.ld + gc] : T(0);
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
            if (gr < pr.m && gc < pr.n) C[(int64_t)gr * pr.ld + gc] = alpha * acc[u][v];
        }
}

// FP32 form of the same product for the large levels of the recursion (m, n >= 128): CTA tile
// 128 x 128, K steps of 8, 256 threads with an 8 x 8 register tile each (rows ty*4 + {0..3}
// and 64 + ty*4 + {0..3}, the same for columns), 128-bit shared-memory reads, and the next K
// step's global loads held in registers while the current one is multiplied (two smem
// buffers, one barrier per step).  m, n, k and the offsets are multiples of 64, so the only
// ragged edge is a half tile in m or n, which is zero-filled.
__device__ __forceinline__ void k_gemm128_body(const float *__restrict__ Abase, const float *__restrict__ Bbase,
                                               float *__restrict__ Cbase, const GemmProb *__restrict__ probs,
                                               float alpha, int tri_a, int tri_b, const int bx, const int by,
                                               const int bz)
{
    constexpr int BM = 128, BN = 128, BK = 8;
    __shared__ __align__(16) float As[2][BK][BM];
    __shared__ __align__(16) float Bs[2][BK][BN];
    const GemmProb pr = probs[bz];
    const int m0 = by * BM, n0 = bx * BN;
    if (m0 >= pr.m || n0 >= pr.n) return;
    const float *A = Abase + pr.a_off;
    const float *B = Bbase + pr.b_off;
    float *C = Cbase + pr.c_off;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    int kbeg = 0, kend = pr.k;
    if (tri_a) kend = min(kend, m0 + BM);
    if (tri_b) kbeg = n0;
    // loader roles: A rows ra (2 threads per row, 4 k each), B row rb (32 threads per row, 4 cols each)
    const int ra = tid / 2, ca = (tid % 2) * 4;
    const int rb = tid / 32, cb = (tid % 32) * 4;
    const bool a_ok = m0 + ra < pr.m, b_ok = n0 + cb < pr.n;
    float4 pa = make_float4(0.f, 0.f, 0.f, 0.f), pb = pa;
    auto fetch = [&](int k0) {
        pa = a_ok ? *reinterpret_cast<const float4 *>(A + (int64_t)(m0 + ra) * pr.ld + k0 + ca) : make_float4(0.f, 0.f, 0.f, 0.f);
        pb = b_ok ? *reinterpret_cast<const float4 *>(B + (int64_t)(k0 + rb) * pr.ld + n0 + cb) : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    auto stash = [&](int buf) {
        As[buf][ca + 0][ra] = pa.x;
        As[buf][ca + 1][ra] = pa.y;
        As[buf][ca + 2][ra] = pa.z;
        As[buf][ca + 3][ra] = pa.w;
        *reinterpret_cast<float4 *>(&Bs[buf][rb][cb]) = pb;
    };
    float acc[8][8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[u][v] = 0.f;
    int buf = 0;
    if (kbeg < kend) {
        fetch(kbeg);
        stash(0);
    }
    __syncthreads();
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        const bool more = k0 + BK < kend;
        if (more) fetch(k0 + BK);
#pragma unroll
        for (int t = 0; t < BK; ++t) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][t][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][t][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][t][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][t][64 + tx * 4]);
            const float x[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float y[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(x[u], y[v], acc[u][v]);
        }
        if (more) stash(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int gr = m0 + (u < 4 ? ty * 4 + u : 64 + ty * 4 + (u - 4));
        if (gr >= pr.m) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int gc = n0 + h * 64 + tx * 4;
            if (gc >= pr.n) continue;
            float4 o = make_float4(alpha * acc[u][h * 4], alpha * acc[u][h * 4 + 1], alpha * acc[u][h * 4 + 2],
                                   alpha * acc[u][h * 4 + 3]);
            *reinterpret_cast<float4 *>(C + (int64_t)gr * pr.ld + gc) = o;
        }
    }
}

// Linv's diagonal blocks from Dinv (rounded to T); everything else zero.
template <typename T>
__device__ __forceinline__ void k_linv_init_body(const double *__restrict__ Dinv, int n_pad, T *__restrict__ Linv, const int bx, const int by)
{
    int64_t t = bx * (int64_t)blockDim.x + threadIdx.x;
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
__device__ __forceinline__ void k_cast_body(const Tin *__restrict__ in, int64_t count, Tout *__restrict__ out, const int bx, const int by)
{
    int64_t t = bx * (int64_t)blockDim.x + threadIdx.x;
    if (t < count) out[t] = convert_to<Tout>((double)in[t]);
}

// BF16 operands with a compensated inverse: hi = bf16(L^-1), lo = bf16(L^-1 - hi).
__device__ __forceinline__ void k_split_bf16_body(const float *__restrict__ in, int64_t count, __nv_bfloat16 *__restrict__ hi,
                             __nv_bfloat16 *__restrict__ lo, const int bx, const int by)
{
    int64_t t = bx * (int64_t)blockDim.x + threadIdx.x;
    if (t >= count) return;
    const float v = in[t];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[t] = h;
    lo[t] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// Zero rows n..n_pad-1 of a 16-bit L^-1 (count rows of width n_pad), so that the cross-kernel
// values of padded observations never reach the variance.
__device__ __forceinline__ void k_zero_pad_rows_body(uint16_t *__restrict__ A, int n, int n_pad, const int bx, const int by)
{
    int64_t t = bx * (int64_t)blockDim.x + threadIdx.x;
    const int64_t cnt = (int64_t)(n_pad - n) * n_pad;
    if (t < cnt) A[(int64_t)n * n_pad + t] = 0;
}

// ------------------------------------------------------------------ standardisation
// ys = (y - mean) / std (population std; 1 when zero), tau = min ys.  One CTA.
__device__ __forceinline__ void k_standardize_body(const double *__restrict__ y, int n, double *__restrict__ ys,
                                                      double *__restrict__ tau, const int bx, const int by)
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


}  // namespace gpbo
