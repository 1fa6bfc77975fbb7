// Internal declarations shared by the CUDA sources of libgpbo.so.
// Nothing here is part of the public ABI (include/gpbo.h is).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <cstdio>

#include "../../include/gpbo.h"

namespace gpbo {

// Block size of the FP64 factorisation and of the padded square layouts.
constexpr int NB = 64;
// The tensor-core variance kernel works on L^-1 in row chunks of this many outputs,
// so tensor-core models pad n to a multiple of it.
constexpr int TC_NCHUNK = 256;

inline int round_up(int v, int m) { return (v + m - 1) / m * m; }
inline int64_t round_up64(int64_t v, int64_t m) { return (v + m - 1) / m * m; }
inline int64_t cdiv64(int64_t a, int64_t b) { return (a + b - 1) / b; }

void note_cuda_error(cudaError_t e, const char *what, const char *file, int line);

#define GPBO_CUDA_TRY(expr)                                                    \
    do {                                                                       \
        cudaError_t e_ = (expr);                                               \
        if (e_ != cudaSuccess) {                                               \
            gpbo::note_cuda_error(e_, #expr, __FILE__, __LINE__);              \
            return e_ == cudaErrorMemoryAllocation ? GPBO_ENOMEM : GPBO_ECUDA; \
        }                                                                      \
    } while (0)

#define GPBO_LAUNCH_CHECK(ctx)                                            \
    do {                                                                  \
        (ctx)->launches++;                                                \
        cudaError_t e_ = cudaGetLastError();                              \
        if (e_ != cudaSuccess) {                                          \
            gpbo::note_cuda_error(e_, "kernel launch", __FILE__, __LINE__); \
            return GPBO_ECUDA;                                            \
        }                                                                 \
    } while (0)

#define GPBO_TRY(expr)                \
    do {                              \
        int s_ = (expr);              \
        if (s_ != GPBO_OK) return s_; \
    } while (0)

// Device-side error word bits (gpbo_ctx::dev_status).
enum : unsigned {
    DEV_NOTSPD = 1u,
    DEV_TIMEOUT = 2u,
    DEV_NAN = 4u,
};

// Default limit of a bounded device wait: about 2 s of SM clock.
constexpr long long WAIT_DEFAULT_CYCLES = 4000000000ll;

// Limit of a wait that may give up: the context's wait limit, a count of SM clock cycles kept as
// a 64-bit word at byte 8 of its status buffer (gpbo_set_wait_limit; 0 means the default).
__device__ __forceinline__ long long wait_limit(const unsigned *status)
{
    const long long v = *(const volatile long long *)(status + 2);
    return v > 0 ? v : WAIT_DEFAULT_CYCLES;
}

}  // namespace gpbo

namespace gpbo {
constexpr int TRACE_PHASES = 6;
enum { PH_FIT = 0, PH_XKERN = 1, PH_VAR = 2, PH_SCREEN = 3, PH_CHOL_UPDATE = 4, PH_LML = 5, PH_FACTOR = 6, PH_INVERSE = 7 };
struct TraceRec {
    int phase;
    cudaEvent_t a, b;
    double flops;
};
}  // namespace gpbo

struct gpbo_ctx {
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int64_t launches = 0;
    int64_t ws_limit = (int64_t)2 << 30;
    void *ws = nullptr;              // grow-only scratch arena
    size_t ws_size = 0;
    unsigned *dev_status = nullptr;  // 64 device bytes: [0] error bits (cleared by each call),
                                     // [4] injected faults, [8] wait limit in cycles (int64)
    void *pinned = nullptr;          // small pinned host staging buffer
    bool trace = false;              // per-phase event timing (gpbo_trace_enable)
    gpbo::TraceRec *trace_recs = nullptr;
    int trace_n = 0, trace_cap = 0;
    int trace_stack[8];              // open intervals (they nest)
    int trace_depth = 0;
    void *batch_plan = nullptr;      // captured batched step for the last set of shapes
    int batch_tile = 0;              // batched variance tile (0: autotune)
    cudaStream_t side = nullptr;     // high-priority streams for work overlapped inside a call
    cudaStream_t side2 = nullptr;
    cudaStream_t side3 = nullptr;    // lowest priority: the fit's leading-half inverse under its factorisation
    cudaStream_t mainf = nullptr;    // the fit's main-stream work, between the chain's priority and side3's
    cudaEvent_t side_ev[12] = {};    // fork / join events between the streams
    gp_model *step_model = nullptr;  // search_step's model, kept for the next call of the same shape
    void *step_buf = nullptr;        // search_step's device staging
    size_t step_buf_bytes = 0;
};

struct gp_model {
    gpbo_ctx *ctx = nullptr;
    int n = 0, d = 0, n_pad = 0;
    int prec = GPBO_PREC_F64;
    double s2 = 1.0, sn2 = 0.0;
    double ls[GPBO_MAX_D];
    // device buffers (n_pad x n_pad squares are row-major; padding rows/cols hold the
    // identity on the diagonal of K and L and zero elsewhere)
    double *X = nullptr;        // n x d FP64 as given
    double *Xs64 = nullptr;     // d x n_pad FP64, x / l, zero padding
    float *Xs32 = nullptr;      // d x n_pad FP32, x / l
    double *K = nullptr;        // n_pad x n_pad kernel matrix (kept for the refinement residual)
    double *L = nullptr;        // n_pad x n_pad factor, lower
    double *Dinv = nullptr;     // n_pad/NB blocks of NB x NB: inverses of L's diagonal blocks
    double *alpha64 = nullptr;  // n_pad, zero padding
    float *alpha32 = nullptr;   // n_pad
    double *Linv64 = nullptr;   // F64 scoring: L^-1
    float *Linv32 = nullptr;    // F32 and tensor-core scoring: L^-1 in FP32
    void *Linv16 = nullptr;     // F16: L^-1 rounded; BF16: hi = bf16(L^-1) then lo = bf16(L^-1 - hi)
    void *Zsplit = nullptr;     // 16-bit models, d <= 32: n_pad x 128 FP16 [hi | lo | hi | 0] of (x - 1/2) / l
    float *nb32 = nullptr;      // 16-bit models: |(x_i - 1/2) / l|^2
    void *cslices = nullptr;    // n_pad >= CHOL_TC_UPDATE_MIN_NPAD: 7 BF16 slices of a Cholesky panel, slice-major
    int *cexps = nullptr;       // their per-row exponents
    unsigned long long *xmax = nullptr;  // n_pad >= CHOL_TC_MIN_NPAD: largest |x / l| as magnitude bits
};

namespace gpbo {

// capi.cu
int ws_reserve(gpbo_ctx *ctx, size_t bytes, void **out);
// Raise kernel fn's dynamic shared-memory limit on `device` (which must be current) to at least
// `bytes`.  The attribute belongs to the device, so what was set is remembered per (kernel,
// device) under a lock: contexts on several devices, or on several host threads, each get it.
int ensure_smem(const void *fn, int device, int bytes);
// The context's high-priority side stream (created on first use).  Every call that forks
// work onto it joins back into ctx->stream before returning.
int side_stream(gpbo_ctx *ctx, cudaStream_t *out);
// Open / close a timed interval of `phase` on the context's stream (no-ops unless tracing).
int trace_begin(gpbo_ctx *ctx, int phase, double flops);
int trace_end(gpbo_ctx *ctx);
int take_device_status(gpbo_ctx *ctx, unsigned *bits_out);
// Allocate a model's device buffers for n x d in the given precision (hyperparameters unset),
// free one, and validate hyperparameters.
int model_create(gpbo_ctx *ctx, int n, int d, int prec, gp_model **out);
int model_n_pad(int n, int prec);
void model_free(gp_model *m);
int check_hyper(const gp_hyper *hyp, int d);

// fit.cu
int fit_model(gpbo_ctx *ctx, gp_model *m, const double *X_dev, const double *y_dev);
int standardize_dev(gpbo_ctx *ctx, const double *y, int n, double *ys, double *tau_dev);

// score.cu
int score_model(gpbo_ctx *ctx, const gp_model *m, const float *Xc_dev, int64_t M, uint64_t seed,
                double y_best, const double *tau_dev, double xi, void *mu, void *sigma, void *ei,
                int64_t *argmax, double *ei_max);
int gen_candidates(gpbo_ctx *ctx, uint64_t seed, int64_t first, int64_t M, int d, float *out);

// score_tc.cu: one chunk of C candidates whose K* (C x n_pad, 16-bit) and mu are ready.
int tc_variance_ei(gpbo_ctx *ctx, const gp_model *m, const void *Kstar, int64_t C, int64_t c0,
                   const float *mu, double y_best, const double *tau_dev, double xi, float *sigma_out,
                   float *ei_out, float *part_ei, int64_t *part_idx, int *n_parts);

// xkern_tc.cu: the cross-kernel on tensor cores for 16-bit models with d <= 32.
int xkern_tc_prepare(gpbo_ctx *ctx, gp_model *m);

// chol_tc.cu: trailing updates of the Cholesky factorisation on the tensor cores at FP64
// accuracy (exact 8-bit slice products).  Models with n_pad >= CHOL_TC_MIN_NPAD also compute
// their kernel matrix distances in integers and the large levels of L^-1 on the tensor cores;
// models with n_pad >= CHOL_TC_UPDATE_MIN_NPAD take the tensor-core update at every step that
// leaves at least CHOL_TC_MIN_T block columns after the lookahead column (the last few small
// updates stay on the FP64 pipe).  The batched step applies the same rule per problem.
constexpr int CHOL_TC_MIN_NPAD = 1536;
constexpr int CHOL_TC_UPDATE_MIN_NPAD = 384;
constexpr int CHOL_TC_MIN_T = 4;
__host__ __device__ inline bool chol_tc_step(int n_pad, int nblk, int kb)
{
    return n_pad >= CHOL_TC_UPDATE_MIN_NPAD && nblk - kb - 2 >= CHOL_TC_MIN_T;
}
// One problem of a tensor-core update: its factor (n_pad x n_pad), its per-row exponents, and the
// first row of its slices in the slice arena (7 n_pad rows of 64 BF16 values, slice-major).
struct CholTcProb {
    double *A;
    int *exps;
    int n_pad, nblk;
    int64_t row_off;
};
bool chol_tc_enabled(const gp_model *m);
size_t chol_tc_slice_bytes(int n_pad);
int chol_tc_maps(const gp_model *m, void *map_a, void *map_b);  // two 128-byte CUtensorMap
// Output tiles (128 x 64) of step kb's tensor-core update: strips of two block rows from block
// row kb + 2 on, each meeting the block columns kb + 2 .. up to its own.
__host__ __device__ inline int64_t chol_tc_tiles(int nblk, int kb)
{
    const int T2 = nblk - (kb + 2);
    int64_t t = 0;
    for (int i2 = 0; 2 * i2 < T2; ++i2) t += 2 * i2 + 2 < T2 ? 2 * i2 + 2 : T2;
    return t;
}
// Step kb of a single model: block columns c0 .. (c0 = kb + 1 or kb + 2) of block rows kb + 2 ..,
// with the maps of chol_tc_maps (row strips of 128, column tiles of 32).
int chol_tc_update(gpbo_ctx *ctx, gp_model *m, int kb, int c0, cudaStream_t st, const void *map_a, const void *map_b);
// The batched form: tensor maps over a slice arena of `rows` rows, and step kb for every problem
// of probs (device, G entries) with chol_tc_step true (blockIdx.y = problem; max_rows and
// max_tiles bound the problems' rows below block row kb + 2 and their tiles).
int chol_tc_arena_maps(const void *slices, int64_t rows, void *map_a, void *map_b);
int chol_tc_update_batched(gpbo_ctx *ctx, cudaStream_t st, const CholTcProb *probs, int G, int kb, int max_rows,
                           int64_t max_tiles, void *slices, const void *map_a, const void *map_b);

// kinv_tc.cu: lower 64 x 64 tiles of K^-1 = L^-T L^-1 on the tensor cores at FP64 accuracy,
// from Linv (n_pad x n_pad FP64; n_pad a multiple of 128).  slices: kinv_tc_slice_bytes(n_pad)
// bytes and exps: n_pad ints of device scratch.
size_t kinv_tc_slice_bytes(int n_pad);

// dgemm_tc.cu: one level of the FP64 triangular inverse's products at FP64 accuracy on the
// tensor cores: C_q = alpha A_q B_q (tri: 1 = B lower triangular, 2 = A lower triangular).
// Batched SIMT GEMM problem: operand offsets (elements) and shape; ld = leading dimension
// of all three operands (the problem's n_pad).
struct GemmProb {
    int64_t a_off, b_off, c_off;
    int m, n, k;
    int ld;
};
size_t dtc_scratch_bytes(int cnt, int mk, int nmax);
int dgemm_tc_level(gpbo_ctx *ctx, cudaStream_t st, const double *A, const double *B, double *C, int ld,
                   const GemmProb *probs, int cnt, double alpha, int tri, void *scratch);
size_t stc_scratch_bytes(int cnt, int mk, int nmax);
int sgemm_tc_level(gpbo_ctx *ctx, cudaStream_t st, const float *A, const float *B, float *C, int ld,
                   const GemmProb *probs, int cnt, double alpha, int tri, void *scratch);
int kinv_tc(gpbo_ctx *ctx, cudaStream_t st, const double *Linv, int n_pad, void *slices, int *exps, double *C);
bool xkern_tc_usable(const gp_model *m);
int xkern_tc(gpbo_ctx *ctx, const gp_model *m, const float *Xc, uint64_t seed, int64_t c0, int64_t C, void *Kst,
             float *mu);

// mlp_tc.cu: the ensemble pre-screen forward on the tensor cores (hidden width 256, d <= 31, E <= 8).
bool mlp_tc_usable(int d, int H, int E);
size_t mlp_tc_weight_bytes(int E);
size_t mlp_tc_aux_floats(int E);
int mlp_tc_pack(gpbo_ctx *ctx, const float *theta, int E, int d, int64_t P, const int64_t off[6], void *wt, float *aux);
int mlp_tc_score(gpbo_ctx *ctx, const void *wt, const float *aux, int E, int d, const double norm[4], const float *Xc,
                 uint64_t seed, int64_t c0, int64_t C, double tau, double xi, float *ei, float *mu, float *sigma);

// batched.cu
void batch_plan_free(void *plan);

// screen.cu
int screen_run(gpbo_ctx *ctx, const gpbo_objective *obj, int d, const screen_opts *o, double *score,
               double *influence, int *group_of, int *n_groups, int *fixed);

// 1 / lengthscale per dimension, passed by value to kernels.
struct Lengthscales_inv {
    double inv[GPBO_MAX_D];
};

// ------------------------------------------------------------------ device helpers
// Two FP32 lanes per instruction (fma.rn.f32x2, mul.rn.f32x2, add.rn.f32x2): each lane is the
// IEEE round-to-nearest FMA, product or sum of its own operands, as the scalar instructions.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c)
{
    float2 d;
    asm("{.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b)
{
    float2 d;
    asm("{.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b)
{
    float2 d;
    asm("{.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

__host__ __device__ inline uint64_t splitmix64(uint64_t seed, uint64_t stream, uint64_t counter)
{
    // SplitMix64 output number `counter` of the generator seeded with seed ^ stream*gamma.
    const uint64_t gamma = 0x9E3779B97F4A7C15ull;
    uint64_t z = (seed ^ (stream * gamma)) + (counter + 1ull) * gamma;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ inline float uniform24f(uint64_t seed, uint64_t stream, uint64_t counter)
{
    return (float)(splitmix64(seed, stream, counter) >> 40) * (1.0f / 16777216.0f);
}

__host__ __device__ inline double uniform24d(uint64_t seed, uint64_t stream, uint64_t counter)
{
    return (double)(splitmix64(seed, stream, counter) >> 40) * (1.0 / 16777216.0);
}

constexpr double SQRT5 = 2.23606797749978969641;

// Matern nu=5/2 shape (1 + sqrt5 r + 5 r^2/3) exp(-sqrt5 r), from the squared distance.
__device__ __forceinline__ double matern52_r2(double r2)
{
    double r = sqrt(r2);
    double t = SQRT5 * r;
    return (1.0 + t + (5.0 / 3.0) * r2) * exp(-t);
}

__device__ __forceinline__ float matern52_r2f(float r2)
{
    float r = sqrtf(r2);
    float t = 2.2360680f * r;
    return (1.0f + t + 1.6666666f * r2) * __expf(-t);
}

// Expected improvement below tau for minimisation (Jones, Schonlau, Welch 1998).
__device__ __forceinline__ double ei_min(double mu, double sigma, double tau, double xi)
{
    double imp = tau - mu - xi;
    if (!(sigma > 0.0)) return imp > 0.0 ? imp : 0.0;
    double z = imp / sigma;
    return imp * (0.5 * erfc(-z * 0.70710678118654752440)) + sigma * (0.39894228040143267794 * exp(-0.5 * z * z));
}

__device__ __forceinline__ float ei_minf(float mu, float sigma, float tau, float xi)
{
    float imp = tau - mu - xi;
    if (!(sigma > 0.0f)) return imp > 0.0f ? imp : 0.0f;
    float z = imp / sigma;
    return imp * (0.5f * erfcf(-z * 0.70710678f)) + sigma * (0.39894228f * expf(-0.5f * z * z));
}

// Argmax tie rule: larger value wins, then the lower index.
template <typename T>
__device__ __forceinline__ bool better(T v, int64_t i, T bv, int64_t bi)
{
    return v > bv || (v == bv && i < bi);
}

}  // namespace gpbo
