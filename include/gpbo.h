/*
 * gpbo.h -- C ABI of libgpbo.so, the B300 (sm_103a) hot path of the GP-BO tuning loop
 * in "Cost-Effective Methodology for Complex Tuning Searches in HPC" (arXiv 2403.08131).
 *
 * The paper runs Bayesian optimisation (a surrogate trained on the evaluated
 * configurations, an acquisition function choosing the next one; §III-A) inside every
 * independent or merged sub-search, after an interdependence analysis decides which
 * routines' parameters are searched together (§IV-B..D).  This library computes, on one
 * GPU, the step every sub-search repeats and the screen that forms the sub-searches:
 *
 *   gp_fit           Matern-5/2 ARD kernel matrix, FP64 Cholesky, refined alpha = K^-1 y,
 *                    and the triangular inverse used to score candidates;
 *   gp_posterior_ei  posterior mean and standard deviation of many candidates, expected
 *                    improvement and its argmax, fused;
 *   interdep_screen  pairwise or per-routine perturbation screen, cut-off, merge, 10-cap;
 *   search_step      one BO iteration: standardise, fit, score, return the next point.
 *
 * Conventions for every call:
 *   - Every function returns a gpbo_status; no C++ exception crosses the ABI.
 *   - Outputs are left untouched when the status is not GPBO_OK.
 *   - Array arguments are DEVICE pointers on the context's device unless `flags`
 *     contains GPBO_HOST_PTRS, in which case they are host pointers and the call copies
 *     them in and out itself.  Small per-call scalars and vectors named "host" below are
 *     always host pointers.
 *   - The caller owns every array it passes.  The library owns gpbo_ctx and gp_model.
 *   - Work is ordered on the context's stream.  Calls that return host scalars
 *     synchronise that stream before returning.
 *   - One context per host thread; contexts are independent.
 *   - Limits: 1 <= d <= 64, 1 <= n <= 16384, 1 <= M < 2^31.
 *   - The library never falls back to the CPU; without a usable GPU, gpbo_create fails.
 */
#ifndef GPBO_H
#define GPBO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GPBO_MAX_D 64
#define GPBO_MAX_N 16384

typedef struct gpbo_ctx gpbo_ctx; /* opaque: stream, workspace arena, device properties */
typedef struct gp_model gp_model; /* opaque: device copies of X, L, L^-1, alpha, hyperparameters */

typedef enum gpbo_status {
    GPBO_OK = 0,
    GPBO_EINVAL = 1,   /* bad size, null pointer, d or n out of range */
    GPBO_ENOTSPD = 2,  /* a Cholesky pivot was not positive */
    GPBO_ENAN = 3,     /* NaN or Inf in X, y or a candidate */
    GPBO_ENOMEM = 4,   /* device allocation failed */
    GPBO_ECUDA = 5,    /* a CUDA runtime call failed */
    GPBO_ETIMEOUT = 6, /* a bounded device-side wait gave up; the kernel exited cleanly */
    GPBO_ENOTSUP = 7,  /* the device is not sm_103 or the request needs a missing feature */
    GPBO_ESCRATCH = 8  /* the problem does not fit the fixed scratch of gp_posterior_ei_noalloc */
} gpbo_status;

/* Scoring precision of the posterior variance (the fit is FP64 in every case).
 *   F64  : all of the scoring in FP64 on CUDA cores.
 *   F32  : cross-kernel and variance products in FP32 on CUDA cores.
 *   BF16 : variance operands on tcgen05 tensor cores with FP32 accumulation in tensor
 *          memory: K* rounded to BF16, L^-1 carried as two BF16 terms (hi + lo) so that its
 *          rounding cancels (twice the tensor work of F16); mean and EI in FP32 from FP32 K*.
 *   F16  : K* and L^-1 rounded to IEEE half, one tensor-core pass (same rate as BF16,
 *          3 more mantissa bits; the fast accurate path). */
typedef enum gpbo_prec {
    GPBO_PREC_F64 = 0,
    GPBO_PREC_F32 = 1,
    GPBO_PREC_BF16 = 2,
    GPBO_PREC_F16 = 3
} gpbo_prec;

#define GPBO_HOST_PTRS 0x1u /* array arguments are host pointers (copied in/out by the call) */
#define GPBO_JITTER 0x2u    /* on a failed Cholesky, retry with noise_var x10, at most 3 times */

/* Fixed GP hyperparameters (the paper leaves the surrogate to GPTune; these are the
 * Matern nu=5/2 ARD covariance's parameters, Rasmussen & Williams 2006 eq. 4.17):
 *   k(a, b) = signal_var * m(r),  r^2 = sum_k ((a_k - b_k) / lengthscale[k])^2,
 *   m(r) = (1 + sqrt5 r + 5 r^2 / 3) exp(-sqrt5 r),
 * plus noise_var on the diagonal of the training covariance.
 * lengthscale: host array of d positive values. */
typedef struct gp_hyper {
    int d;
    const double *lengthscale;
    double signal_var;
    double noise_var;
} gp_hyper;

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device`.  cuda_stream: a cudaStream_t to order work
 * on, or NULL for a stream the context creates and owns.  Fails with GPBO_ENOTSUP on a
 * device that is not compute capability 10.3. */
int gpbo_create(gpbo_ctx **out, int device, void *cuda_stream);
int gpbo_destroy(gpbo_ctx *ctx);
/* Re-target the context at another stream (NULL = its own). */
int gpbo_set_stream(gpbo_ctx *ctx, void *cuda_stream);
/* Static string for a status code. */
const char *gpbo_strerror(int status);
/* Kernels the context has launched since creation (for launch accounting). */
int64_t gpbo_launch_count(const gpbo_ctx *ctx);
/* Per-phase device timing with CUDA events recorded on the context's stream around each
 * phase's kernels (phases: 0 fit, 1 cross-kernel + mean, 2 variance + EI + argmax,
 * 3 screen, 4 Cholesky trailing updates, 5 the K^-1 tiles of the likelihood gradient:
 * 2 (p + 1)(n - p) flops for row p of the lower triangle of L^-T L^-1, 6 the fit's kernel
 * matrix and factorisation, 7 the fit's L^-1 and the solve for alpha after it; 6 and 7
 * lie inside 0, and 4 inside 6).
 * gpbo_trace_enable(ctx, 1) clears and starts collection, 0 stops it.
 * gpbo_trace_read synchronises, then writes for each of the first nphase phases the total
 * milliseconds, the number of timed intervals, and the algorithmic flops the phase's
 * kernels were asked to do (variance: n(n+1) per candidate; cross-kernel: 3nd + 2n;
 * trailing updates: 2 * 64^3 per updated 64 x 64 tile). */
int gpbo_trace_enable(gpbo_ctx *ctx, int on);
int gpbo_trace_read(gpbo_ctx *ctx, int nphase, double *ms, int64_t *intervals, double *flops);
/* Measured CUDA-core FMA throughput of the context's device, for roofline denominators:
 * kind 0 = FP64 DFMA, 1 = FP32 FFMA.  Runs a short in-bounds FMA-chain kernel (about 50 ms)
 * and writes TFLOP/s (2 flops per FMA) to *tflops.  Synchronises. */
int gpbo_probe_fma(gpbo_ctx *ctx, int kind, double *tflops);
/* Bounded device waits.  Every wait inside the library's kernels that can give up (the
 * producer / consumer waits of the tensor-core kernels, the flag waits of the wavefront
 * substitutions) does so after `cycles` SM clock cycles; 0 restores the default, about 2 s.
 * A kernel whose wait gives up sets an error bit, leaves its loops, lets the copies and MMAs it
 * issued finish (those drains always allow the default limit, so shared and tensor memory are
 * never released under an asynchronous operation), frees its tensor memory and exits; the call
 * then returns GPBO_ETIMEOUT and the context stays usable.  A short limit can make ordinary
 * calls time out: it is meant for tests of that error path.  Synchronises. */
int gpbo_set_wait_limit(gpbo_ctx *ctx, int64_t cycles);
/* Failure injection for tests of the error path above, with no fault and no unbounded wait:
 * with stall = 1 the epilogue warps of the tensor-core variance kernel (16-bit models) first
 * wait on a barrier that nothing arrives at, so that the wait runs out after the wait limit and
 * the scoring call returns GPBO_ETIMEOUT.  stall = 0 turns it off.  Synchronises. */
int gpbo_inject_wait_stall(gpbo_ctx *ctx, int stall);
/* Upper bound, in bytes, of the scratch arena the context may grow to (default 2 GiB).
 * Candidate scoring works through the pool in chunks that fit in this bound. */
int gpbo_set_workspace_limit(gpbo_ctx *ctx, int64_t bytes);

/* ------------------------------------------------------------------ fit (§III-A)
 * Train the surrogate on n evaluated configurations (§III-A: the surrogate is trained
 * on the configurations evaluated so far; §IV-D: GP training is O(N^3)).
 *   X : n x d row-major FP64, the configurations scaled into [0,1]^d.
 *   y : n FP64 objective values, used as given (zero prior mean).
 * Computes K, L with K = L L^T in FP64, alpha = K^-1 y by FP64 blocked substitution
 * with one refinement step r = y - K alpha, alpha += K^-1 r, and L^-1 in the scoring
 * precision's working type (FP64 for F64, FP32 otherwise).
 * flags: GPBO_HOST_PTRS, GPBO_JITTER.  On success *out owns the model; free it with
 * gp_model_free.  GPBO_ENOTSPD when a pivot is not positive (after any jitter retries). */
int gp_fit(gpbo_ctx *ctx, const double *X, const double *y, int n, int d, const gp_hyper *hyp,
           gpbo_prec prec, unsigned flags, gp_model **out);
/* Free a model.  Models must be freed before the context they were fitted on. */
int gp_model_free(gp_model *model);
/* Shape and the noise variance actually used (differs from hyp->noise_var after jitter). */
int gp_model_info(const gp_model *model, int *n, int *d, int *prec, double *noise_var_used);
/* Copy the FP64 factor L (n x n row-major, zeros above the diagonal) or alpha (n) to host
 * memory.  Either pointer may be NULL.  Synchronises. */
int gp_model_read(const gp_model *model, double *L_host, double *alpha_host);

/* ------------------------------------------------------------------ score (§III-A)
 * Posterior of the latent objective at M candidates and expected improvement below the
 * incumbent y_best (minimisation; Jones et al. 1998), fused with its argmax:
 *   mu_c    = sum_i k(x_c, x_i) alpha_i
 *   sigma_c = sqrt(max(signal_var - |L^-1 k_c|^2, 0))
 *   EI_c    = (y_best - mu_c - xi) Phi(z) + sigma_c phi(z),  z = (y_best - mu_c - xi)/sigma_c,
 *             and max(y_best - mu_c - xi, 0) where sigma_c = 0.
 * Xc : M x d row-major FP32 candidates in [0,1]^d, or NULL to draw them on the device
 *      from `seed` (SplitMix64 counter stream 2, 24-bit uniforms; gpbo_gen_candidates).
 * mu, sigma, ei : M-element outputs, each may be NULL.  Element type is double for a
 *      GPBO_PREC_F64 model and float otherwise.
 * argmax, ei_max : host scalars, required.  Ties go to the lowest index.
 * flags : GPBO_HOST_PTRS applies to Xc, mu, sigma and ei.  Synchronises. */
int gp_posterior_ei(gpbo_ctx *ctx, const gp_model *model, const float *Xc, int64_t M, uint64_t seed,
                    double y_best, double xi, unsigned flags, void *mu, void *sigma, void *ei,
                    int64_t *argmax, double *ei_max);

/* Allocation-free scoring (no counterpart in the paper; a deployment convenience).
 * Same results as gp_posterior_ei for an FP32 or FP64 model, but the call allocates no
 * memory at all: no cudaMalloc, no cudaFree, no allocating library routine.  It is meant
 * for callers that must not allocate device memory while they run -- a serving loop whose
 * memory is owned by a pooling allocator (PyTorch's caching allocator, an arena sized at
 * start-up), a process running under a hard device-memory cap, or code that already holds
 * every buffer it will ever use.  Its scratch space is one fixed array of
 * GPBO_NOALLOC_SCRATCH_BYTES (4 MiB) in the library's device memory, which every GPU that
 * loads the library holds until the process exits.
 *   - Xc, mu, sigma, ei are DEVICE pointers (no GPBO_HOST_PTRS); argmax, ei_max are host.
 *     Xc may be NULL to draw the candidates from `seed` as gp_posterior_ei does.
 *   - The model must be GPBO_PREC_F32 or GPBO_PREC_F64 (GPBO_ENOTSUP otherwise).
 *   - The pool is scored in chunks that fit the scratch; a model whose padded size is
 *     too large for even 64 candidates per chunk (FP32: n_pad > 16320; FP64: n_pad > 8128)
 *     is rejected with GPBO_ESCRATCH before any work is queued.
 *   - The first call on a device looks up the scratch array's device address (once per
 *     device, with that device current); make that first call before any stream capture.
 *     The address is kept for the life of the process: after cudaDeviceReset on that device
 *     it is stale, so do not call this entry point on a device that has been reset.
 *   - All calls share the one array and it keeps the last call's contents; each call
 *     clears what it needs.  Calls that overlap on the GPU (several streams or host
 *     threads at once on one device) race on the scratch: order them on one stream.
 *   - Synchronises the context's stream (to return argmax and ei_max). */
#define GPBO_NOALLOC_SCRATCH_BYTES (4u << 20)
int gp_posterior_ei_noalloc(gpbo_ctx *ctx, const gp_model *model, const float *Xc, int64_t M, uint64_t seed,
                            double y_best, double xi, void *mu, void *sigma, void *ei, int64_t *argmax,
                            double *ei_max);

/* Candidate c, coordinate k = uniform24(seed, stream 2, (first + c) * d + k) for
 * c < M, written as FP32 into the device array out (M x d).  SplitMix64 (Steele, Lea,
 * Flood 2014), output number `counter` of the generator seeded with
 * seed ^ (stream * 0x9E3779B97F4A7C15), top 24 bits scaled by 2^-24. */
int gpbo_gen_candidates(gpbo_ctx *ctx, uint64_t seed, int64_t first, int64_t M, int d, float *out);

/* ------------------------------------------------------------------ screen (§IV-B..D)
 * Built-in synthetic objectives: additive blocks, block b owns the next block_dim[b]
 * inputs, each mapped from [0,1] onto the function's usual domain (Ackley
 * [-32.768, 32.768], Rastrigin [-5.12, 5.12], chained Rosenbrock [-2, 2]).  The block
 * values are the "routine" outputs (§III-C: groups of a synthetic function stand for
 * routines of an application).  Each evaluation adds noise_sd * N(0,1) from counter
 * stream 4 of `seed` (Box-Muller).
 * Host black box instead: set fn (non-NULL); it is called on the host with one point
 * and must write f_total and, in ROUTINE mode, n_routines routine outputs; nonzero
 * return = failed evaluation (the screen then fails with GPBO_EINVAL).  param_owner[i]
 * (host, d entries) names the routine that owns parameter i in ROUTINE mode. */
typedef enum gpbo_fn { GPBO_FN_ACKLEY = 0, GPBO_FN_RASTRIGIN = 1, GPBO_FN_ROSENBROCK = 2 } gpbo_fn;
typedef int (*gpbo_host_fn)(const double *x, int d, double *f_total, double *f_routines, void *user);
typedef struct gpbo_objective {
    int n_blocks;
    const int *block_dim;   /* host, n_blocks entries */
    const int *block_fn;    /* host, n_blocks gpbo_fn codes */
    double noise_sd;
    uint64_t seed;
    gpbo_host_fn fn;        /* NULL = built-in blocks */
    int n_routines;         /* host black box only */
    const int *param_owner; /* host black box only, ROUTINE mode */
    void *user;
} gpbo_objective;

typedef enum gpbo_screen_mode {
    GPBO_SCREEN_PAIRWISE = 0,
    GPBO_SCREEN_ROUTINE = 1,
    GPBO_SCREEN_ROUTINE_SERIES = 2
} gpbo_screen_mode;
/* n_base base points b_k = (1-h) u, u uniform in [0,1)^d (stream 3); step h along each axis.
 * PAIRWISE: score_ij = mean_k |f(b+he_i+he_j) - f(b+he_i) - f(b+he_j) + f(b)|
 *                      / (mean_k(|f(b+he_i) - f(b)| + |f(b+he_j) - f(b)|) + 1e-12),
 *           edge i-j when score_ij > cutoff; influence_i = mean_k |f(b+he_i)-f(b)|/(|f(b)|+1e-12).
 * ROUTINE:  score_gi = mean_k |(f_g(b_k) - f_g(b_k + h e_i)) / f_g(b_k)| (§IV-B's score with
 *           V = n_base), routine g linked to the owner of parameter i when score_gi > cutoff
 *           (§IV-C); influence_i = max_g score_gi.
 * Linked parameters (PAIRWISE) or routines (ROUTINE) merge (union-find); a group's label is
 * its smallest parameter index.  A group with more than max_dims members keeps its max_dims
 * most influential ones and marks the rest fixed (§IV-D; max_dims <= 0 disables the cap).
 * Noise counters: PAIRWISE evaluation e of base k uses k*E + e, E = 1 + d + d(d-1)/2, with
 * e = 0 the base, 1+i the step along i, 1+d+p the double step of the p-th pair i<j in
 * lexicographic order.  ROUTINE output g of evaluation e (0 base, 1+i step) uses
 * (k*(1+d) + e)*R + g.
 * ROUTINE_SERIES: the paper's schedule for its synthetic functions (§IV-B): one baseline b
 *           (point 0 of stream 3, in [0,1)^d) and, for each parameter i in turn, V = n_base
 *           variations: the parameter's value in its own units, x = lo_i + (hi_i - lo_i) u,
 *           multiplied by (1 + growth) once per variation (10% in the paper), clamped to
 *           [lo_i, hi_i]; the other parameters stay at b.  score_gi = (1/V) sum_v
 *           |(f_g(b) - f_g(variation v of i)) / f_g(b)|; links, merge and cap as ROUTINE.
 *           The ranges are the built-in blocks' own domains, or lo / hi (host, d each; NULL:
 *           [0, 1]) for a host black box.  h is not used.  Output g of evaluation e (0 the
 *           baseline, 1 + i V + v - 1 the v-th variation of i) uses noise counter e R + g.
 * In both ROUTINE modes a host black box may give param_owner[i] = -1 for a parameter that
 * several routines share: it is assigned to the routine it influences most (premise 5 of
 * §IV: the kernel with the highest impact has priority). */
typedef struct screen_opts {
    int mode;
    int n_base;
    double h;
    double cutoff;
    int max_dims;
    uint64_t seed;
    double growth;     /* ROUTINE_SERIES */
    const double *lo;  /* ROUTINE_SERIES, host black box: parameter ranges (may be NULL) */
    const double *hi;
} screen_opts;

/* score: host, d x d (PAIRWISE) or R x d (ROUTINE; R = n_blocks or n_routines) FP64.
 * influence, group_of, fixed: host, d entries each.  n_groups: host scalar.
 * Any output may be NULL except group_of and n_groups.  Synchronises. */
int interdep_screen(gpbo_ctx *ctx, const gpbo_objective *obj, int d, const screen_opts *opts,
                    double *score, double *influence, int *group_of, int *n_groups, int *fixed);

/* ------------------------------------------------------------------ one BO step (§III-A)
 * z-score y (population std, 1 when zero), fit on (X, y'), score the M candidates (Xc, or
 * drawn from seed when Xc is NULL) with EI below tau = min y', and return the EI argmax:
 * x_next (host, d doubles), ei_max (host, standardised units), argmax (host, may be NULL).
 * flags: GPBO_HOST_PTRS applies to X, y and Xc.  The context keeps the step's model and
 * staging buffers for its next search_step of the same d and precision whose n pads to the
 * same size (a BO loop calls it with n growing by one), and frees them on any other shape
 * or in gpbo_destroy.  Synchronises. */
int search_step(gpbo_ctx *ctx, const double *X, const double *y, int n, int d, const gp_hyper *hyp,
                const float *Xc, int64_t M, uint64_t seed, double xi, gpbo_prec prec, unsigned flags,
                double *x_next, double *ei_max, int64_t *argmax);

/* ------------------------------------------------------------------ batched step (§IV-D)
 * G independent sub-searches -- the paper runs the independent and merged searches its
 * analysis produces in parallel (§IV-D) -- each of its own dimension d[g], size n[g] and
 * hyperparameters hyp[g], in one graph launch: every kernel of search_step covers all G
 * problems at once, with the same device code, so problem g's result equals search_step
 * on it bit for bit while n[g] pads to less than 1536 (search_step moves the Cholesky updates
 * and the large levels of L^-1 to the tensor cores from there on; larger problems agree
 * within the FP32 tolerances).  FP32 scoring only (GPBO_ENOTSUP otherwise); M[g] candidates
 * are drawn on the device from seed[g].
 *   X, y : host arrays of G pointers; the pointed-to data are device arrays (n[g] x d[g]
 *          and n[g]) unless flags has GPBO_HOST_PTRS.
 *   x_next : host, G x 64 doubles; row g holds the d[g] coordinates of problem g's pick.
 *   ei_max : host, G.  argmax : host, G, may be NULL.
 * The first call for a set of shapes (G, n, d, M, hyperparameters, xi) builds device arenas
 * and captures the step into CUDA graphs held by the context; later calls with the same
 * shapes take the new X, y and seeds and replay the graphs.  The problems that pad to at
 * most 512 rows form a second plan whose graph runs beside the larger problems' on a
 * lower-priority stream (its whole step under their factorisation); the split changes no
 * result.  Synchronises. */
int search_step_batched(gpbo_ctx *ctx, int G, const double *const *X, const double *const *y, const int *n,
                        const int *d, const gp_hyper *hyp, const int64_t *M, const uint64_t *seed, double xi,
                        gpbo_prec prec, unsigned flags, double *x_next, double *ei_max, int64_t *argmax);

/* Variance tile of the batched step (candidates per CTA of its FP32 variance kernel: 64,
 * 128 or 256), or 0 (the default) for the autotuner: when a call meets a new set of shapes it
 * times each tile on the plan's own buffers (one warm-up and three launches each) and
 * captures the fastest into the graph.  The tile changes no result: every candidate's sums
 * run in the same order.  Takes effect at the next search_step_batched call. */
int search_step_batched_tile(gpbo_ctx *ctx, int tile);
/* The tile of the plan that holds the largest problems of the last batched call, and the
 * autotuner's mean time per launch (ms) of its 64, 128 and 256 tiles (negative when not
 * measured).  members: NULL, or host room for that call's G ints, set to 1 for the problems
 * of that plan and 0 for the others.  GPBO_EINVAL before the first batched call. */
int search_step_batched_tuning(const gpbo_ctx *ctx, int *tile, float *ms3, int *members);

/* ------------------------------------------------------------------ learned pre-screen
 * Not in the paper: a cheap surrogate of the GP posterior that pre-screens very large
 * candidate pools so that the exact GP-EI (§III-A's acquisition) only scores the best k.
 * An ensemble of E networks d -> H -> H -> 2 with the exact GELU g(z) = z Phi(z) predicts
 * (mu, log sigma) in standardised units; members combine as mu_bar = mean mu_e and
 * sigma_bar^2 = mean sigma_e^2 + var mu_e.  Per-network parameters (FP32, contiguous):
 * W1 [d x H], b1 [H], W2 [H x H], b2 [H], W3 [H x 2], b3 [2] (weights input-major).
 * Training loss per network: L = 1/(2B) sum (o - t)^2; Adam (lr, 0.9, 0.999, 1e-8). */
typedef struct gpbo_mlp gpbo_mlp;
/* E networks, Glorot-uniform weights from counter stream 5 of seed, zero biases. */
int mlp_create(gpbo_ctx *ctx, int E, int d, int H, uint64_t seed, gpbo_mlp **out);
/* Free the networks; like models, before the context they were created on. */
int mlp_free(gpbo_mlp *net);
/* Read (host_out) and/or write (host_in) all E x P parameters, host FP32.  Synchronises. */
int mlp_params(gpbo_mlp *net, float *host_out, const float *host_in);
/* Outputs of every network on B device rows X (B x d): out device E x B x 2.  Synchronises. */
int mlp_forward(gpbo_ctx *ctx, gpbo_mlp *net, const float *X, int B, float *out);
/* Loss and gradient of every network on one batch (device X: B x d, T: B x 2 targets);
 * grads_host: E x P, loss_host: E (either may be NULL).  Synchronises. */
int mlp_gradients(gpbo_ctx *ctx, gpbo_mlp *net, const float *X, const float *T, int B, float *grads_host,
                  float *loss_host);
/* Train on N device rows: inputs X (N x d) and the GP posterior mu, sigma (N each).  The
 * targets are (mu, log sigma) standardised by their means and standard deviations over
 * the N rows (kept in the net for scoring).  `steps` Adam steps on minibatches of `batch`
 * rows drawn with replacement from counter stream 7 of seed.  final_loss: host, mean loss
 * of the last step over the networks (may be NULL).  Synchronises. */
int mlp_train(gpbo_ctx *ctx, gpbo_mlp *net, const float *X, const float *mu, const float *sigma, int64_t N, int steps,
              int batch, float lr, uint64_t seed, float *final_loss);
/* Target standardisation (mu mean, mu sd, log-sigma mean, log-sigma sd), host. */
int mlp_norm(const gpbo_mlp *net, double *norm4);
/* Ensemble scores of M candidates: rows of X (device, M x d FP32) or, with X = NULL,
 * candidates 0 .. M-1 drawn from seed (stream 2, as gpbo_gen_candidates draws them).
 * Writes device arrays of M floats: ei = EI(mu_bar, sigma_bar) below y_best (minimisation),
 * mu = mu_bar and sigma = sigma_bar (mu and sigma may be NULL).
 * prec GPBO_PREC_F32: FP32 forward on the CUDA cores (any d, H), exact GELU.
 * prec GPBO_PREC_F16: one tensor-core launch (tcgen05): FP16 inputs, first-layer weights,
 * first-layer activations and second-layer weights; FP32 accumulation, FP32 GELU in the
 * tanh form and FP32 from the second layer's output on; fused with the combine and the
 * EI.  Needs H = 256, d <= 31 and E <= 8, else GPBO_ENOTSUP.  GPBO_PREC_BF16: GPBO_ENOTSUP.
 * GPBO_ETIMEOUT if a bounded device wait gave up.  Synchronises. */
int mlp_score(gpbo_ctx *ctx, gpbo_mlp *net, const float *X, int64_t M, uint64_t seed, double y_best, double xi,
              int prec, float *ei, float *mu, float *sigma);
/* Draw M candidates from seed (stream 2), score them with the ensemble's EI below y_best
 * (the FP16 tensor-core path of mlp_score when H = 256, d <= 31 and E <= 8, else FP32),
 * keep the k best (radix select; ties at the k-th value taken in any order), re-score those
 * k with the exact GP-EI of `model` (FP32 or 16-bit scoring) and return the best pool index
 * and its exact EI.  ei_pool: device M floats for the surrogate EI, or NULL (then the call
 * allocates it); top_idx: host k pool indices of the selected set, or NULL.  Synchronises. */
int surrogate_screen(gpbo_ctx *ctx, const gp_model *model, gpbo_mlp *net, int64_t M, uint64_t seed, int k,
                     double y_best, double xi, float *ei_pool, int64_t *top_idx, int64_t *argmax, double *ei_max);

/* ------------------------------------------------------------------ a BO search (§III-A, §IV-D)
 * One Bayesian-optimisation search over k variables scaled into the unit cube: n_init initial
 * configurations (given: the caller draws them, 5 random ones in the paper), then one
 * search_step per evaluation until `budget` evaluations (the paper: 10 x k): standardise y,
 * fit, score M candidates drawn on the device from seed + t (gpbo_gen_candidates, t the
 * evaluation index), evaluate the EI argmax.  With refit = 1 each step first refits the
 * hyperparameters by gp_fit_mle on the standardised observations (box: lengthscales
 * 0.01..100, signal variance e^-3..e^3, noise variance e^-14..1; starts: the previous
 * step's fit, then hyp), at most mle_iters L-BFGS iterations (30 when 0); with refit = 0 the
 * hyperparameters are hyp throughout.  Fits use GPBO_JITTER.
 * fn: the objective, called on the host with one configuration u (k values in [0,1]); it
 * writes f and returns 0, nonzero for a failed evaluation (bo_search then returns
 * GPBO_EINVAL).  X (host, budget x k) and y (host, budget) receive every evaluated
 * configuration and value in order; best (host, may be NULL) the index of the smallest y. */
typedef int (*gpbo_eval_fn)(const double *u, int k, double *f, void *user);
typedef struct bo_opts {
    int budget;
    int n_init;
    const double *x_init; /* host, n_init x k, in [0,1] */
    int64_t M;
    uint64_t seed;
    int prec;             /* gpbo_prec of the scoring */
    int refit;
    gp_hyper hyp;
    double xi;
    int mle_iters;
} bo_opts;
int bo_search(gpbo_ctx *ctx, int k, gpbo_eval_fn fn, void *user, const bo_opts *opts, double *X, double *y,
              int *best);

/* ------------------------------------------------------------------ hyperparameters by maximum likelihood
 * The surrogate's hyperparameters theta = (log l_1 .. log l_d, log signal_var, log noise_var)
 * fitted by maximising the log marginal likelihood of the evaluated configurations (§III-A:
 * the surrogate is trained on them; Rasmussen & Williams 2006, §5.4.1):
 *   LML(theta)      = -1/2 y^T alpha - sum_i log L_ii - n/2 log(2 pi),   alpha = K^-1 y,
 *   dLML/dtheta_j   = 1/2 sum_pq (alpha_p alpha_q - [K^-1]_pq) dK_pq/dtheta_j,
 * with K, L and alpha as gp_fit computes them in FP64 (y used as given: zero prior mean) and
 * K^-1 = L^-T L^-1 formed tile by tile in FP64 and reduced into the gradient without being
 * stored.  For r the scaled distance and t_k = (x_k - x'_k) / l_k:
 *   dK/dlog l_k = s2 (5/3) (1 + sqrt5 r) exp(-sqrt5 r) t_k^2,  dK/dlog s2 = s2 m(r),
 *   dK/dlog sn2 = sn2 I.
 * X, y: n x d row-major and n FP64, device pointers or host with GPBO_HOST_PTRS.
 *
 * gp_lml: LML and its gradient (host, d + 2 values; grad may be NULL) at the hyperparameters
 * in hyp (noise_var > 0).  GPBO_ENOTSPD when K is not positive definite.  Synchronises. */
int gp_lml(gpbo_ctx *ctx, const double *X, const double *y, int n, int d, const gp_hyper *hyp, unsigned flags,
           double *lml, double *grad);
/* gp_fit_mle: maximise the LML over the box lo <= theta <= hi (host, d + 2 each) with a
 * projected L-BFGS (memory 10, Armijo backtracking) from each of n_starts starting points
 * theta0 (host, n_starts x (d + 2) row-major; the caller draws them, so the fit has no
 * randomness of its own).  Each start runs at most max_iter iterations and stops when the
 * projected gradient's largest component is at most gtol or the LML stops improving
 * (relative change 1e-12).  A trial point whose K is not positive definite is a rejected
 * step; a start whose own K is not is skipped.  Writes the best start's theta (host, d + 2),
 * its LML and the number of LML evaluations over all starts (evals may be NULL).
 * GPBO_ENOTSPD when no start could be factored.  Synchronises. */
int gp_fit_mle(gpbo_ctx *ctx, const double *X, const double *y, int n, int d, int n_starts, const double *theta0,
               const double *lo, const double *hi, int max_iter, double gtol, unsigned flags, double *theta_best,
               double *lml_best, int64_t *evals);

#ifdef __cplusplus
}
#endif
#endif /* GPBO_H */
