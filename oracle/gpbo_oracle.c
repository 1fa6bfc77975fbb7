/*
 * gpbo_oracle.c -- plain FP64 CPU oracle for the GP-BO hot path of
 * "Cost-Effective Methodology for Complex Tuning Searches in HPC" (arXiv 2403.08131).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct statement of
 * what the GPU library computes.  Only the test suite, the smoke check and the
 * bench's CPU-baseline leg may load it.  It shares no code, header, table or
 * constant generator with the CUDA library, and it includes nothing from it.
 *
 * What follows the paper directly:
 *   - surrogate trained on evaluated configurations, acquisition picks the next one,
 *     evaluate, retrain (§III-A, Bayesian Optimization)               -> search_step
 *   - first-order sensitivity score (1/V) * sum |(t_base - t_i)/t_base| (§IV-B)
 *                                                                      -> screen_routine
 *   - per-routine sensitivity, DAG with parameters as edges, pruning by a
 *     cut-off, merging of linked routines (§IV-C, §IV-D)              -> partition_*
 *   - at most 10 parameters per search, keeping the most influential (§IV, premise 4;
 *     §IV-D)                                                           -> cap in partition_*
 * What the paper leaves to GPTune and this oracle takes from the textbook:
 *   - Matern nu=5/2 ARD covariance (Rasmussen & Williams 2006, eq. 4.17)
 *   - Cholesky-Banachiewicz factorisation, forward/back substitution
 *   - GP posterior mean and latent variance (Rasmussen & Williams 2006, Alg. 2.1)
 *   - expected improvement for minimisation (Jones, Schonlau, Welch 1998)
 *   - the pairwise mixed-difference screen (the classical second-order route the
 *     paper contrasts with in §II and §IV-C)
 * Readings of silent points (noise draw, base-point range, score normalisation,
 * tie rules) are the ones the design document lists; each is restated at its use.
 *
 * Parity pins: every function here is checked by tests/test_oracle_pins.py against
 * closed forms, library routines (numpy, scipy, scikit-learn) or brute force.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOTSPD 2
#define ORC_ENAN 3
#define ORC_ENOMEM 4

static const double ORC_PI = 3.14159265358979323846;
static const double ORC_E = 2.71828182845904523536;

/* ------------------------------------------------------------------ RNG
 * SplitMix64 (Steele, Lea, Flood 2014): state advances by the golden gamma and each
 * output is the 64-bit finaliser of the state.  Used counter-style: output number
 * `counter` (0-based) of the generator seeded with seed ^ (stream * gamma). */
static const uint64_t ORC_GAMMA = 0x9E3779B97F4A7C15ULL;

uint64_t orc_splitmix64(uint64_t seed, uint64_t stream, uint64_t counter)
{
    uint64_t z = (seed ^ (stream * ORC_GAMMA)) + (counter + 1) * ORC_GAMMA;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

double orc_uniform24(uint64_t seed, uint64_t stream, uint64_t counter)
{
    return (double)(orc_splitmix64(seed, stream, counter) >> 40) * (1.0 / 16777216.0);
}

/* Box-Muller on the draws 2c and 2c+1; u1 in (0,1], u2 in [0,1). */
double orc_normal(uint64_t seed, uint64_t stream, uint64_t counter)
{
    double u1 = ((double)(orc_splitmix64(seed, stream, 2 * counter) >> 11) + 1.0) * ldexp(1.0, -53);
    double u2 = (double)(orc_splitmix64(seed, stream, 2 * counter + 1) >> 11) * ldexp(1.0, -53);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * ORC_PI * u2);
}

/* count x d uniform points, point p coordinate k at counter (first+p)*d + k. */
void orc_uniform_points(uint64_t seed, uint64_t stream, int64_t first, int64_t count, int d, double *out)
{
    for (int64_t p = 0; p < count; ++p)
        for (int k = 0; k < d; ++k)
            out[p * d + k] = orc_uniform24(seed, stream, (uint64_t)((first + p) * d + k));
}

/* ------------------------------------------------------------------ objectives
 * Synthetic black boxes: additive blocks of Ackley, Rastrigin and (chained)
 * Rosenbrock, each on the affine image of [0,1]^m in its customary domain.  The
 * paper builds its 20-D test function from additive groups in the same way (§III-C). */
enum { ORC_ACKLEY = 0, ORC_RASTRIGIN = 1, ORC_ROSENBROCK = 2 };

double orc_block_value(int fn, const double *x01, int m)
{
    double lo, hi;
    if (fn == ORC_ACKLEY) { lo = -32.768; hi = 32.768; }
    else if (fn == ORC_RASTRIGIN) { lo = -5.12; hi = 5.12; }
    else { lo = -2.0; hi = 2.0; }
    double z[64];
    for (int k = 0; k < m; ++k) z[k] = lo + (hi - lo) * x01[k];
    if (fn == ORC_ACKLEY) {
        double sq = 0.0, cs = 0.0;
        for (int k = 0; k < m; ++k) { sq += z[k] * z[k]; cs += cos(2.0 * ORC_PI * z[k]); }
        return -20.0 * exp(-0.2 * sqrt(sq / m)) - exp(cs / m) + 20.0 + ORC_E;
    }
    if (fn == ORC_RASTRIGIN) {
        double s = 10.0 * m;
        for (int k = 0; k < m; ++k) s += z[k] * z[k] - 10.0 * cos(2.0 * ORC_PI * z[k]);
        return s;
    }
    double s = 0.0;
    for (int k = 0; k + 1 < m; ++k) {
        double a = z[k + 1] - z[k] * z[k], b = 1.0 - z[k];
        s += 100.0 * a * a + b * b;
    }
    return s;
}

/* Evaluate every block at x; f_routines[b] = block b's value plus its own noise draw
 * (when routine noise is requested), f_total = sum of blocks + one noise draw.
 * noise counters: total uses `counter`, block b uses counter*nb + b (caller picks). */
void orc_objective(int nb, const int *bdim, const int *bfn, const double *x,
                   double *f_routines, double *f_total)
{
    int o = 0;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) {
        double v = orc_block_value(bfn[b], x + o, bdim[b]);
        if (f_routines) f_routines[b] = v;
        s += v;
        o += bdim[b];
    }
    if (f_total) *f_total = s;
}

/* ------------------------------------------------------------------ GP pieces
 * Matern nu=5/2: m(r) = (1 + sqrt5 r + 5 r^2 / 3) exp(-sqrt5 r). */
double orc_matern52(double r)
{
    double s5r = sqrt(5.0) * r;
    return (1.0 + s5r + 5.0 * r * r / 3.0) * exp(-s5r);
}

/* Scaled distance r = sqrt(sum_k ((a_k - b_k)/l_k)^2), difference form. */
double orc_scaled_dist(const double *a, const double *b, int d, const double *ls)
{
    double s = 0.0;
    for (int k = 0; k < d; ++k) { double t = (a[k] - b[k]) / ls[k]; s += t * t; }
    return sqrt(s);
}

/* K_ij = s2 m(r_ij) + sn2 [i == j], full n x n row-major. */
void orc_kmat(const double *X, int n, int d, const double *ls, double s2, double sn2, double *K)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double v = s2 * orc_matern52(orc_scaled_dist(X + (size_t)i * d, X + (size_t)j * d, d, ls));
            K[(size_t)i * n + j] = v + (i == j ? sn2 : 0.0);
        }
}

/* Cholesky-Banachiewicz, row by row: K = L L^T, L lower with zeros above. */
int orc_cholesky(const double *K, int n, double *L)
{
    memset(L, 0, sizeof(double) * (size_t)n * n);
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = K[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) s -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            if (i == j) {
                if (!(s > 0.0)) return ORC_ENOTSPD;
                L[(size_t)i * n + i] = sqrt(s);
            } else {
                L[(size_t)i * n + j] = s / L[(size_t)j * n + j];
            }
        }
    }
    return ORC_OK;
}

/* L x = b (forward substitution). */
void orc_forward(const double *L, int n, const double *b, double *x)
{
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * x[k];
        x[i] = s / L[(size_t)i * n + i];
    }
}

/* L^T x = b (back substitution on the transpose). */
void orc_backward_t(const double *L, int n, const double *b, double *x)
{
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * x[k];
        x[i] = s / L[(size_t)i * n + i];
    }
}

/* L^{-1} by forward substitution on the unit vectors (column by column). */
void orc_tri_inverse(const double *L, int n, double *Linv)
{
    double *e = (double *)calloc((size_t)n, sizeof(double));
    double *c = (double *)malloc(sizeof(double) * (size_t)n);
    for (int j = 0; j < n; ++j) {
        memset(e, 0, sizeof(double) * (size_t)n);
        e[j] = 1.0;
        orc_forward(L, n, e, c);
        for (int i = 0; i < n; ++i) Linv[(size_t)i * n + j] = c[i];
    }
    free(e);
    free(c);
}

/* Fit with fixed hyperparameters: K, L, alpha = K^{-1} y by two triangular solves,
 * then one refinement step r = y - K alpha (unfactored K), alpha += K^{-1} r.
 * Outputs L (n x n) and alpha (n); K is scratch supplied by the caller (n x n). */
int orc_gp_fit(const double *X, const double *y, int n, int d, const double *ls, double s2, double sn2,
               double *K, double *L, double *alpha)
{
    if (n <= 0 || d <= 0) return ORC_EINVAL;
    for (int i = 0; i < n; ++i) if (!isfinite(y[i])) return ORC_ENAN;
    for (int64_t i = 0; i < (int64_t)n * d; ++i) if (!isfinite(X[i])) return ORC_ENAN;
    orc_kmat(X, n, d, ls, s2, sn2, K);
    int st = orc_cholesky(K, n, L);
    if (st) return st;
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *dl = (double *)malloc(sizeof(double) * (size_t)n);
    orc_forward(L, n, y, z);
    orc_backward_t(L, n, z, alpha);
    for (int i = 0; i < n; ++i) {
        double s = y[i];
        for (int j = 0; j < n; ++j) s -= K[(size_t)i * n + j] * alpha[j];
        r[i] = s;
    }
    orc_forward(L, n, r, z);
    orc_backward_t(L, n, z, dl);
    for (int i = 0; i < n; ++i) alpha[i] += dl[i];
    free(z); free(r); free(dl);
    return ORC_OK;
}

/* Posterior of the latent f at M candidates: k*_i = s2 m(r(x*, x_i)); mu = k*^T alpha;
 * v = L^{-1} k* by forward substitution; sigma^2 = max(s2 - v^T v, 0). */
void orc_posterior(const double *X, int n, int d, const double *ls, double s2,
                   const double *L, const double *alpha, const double *Xc, int64_t M,
                   double *mu, double *sigma)
{
#pragma omp parallel
    {
        double *ks = (double *)malloc(sizeof(double) * (size_t)n);
        double *v = (double *)malloc(sizeof(double) * (size_t)n);
#pragma omp for schedule(static)
        for (int64_t c = 0; c < M; ++c) {
            const double *xc = Xc + c * d;
            double m = 0.0;
            for (int i = 0; i < n; ++i) {
                ks[i] = s2 * orc_matern52(orc_scaled_dist(xc, X + (size_t)i * d, d, ls));
                m += ks[i] * alpha[i];
            }
            orc_forward(L, n, ks, v);
            double q = 0.0;
            for (int i = 0; i < n; ++i) q += v[i] * v[i];
            double var = s2 - q;
            if (var < 0.0) var = 0.0;
            mu[c] = m;
            sigma[c] = sqrt(var);
        }
        free(ks);
        free(v);
    }
}

/* Expected improvement below the incumbent tau (minimisation), margin xi.
 * imp = tau - mu - xi; EI = imp Phi(imp/sigma) + sigma phi(imp/sigma); sigma = 0 -> max(imp, 0). */
double orc_ei(double mu, double sigma, double tau, double xi)
{
    double imp = tau - mu - xi;
    if (!(sigma > 0.0)) return imp > 0.0 ? imp : 0.0;
    double z = imp / sigma;
    double Phi = 0.5 * erfc(-z / sqrt(2.0));
    double phi = exp(-0.5 * z * z) / sqrt(2.0 * ORC_PI);
    return imp * Phi + sigma * phi;
}

void orc_ei_batch(const double *mu, const double *sigma, int64_t M, double tau, double xi, double *ei)
{
    for (int64_t c = 0; c < M; ++c) ei[c] = orc_ei(mu[c], sigma[c], tau, xi);
}

/* First index of the largest value (strict > scan, so ties go to the lowest index). */
int64_t orc_argmax(const double *v, int64_t M)
{
    int64_t best = 0;
    for (int64_t c = 1; c < M; ++c) if (v[c] > v[best]) best = c;
    return best;
}

/* z-score with the population standard deviation; a zero spread divides by 1. */
void orc_standardize(const double *y, int n, double *ys, double *mean_out, double *std_out)
{
    double m = 0.0;
    for (int i = 0; i < n; ++i) m += y[i];
    m /= n;
    double v = 0.0;
    for (int i = 0; i < n; ++i) v += (y[i] - m) * (y[i] - m);
    double s = sqrt(v / n);
    if (!(s > 0.0)) s = 1.0;
    for (int i = 0; i < n; ++i) ys[i] = (y[i] - m) / s;
    if (mean_out) *mean_out = m;
    if (std_out) *std_out = s;
}

/* One BO iteration (§III-A): standardise y, fit, score the candidates (given, or drawn
 * from stream 2 of `seed` when Xc is NULL), take the EI argmax, return that point.
 * tau is the smallest standardised observation.  mu/sigma/ei may be NULL. */
int orc_search_step(const double *X, const double *y, int n, int d, const double *ls, double s2, double sn2,
                    const double *Xc_in, int64_t M, uint64_t seed, double xi,
                    double *x_next, double *ei_max, int64_t *argmax,
                    double *mu_out, double *sigma_out, double *ei_out)
{
    if (n <= 0 || d <= 0 || M <= 0) return ORC_EINVAL;
    double *ys = (double *)malloc(sizeof(double) * (size_t)n);
    double *K = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *L = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *alpha = (double *)malloc(sizeof(double) * (size_t)n);
    double *Xc = (double *)Xc_in;
    if (!Xc_in) {
        Xc = (double *)malloc(sizeof(double) * (size_t)M * d);
        orc_uniform_points(seed, 2, 0, M, d, Xc);
    }
    double *mu = mu_out ? mu_out : (double *)malloc(sizeof(double) * (size_t)M);
    double *sg = sigma_out ? sigma_out : (double *)malloc(sizeof(double) * (size_t)M);
    double *ei = ei_out ? ei_out : (double *)malloc(sizeof(double) * (size_t)M);
    orc_standardize(y, n, ys, NULL, NULL);
    int st = orc_gp_fit(X, ys, n, d, ls, s2, sn2, K, L, alpha);
    if (st == ORC_OK) {
        double tau = ys[0];
        for (int i = 1; i < n; ++i) if (ys[i] < tau) tau = ys[i];
        orc_posterior(X, n, d, ls, s2, L, alpha, Xc, M, mu, sg);
        orc_ei_batch(mu, sg, M, tau, xi, ei);
        int64_t a = orc_argmax(ei, M);
        for (int k = 0; k < d; ++k) x_next[k] = Xc[a * d + k];
        *ei_max = ei[a];
        if (argmax) *argmax = a;
    }
    if (!Xc_in) free(Xc);
    if (!mu_out) free(mu);
    if (!sigma_out) free(sg);
    if (!ei_out) free(ei);
    free(ys); free(K); free(L); free(alpha);
    return st;
}

/* ------------------------------------------------------------------ screens
 * Base points b_k: b_k,t = (1 - h) * u(k*d + t) with u uniform on stream 3, so that
 * b + h e_i + h e_j stays in the unit box.
 * Pairwise evaluation e of base k: e = 0 base; e = 1+i single step along i;
 * e = 1+d+p(i,j) double step along i and j (p = lexicographic pair index, i<j).
 * Noise (stream 4): total f of evaluation e at base k adds noise_sd * N(counter k*E + e),
 * E = 1 + d + d(d-1)/2. */
static int64_t pair_index(int i, int j, int d) { return (int64_t)i * d - (int64_t)i * (i + 1) / 2 + (j - i - 1); }

static void screen_point(const double *b, int d, int i, int j, double h, double *x)
{
    for (int t = 0; t < d; ++t) x[t] = b[t];
    if (i >= 0) x[i] = b[i] + h;
    if (j >= 0) x[j] = b[j] + h;
}

/* PAIRWISE screen.
 *   delta_ijk = f(b+he_i+he_j) - f(b+he_i) - f(b+he_j) + f(b)
 *   score_ij  = mean_k |delta_ijk| / (mean_k(|f(b+he_i)-f(b)| + |f(b+he_j)-f(b)|) + 1e-12)
 *   sens_i    = mean_k |f(b+he_i) - f(b)| / (|f(b)| + 1e-12)     (the §IV-B score, V = n_base)
 * score is d x d symmetric with a zero diagonal. */
int orc_screen_pairwise(int nb, const int *bdim, const int *bfn, double noise_sd, uint64_t seed,
                        int d, int n_base, double h, double *score, double *sens)
{
    int sum = 0;
    for (int b = 0; b < nb; ++b) sum += bdim[b];
    if (sum != d || d < 1 || d > 64 || n_base < 1) return ORC_EINVAL;
    const int64_t P = (int64_t)d * (d - 1) / 2, E = 1 + d + P;
    double *fv = (double *)malloc(sizeof(double) * (size_t)(n_base * E));
#pragma omp parallel for schedule(static)
    for (int k = 0; k < n_base; ++k) {
        double b[64], x[64];
        for (int t = 0; t < d; ++t) b[t] = (1.0 - h) * orc_uniform24(seed, 3, (uint64_t)k * d + t);
        for (int64_t e = 0; e < E; ++e) {
            int i = -1, j = -1;
            if (e >= 1 && e <= d) i = (int)e - 1;
            else if (e > d) {
                int64_t p = e - 1 - d;
                for (int a = 0; a < d; ++a)
                    for (int c = a + 1; c < d; ++c)
                        if (pair_index(a, c, d) == p) { i = a; j = c; }
            }
            screen_point(b, d, i, j, h, x);
            double f;
            orc_objective(nb, bdim, bfn, x, NULL, &f);
            if (noise_sd > 0.0) f += noise_sd * orc_normal(seed, 4, (uint64_t)(k * E + e));
            fv[k * E + e] = f;
        }
    }
    for (int i = 0; i < d; ++i) {
        double s = 0.0;
        for (int k = 0; k < n_base; ++k) {
            const double *F = fv + k * E;
            s += fabs(F[1 + i] - F[0]) / (fabs(F[0]) + 1e-12);
        }
        sens[i] = s / n_base;
    }
    for (int i = 0; i < d; ++i) {
        score[i * d + i] = 0.0;
        for (int j = i + 1; j < d; ++j) {
            double num = 0.0, den = 0.0;
            for (int k = 0; k < n_base; ++k) {
                const double *F = fv + k * E;
                double dij = F[1 + d + pair_index(i, j, d)] - F[1 + i] - F[1 + j] + F[0];
                num += fabs(dij);
                den += fabs(F[1 + i] - F[0]) + fabs(F[1 + j] - F[0]);
            }
            double v = (num / n_base) / (den / n_base + 1e-12);
            score[i * d + j] = v;
            score[j * d + i] = v;
        }
    }
    free(fv);
    return ORC_OK;
}

/* ROUTINE screen (§IV-B formula applied per routine output, §IV-C):
 *   S_gi = mean_k |(f_g(b_k) - f_g(b_k + h e_i)) / f_g(b_k)|   (denominator |f_g| + 1e-12)
 * Routine outputs are the block values; each routine output of evaluation e at base k
 * adds its own noise draw noise_sd * N(counter (k*(1+d) + e)*R + g).  S is R x d. */
int orc_screen_routine(int nb, const int *bdim, const int *bfn, double noise_sd, uint64_t seed,
                       int d, int n_base, double h, double *S)
{
    int sum = 0;
    for (int b = 0; b < nb; ++b) sum += bdim[b];
    if (sum != d || d < 1 || d > 64 || n_base < 1 || nb < 1 || nb > 64) return ORC_EINVAL;
    const int R = nb, E = 1 + d;
    double *fv = (double *)malloc(sizeof(double) * (size_t)n_base * E * R);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < n_base; ++k) {
        double b[64], x[64];
        for (int t = 0; t < d; ++t) b[t] = (1.0 - h) * orc_uniform24(seed, 3, (uint64_t)k * d + t);
        for (int e = 0; e < E; ++e) {
            screen_point(b, d, e - 1, -1, h, x);
            double *fr = fv + ((size_t)k * E + e) * R;
            orc_objective(nb, bdim, bfn, x, fr, NULL);
            if (noise_sd > 0.0)
                for (int g = 0; g < R; ++g)
                    fr[g] += noise_sd * orc_normal(seed, 4, (uint64_t)(((int64_t)k * E + e) * R + g));
        }
    }
    for (int g = 0; g < R; ++g)
        for (int i = 0; i < d; ++i) {
            double s = 0.0;
            for (int k = 0; k < n_base; ++k) {
                double f0 = fv[((size_t)k * E + 0) * R + g];
                double fi = fv[((size_t)k * E + 1 + i) * R + g];
                s += fabs((f0 - fi) / (fabs(f0) + 1e-12));
            }
            S[g * d + i] = s / n_base;
        }
    free(fv);
    return ORC_OK;
}

/* ------------------------------------------------------------------ partition
 * Union-find in which the smaller root wins, so every label is its group's smallest
 * member.  The 10-dimension cap (§IV-D): a group larger than max_dims keeps its
 * max_dims most influential members (larger `influence` first, ties to the lower
 * index) and marks the others fixed (they take default values in the search). */
static int uf_find(int *parent, int a) { while (parent[a] != a) a = parent[a]; return a; }
static void uf_union(int *parent, int a, int b)
{
    int ra = uf_find(parent, a), rb = uf_find(parent, b);
    if (ra == rb) return;
    if (ra < rb) parent[rb] = ra; else parent[ra] = rb;
}

static void apply_cap(int d, const int *group_of, const double *influence, int max_dims, int *fixed)
{
    for (int i = 0; i < d; ++i) fixed[i] = 0;
    if (max_dims <= 0) return;
    for (int g = 0; g < d; ++g) {
        int size = 0;
        for (int i = 0; i < d; ++i) size += group_of[i] == g;
        if (size <= max_dims) continue;
        /* rank of member i = number of members that beat it */
        for (int i = 0; i < d; ++i) {
            if (group_of[i] != g) continue;
            int rank = 0;
            for (int j = 0; j < d; ++j) {
                if (group_of[j] != g || j == i) continue;
                if (influence[j] > influence[i] || (influence[j] == influence[i] && j < i)) rank++;
            }
            if (rank >= max_dims) fixed[i] = 1;
        }
    }
}

/* PAIRWISE partition: edge i-j when score_ij > cutoff. */
int orc_partition_pairwise(const double *score, int d, double cutoff, int max_dims, const double *influence,
                           int *group_of, int *n_groups, int *fixed)
{
    int parent[64];
    if (d < 1 || d > 64) return ORC_EINVAL;
    for (int i = 0; i < d; ++i) parent[i] = i;
    for (int i = 0; i < d; ++i)
        for (int j = i + 1; j < d; ++j)
            if (score[i * d + j] > cutoff) uf_union(parent, i, j);
    int ng = 0;
    for (int i = 0; i < d; ++i) { group_of[i] = uf_find(parent, i); ng += group_of[i] == i; }
    *n_groups = ng;
    apply_cap(d, group_of, influence, max_dims, fixed);
    return ORC_OK;
}

/* ROUTINE partition (§IV-C): vertices are routines; parameter i (owned by routine
 * owner[i]) links its owner to every routine g with S_gi > cutoff.  Linked routines
 * merge; a parameter's group is its merged routine set, labelled by the smallest
 * parameter index in it.  influence_i = max_g S_gi feeds the cap. */
int orc_partition_routine(const double *S, int R, int d, const int *owner, double cutoff, int max_dims,
                          int *group_of, int *n_groups, int *fixed)
{
    int rparent[64];
    double infl[64];
    if (d < 1 || d > 64 || R < 1 || R > 64) return ORC_EINVAL;
    for (int g = 0; g < R; ++g) rparent[g] = g;
    for (int i = 0; i < d; ++i) {
        if (owner[i] < 0 || owner[i] >= R) return ORC_EINVAL;
        infl[i] = 0.0;
        for (int g = 0; g < R; ++g) {
            double s = S[g * d + i];
            if (s > infl[i]) infl[i] = s;
            if (g != owner[i] && s > cutoff) uf_union(rparent, owner[i], g);
        }
    }
    /* label each parameter by the smallest parameter index in its merged routine set */
    for (int i = 0; i < d; ++i) {
        int ri = uf_find(rparent, owner[i]);
        int lab = i;
        for (int j = 0; j < i; ++j)
            if (uf_find(rparent, owner[j]) == ri) { lab = j; break; }
        group_of[i] = lab;
    }
    int ng = 0;
    for (int i = 0; i < d; ++i) ng += group_of[i] == i;
    *n_groups = ng;
    apply_cap(d, group_of, infl, max_dims, fixed);
    return ORC_OK;
}
