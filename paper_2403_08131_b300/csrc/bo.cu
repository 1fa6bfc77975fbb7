// One Bayesian-optimisation search, the loop every independent or merged sub-search runs
// (§III-A: a surrogate trained on the configurations evaluated so far, an acquisition
// choosing the next one; §IV-D: 5 random initial configurations, then a fixed budget of
// evaluations).  Each iteration is a search_step (standardise, fit, score the candidates
// drawn on the device, EI argmax); with refit the GP hyperparameters are first refitted by
// maximum marginal likelihood (gp_fit_mle) on the standardised observations, warm-started
// from the previous iteration's.  The objective is the caller's black box, called on the host
// with one configuration at a time (in the paper: a run of the tuned application).

#include "gpbo_internal.cuh"
#include "gpbo.h"

#include <cmath>
#include <vector>

extern "C" {

int bo_search(gpbo_ctx *ctx, int k, gpbo_eval_fn fn, void *user, const bo_opts *o, double *X, double *y, int *best)
{
    if (!ctx || !fn || !o || !X || !y || k < 1 || k > GPBO_MAX_D || o->budget < 1 || o->budget > GPBO_MAX_N ||
        o->n_init < 1 || o->n_init > o->budget || !o->x_init || o->M < 1 || o->M > 0x7fffffffll)
        return GPBO_EINVAL;
    if (o->prec < GPBO_PREC_F64 || o->prec > GPBO_PREC_F16) return GPBO_EINVAL;
    if (!o->hyp.lengthscale || o->hyp.d != k) return GPBO_EINVAL;
    for (int i = 0; i < o->n_init * k; ++i)
        if (!(o->x_init[i] >= 0.0 && o->x_init[i] <= 1.0)) return GPBO_EINVAL;
    // initial design
    for (int e = 0; e < o->n_init; ++e) {
        for (int j = 0; j < k; ++j) X[(size_t)e * k + j] = o->x_init[(size_t)e * k + j];
        if (fn(X + (size_t)e * k, k, y + e, user) != 0 || !std::isfinite(y[e])) return GPBO_EINVAL;
    }
    std::vector<double> ls(o->hyp.lengthscale, o->hyp.lengthscale + k), ys, theta(k + 2), prev, lo(k + 2),
        hi(k + 2), starts;
    double s2 = o->hyp.signal_var, sn2 = o->hyp.noise_var;
    // the refit's box of log parameters: lengthscales 0.01..100, signal e^-3..e^3, noise e^-14..1
    for (int j = 0; j < k; ++j) {
        lo[j] = std::log(0.01);
        hi[j] = std::log(100.0);
    }
    lo[k] = -3.0;
    hi[k] = 3.0;
    lo[k + 1] = -14.0;
    hi[k + 1] = 0.0;
    std::vector<double> x_next(k);
    for (int t = o->n_init; t < o->budget; ++t) {
        const int n = t;
        if (o->refit) {
            // y standardised as search_step does it (population std, 1 when zero)
            double mean = 0.0, var = 0.0;
            for (int i = 0; i < n; ++i) mean += y[i];
            mean /= n;
            for (int i = 0; i < n; ++i) var += (y[i] - mean) * (y[i] - mean);
            const double sd = var > 0.0 ? std::sqrt(var / n) : 1.0;
            ys.resize(n);
            for (int i = 0; i < n; ++i) ys[i] = (y[i] - mean) / sd;
            starts.clear();
            if (!prev.empty()) starts.insert(starts.end(), prev.begin(), prev.end());
            for (int j = 0; j < k; ++j) starts.push_back(std::log(o->hyp.lengthscale[j]));
            starts.push_back(std::log(o->hyp.signal_var));
            starts.push_back(std::log(std::fmax(o->hyp.noise_var, 1e-6)));
            for (size_t i = 0; i < starts.size(); ++i) {
                const int q = (int)(i % (size_t)(k + 2));
                starts[i] = std::fmin(std::fmax(starts[i], lo[q]), hi[q]);
            }
            double lml = 0.0;
            const int st = gp_fit_mle(ctx, X, ys.data(), n, k, (int)(starts.size() / (k + 2)), starts.data(), lo.data(),
                                      hi.data(), o->mle_iters > 0 ? o->mle_iters : 30, 1e-5, GPBO_HOST_PTRS,
                                      theta.data(), &lml, nullptr);
            if (st == GPBO_OK) {
                for (int j = 0; j < k; ++j) ls[j] = std::exp(theta[j]);
                s2 = std::exp(theta[k]);
                sn2 = std::exp(theta[k + 1]);
                prev = theta;
            } else if (st != GPBO_ENOTSPD) {
                return st;
            }  // no start could be factored: keep the previous hyperparameters
        }
        gp_hyper h = {k, ls.data(), s2, sn2};
        double ei = 0.0;
        int64_t am = -1;
        const int st = search_step(ctx, X, y, n, k, &h, nullptr, o->M, o->seed + (uint64_t)t, o->xi, (gpbo_prec)o->prec,
                                   GPBO_HOST_PTRS | GPBO_JITTER, x_next.data(), &ei, &am);
        if (st != GPBO_OK) return st;
        for (int j = 0; j < k; ++j) X[(size_t)t * k + j] = x_next[j];
        if (fn(X + (size_t)t * k, k, y + t, user) != 0 || !std::isfinite(y[t])) return GPBO_EINVAL;
    }
    if (best) {
        int b = 0;
        for (int e = 1; e < o->budget; ++e)
            if (y[e] < y[b]) b = e;
        *best = b;
    }
    return GPBO_OK;
}

}  // extern "C"
