// Interdependence screen (§IV-B..D): which parameters, or which routines, must be
// searched together.
//
// ROUTINE mode follows the paper: a first-order sensitivity score per routine output,
// (1/V) sum |(f_base - f_i)/f_base| (§IV-B), with V = n_base random base points each
// varied by +h along one parameter; a parameter of routine A whose score on routine B
// exceeds the cut-off links A and B (§IV-C, the DAG with parameters as edges and the
// cut-off pruning); linked routines merge; a merged search above max_dims keeps its most
// influential parameters (§IV-D and premise 4 of §IV).
// ROUTINE_SERIES mode takes the paper's own schedule for the synthetic functions (§IV-B):
// one random baseline, then V variations of each parameter in turn, each 10% (growth) above
// the one before in the parameter's own units, clamped to its range; the same score and
// merge.  A parameter shared by several routines (owner -1) goes to the routine it
// influences most (§IV, premise 5).
// PAIRWISE mode is the classical second-order screen: mixed differences over all d(d-1)/2
// parameter pairs at the same base points.
//
// Device work: one thread per (base point, evaluation) evaluates the objective; one
// thread per score entry reduces over base points.  The union-find and the cap run on
// the host on the d x d (or R x d) score matrix.
#include "gpbo_internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace gpbo {

struct ObjSpec {
    int nb;
    int dim[GPBO_MAX_D];
    int fn[GPBO_MAX_D];
};

constexpr double PI_D = 3.14159265358979323846;
constexpr double E_D = 2.71828182845904523536;

__device__ double block_value(int fn, const double *x, int m)
{
    double lo, hi;
    if (fn == GPBO_FN_ACKLEY) { lo = -32.768; hi = 32.768; }
    else if (fn == GPBO_FN_RASTRIGIN) { lo = -5.12; hi = 5.12; }
    else { lo = -2.0; hi = 2.0; }
    const double w = hi - lo;
    if (fn == GPBO_FN_ACKLEY) {
        double q = 0.0, c = 0.0;
        for (int k = 0; k < m; ++k) {
            double z = lo + w * x[k];
            q += z * z;
            c += cos(2.0 * PI_D * z);
        }
        return -20.0 * exp(-0.2 * sqrt(q / m)) - exp(c / m) + 20.0 + E_D;
    }
    if (fn == GPBO_FN_RASTRIGIN) {
        double s = 10.0 * m;
        for (int k = 0; k < m; ++k) {
            double z = lo + w * x[k];
            s += z * z - 10.0 * cos(2.0 * PI_D * z);
        }
        return s;
    }
    double s = 0.0;
    for (int k = 0; k + 1 < m; ++k) {
        double z0 = lo + w * x[k], z1 = lo + w * x[k + 1];
        double a = z1 - z0 * z0, b = 1.0 - z0;
        s += 100.0 * a * a + b * b;
    }
    return s;
}

__device__ double normal_draw(uint64_t seed, uint64_t counter)
{
    // Box-Muller on draws 2c and 2c+1 of stream 4: u1 in (0,1], u2 in [0,1)
    double u1 = ((double)(splitmix64(seed, 4, 2 * counter) >> 11) + 1.0) * 0x1.0p-53;
    double u2 = (double)(splitmix64(seed, 4, 2 * counter + 1) >> 11) * 0x1.0p-53;
    return sqrt(-2.0 * log(u1)) * cos(2.0 * PI_D * u2);
}

// Which axes evaluation e perturbs: e = 0 none, 1..d one axis, then pairs i<j in order.
__device__ void eval_axes(int64_t e, int d, int &i, int &j)
{
    i = -1;
    j = -1;
    if (e == 0) return;
    if (e <= d) { i = (int)e - 1; return; }
    int64_t p = e - 1 - d;
    int a = 0;
    while (p >= d - 1 - a) { p -= d - 1 - a; ++a; }
    i = a;
    j = a + 1 + (int)p;
}

__device__ void base_point(uint64_t seed, int k, int d, double h, double *x)
{
    for (int t = 0; t < d; ++t) x[t] = (1.0 - h) * uniform24d(seed, 3, (uint64_t)k * d + t);
}

// Variation v (1..V) of one coordinate in the series schedule: the baseline's value in the
// parameter's units, grown by (1 + growth) v times in turn, clamped to [lo, hi], back in the
// unit interval.  Host and device take the same steps.
__host__ __device__ inline double series_value(double u0, double lo, double hi, double growth, int v)
{
    double x = lo + (hi - lo) * u0;
    for (int s = 0; s < v; ++s) x *= 1.0 + growth;
    x = fmin(fmax(x, lo), hi);
    return (x - lo) / (hi - lo);
}

struct SeriesRange {
    double lo[GPBO_MAX_D], hi[GPBO_MAX_D];
};

// Evaluation e = 0 is the baseline (point 0 of stream 3), e = 1 + i V + (v - 1) varies
// parameter i for the v-th time.  Outputs f[e R + g]; the noise of output g of evaluation e
// uses counter e R + g.
__global__ void k_screen_eval_series(ObjSpec spec, SeriesRange rg, int d, int V, double growth, uint64_t seed,
                                     double noise_sd, double *__restrict__ f)
{
    const int R = spec.nb;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= 1 + (int64_t)d * V) return;
    double x[GPBO_MAX_D];
    for (int k = 0; k < d; ++k) x[k] = uniform24d(seed, 3, (uint64_t)k);
    if (t > 0) {
        const int i = (int)((t - 1) / V), v = (int)((t - 1) % V) + 1;
        x[i] = series_value(x[i], rg.lo[i], rg.hi[i], growth, v);
    }
    int o = 0;
    for (int g = 0; g < R; ++g) {
        double val = block_value(spec.fn[g], x + o, spec.dim[g]);
        o += spec.dim[g];
        if (noise_sd > 0.0) val += noise_sd * normal_draw(seed, (uint64_t)(t * R + g));
        f[t * R + g] = val;
    }
}

// S_gi = (1/V) sum_v |(f_g(base) - f_g(variation v of i)) / f_g(base)|.
__global__ void k_screen_score_series(const double *__restrict__ f, int R, int d, int V, double *__restrict__ S)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= R * d) return;
    const int g = t / d, i = t % d;
    const double f0 = f[g];
    double s = 0.0;
    for (int v = 0; v < V; ++v) {
        const double fi = f[(1 + (int64_t)i * V + v) * R + g];
        s += fabs((f0 - fi) / (fabs(f0) + 1e-12));
    }
    S[t] = s / V;
}

__global__ void k_screen_eval_pairwise(ObjSpec spec, int d, int n_base, double h, uint64_t seed, double noise_sd,
                                       double *__restrict__ f)
{
    const int64_t E = 1 + d + (int64_t)d * (d - 1) / 2;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= E * n_base) return;
    const int k = (int)(t / E);
    const int64_t e = t % E;
    double x[GPBO_MAX_D];
    base_point(seed, k, d, h, x);
    int i, j;
    eval_axes(e, d, i, j);
    if (i >= 0) x[i] += h;
    if (j >= 0) x[j] += h;
    double s = 0.0;
    int o = 0;
    for (int b = 0; b < spec.nb; ++b) {
        s += block_value(spec.fn[b], x + o, spec.dim[b]);
        o += spec.dim[b];
    }
    if (noise_sd > 0.0) s += noise_sd * normal_draw(seed, (uint64_t)t);
    f[t] = s;
}

__global__ void k_screen_eval_routine(ObjSpec spec, int d, int n_base, double h, uint64_t seed, double noise_sd,
                                      double *__restrict__ f)
{
    const int E = 1 + d, R = spec.nb;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)E * n_base) return;
    const int k = (int)(t / E), e = (int)(t % E);
    double x[GPBO_MAX_D];
    base_point(seed, k, d, h, x);
    if (e > 0) x[e - 1] += h;
    int o = 0;
    for (int g = 0; g < R; ++g) {
        double v = block_value(spec.fn[g], x + o, spec.dim[g]);
        o += spec.dim[g];
        if (noise_sd > 0.0) v += noise_sd * normal_draw(seed, (uint64_t)(t * R + g));
        f[t * R + g] = v;
    }
}

// score_ij (i < j mirrored, zero diagonal) and influence_i from the evaluations.
__global__ void k_screen_score_pairwise(const double *__restrict__ f, int d, int n_base, double *__restrict__ score,
                                        double *__restrict__ infl)
{
    const int64_t E = 1 + d + (int64_t)d * (d - 1) / 2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= d * d) return;
    const int i = t / d, j = t % d;
    if (i == j) {
        double s = 0.0;
        for (int k = 0; k < n_base; ++k) {
            const double *F = f + (int64_t)k * E;
            s += fabs(F[1 + i] - F[0]) / (fabs(F[0]) + 1e-12);
        }
        infl[i] = s / n_base;
        score[t] = 0.0;
        return;
    }
    const int a = min(i, j), b = max(i, j);
    const int64_t p = (int64_t)a * d - (int64_t)a * (a + 1) / 2 + (b - a - 1);
    double num = 0.0, den = 0.0;
    for (int k = 0; k < n_base; ++k) {
        const double *F = f + (int64_t)k * E;
        double dlt = F[1 + d + p] - F[1 + a] - F[1 + b] + F[0];
        num += fabs(dlt);
        den += fabs(F[1 + a] - F[0]) + fabs(F[1 + b] - F[0]);
    }
    score[t] = (num / n_base) / (den / n_base + 1e-12);
}

__global__ void k_screen_score_routine(const double *__restrict__ f, int R, int d, int n_base,
                                       double *__restrict__ S)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= R * d) return;
    const int g = t / d, i = t % d;
    const int E = 1 + d;
    double s = 0.0;
    for (int k = 0; k < n_base; ++k) {
        double f0 = f[((int64_t)k * E) * R + g];
        double fi = f[((int64_t)k * E + 1 + i) * R + g];
        s += fabs((f0 - fi) / (fabs(f0) + 1e-12));
    }
    S[t] = s / n_base;
}

// ------------------------------------------------------------------ host partition
namespace {

struct DisjointSets {
    std::vector<int> up;
    explicit DisjointSets(int n) : up(n) { for (int i = 0; i < n; ++i) up[i] = i; }
    int root(int a) { while (up[a] != a) a = up[a] = up[up[a]]; return a; }
    void join(int a, int b)
    {
        a = root(a);
        b = root(b);
        if (a != b) up[std::max(a, b)] = std::min(a, b);  // the smaller root survives
    }
};

// Keep the max_dims most influential members of every oversized group.
void cap_groups(int d, const int *label, const double *infl, int max_dims, int *fixed)
{
    for (int i = 0; i < d; ++i) fixed[i] = 0;
    if (max_dims <= 0) return;
    std::vector<int> members;
    for (int g = 0; g < d; ++g) {
        members.clear();
        for (int i = 0; i < d; ++i)
            if (label[i] == g) members.push_back(i);
        if ((int)members.size() <= max_dims) continue;
        std::stable_sort(members.begin(), members.end(),
                         [&](int a, int b) { return infl[a] > infl[b] || (infl[a] == infl[b] && a < b); });
        for (size_t r = max_dims; r < members.size(); ++r) fixed[members[r]] = 1;
    }
}

}  // namespace

int screen_run(gpbo_ctx *ctx, const gpbo_objective *obj, int d, const screen_opts *o, double *score_out,
               double *infl_out, int *group_of, int *n_groups, int *fixed_out)
{
    const bool series = o->mode == GPBO_SCREEN_ROUTINE_SERIES;
    const bool routine = o->mode == GPBO_SCREEN_ROUTINE || series;
    const bool host_fn = obj->fn != nullptr;
    const int R = host_fn ? obj->n_routines : obj->n_blocks;
    if (routine && (R < 1 || R > GPBO_MAX_D)) return GPBO_EINVAL;
    std::vector<int> owner(d);
    ObjSpec spec{};
    if (!host_fn) {
        if (obj->n_blocks < 1 || obj->n_blocks > GPBO_MAX_D || !obj->block_dim || !obj->block_fn) return GPBO_EINVAL;
        spec.nb = obj->n_blocks;
        int sum = 0;
        for (int b = 0; b < spec.nb; ++b) {
            spec.dim[b] = obj->block_dim[b];
            spec.fn[b] = obj->block_fn[b];
            if (spec.dim[b] < 1 || spec.fn[b] < 0 || spec.fn[b] > 2) return GPBO_EINVAL;
            for (int k = 0; k < spec.dim[b] && sum + k < d; ++k) owner[sum + k] = b;
            sum += spec.dim[b];
        }
        if (sum != d) return GPBO_EINVAL;
    } else if (routine) {
        if (!obj->param_owner) return GPBO_EINVAL;
        for (int i = 0; i < d; ++i) {
            owner[i] = obj->param_owner[i];  // -1: shared, settled by the scores below
            if (owner[i] < -1 || owner[i] >= R) return GPBO_EINVAL;
        }
    }
    // the series schedule's ranges: the built-in blocks' own domains, else the caller's
    SeriesRange rg{};
    for (int i = 0; i < d; ++i) {
        rg.lo[i] = host_fn && o->lo ? o->lo[i] : 0.0;
        rg.hi[i] = host_fn && o->hi ? o->hi[i] : 1.0;
    }
    if (series && !host_fn) {
        int o2 = 0;
        for (int b = 0; b < spec.nb; ++b)
            for (int k = 0; k < spec.dim[b]; ++k, ++o2) {
                const double w = spec.fn[b] == GPBO_FN_ACKLEY ? 32.768 : spec.fn[b] == GPBO_FN_RASTRIGIN ? 5.12 : 2.0;
                rg.lo[o2] = -w;
                rg.hi[o2] = w;
            }
    }
    const int64_t E = series ? 1 + (int64_t)d * o->n_base : routine ? 1 + d : 1 + d + (int64_t)d * (d - 1) / 2;
    const int per = routine ? R : 1;
    const int64_t nf = series ? E * R : E * o->n_base * per;
    const int srows = routine ? R : d;
    void *w = nullptr;
    GPBO_TRY(ws_reserve(ctx, sizeof(double) * (nf + (int64_t)srows * d + d), &w));
    double *f = (double *)w, *S = f + nf, *infl = S + (int64_t)srows * d;
    cudaStream_t st = ctx->stream;

    if (!host_fn && series) {
        k_screen_eval_series<<<(unsigned)cdiv64(E, 128), 128, 0, st>>>(spec, rg, d, o->n_base, o->growth, o->seed,
                                                                         obj->noise_sd, f);
        GPBO_LAUNCH_CHECK(ctx);
    } else if (host_fn && series) {
        std::vector<double> hf(nf), u0(d), x(d), fr(R);
        for (int k = 0; k < d; ++k) u0[k] = uniform24d(o->seed, 3, (uint64_t)k);
        for (int64_t e = 0; e < E; ++e) {
            x = u0;
            if (e > 0) {
                const int i = (int)((e - 1) / o->n_base), v = (int)((e - 1) % o->n_base) + 1;
                x[i] = series_value(u0[i], rg.lo[i], rg.hi[i], o->growth, v);
            }
            double ft = 0.0;
            if (obj->fn(x.data(), d, &ft, fr.data(), obj->user) != 0) return GPBO_EINVAL;
            for (int g = 0; g < R; ++g) hf[e * R + g] = fr[g];
        }
        GPBO_CUDA_TRY(cudaMemcpyAsync(f, hf.data(), sizeof(double) * nf, cudaMemcpyHostToDevice, st));
        GPBO_CUDA_TRY(cudaStreamSynchronize(st));
    } else if (!host_fn) {
        const int64_t threads = E * o->n_base;
        if (routine)
            k_screen_eval_routine<<<(unsigned)cdiv64(threads, 128), 128, 0, st>>>(spec, d, o->n_base, o->h, o->seed,
                                                                                   obj->noise_sd, f);
        else
            k_screen_eval_pairwise<<<(unsigned)cdiv64(threads, 128), 128, 0, st>>>(spec, d, o->n_base, o->h, o->seed,
                                                                                    obj->noise_sd, f);
        GPBO_LAUNCH_CHECK(ctx);
    } else {
        // host black box: evaluate the same points on the host, then score on the device
        std::vector<double> hf(nf), x(d), fr(std::max(R, 1));
        for (int k = 0; k < o->n_base; ++k) {
            for (int64_t e = 0; e < E; ++e) {
                for (int t = 0; t < d; ++t) x[t] = (1.0 - o->h) * uniform24d(o->seed, 3, (uint64_t)k * d + t);
                int i = -1, j = -1;
                if (e >= 1 && e <= d) i = (int)e - 1;
                else if (e > d) {
                    int64_t p = e - 1 - d;
                    int a = 0;
                    while (p >= d - 1 - a) { p -= d - 1 - a; ++a; }
                    i = a;
                    j = a + 1 + (int)p;
                }
                if (i >= 0) x[i] += o->h;
                if (j >= 0) x[j] += o->h;
                double ft = 0.0;
                if (obj->fn(x.data(), d, &ft, fr.data(), obj->user) != 0) return GPBO_EINVAL;
                if (routine)
                    for (int g = 0; g < R; ++g) hf[((int64_t)k * E + e) * R + g] = fr[g];
                else
                    hf[(int64_t)k * E + e] = ft;
            }
        }
        GPBO_CUDA_TRY(cudaMemcpyAsync(f, hf.data(), sizeof(double) * nf, cudaMemcpyHostToDevice, st));
        GPBO_CUDA_TRY(cudaStreamSynchronize(st));
    }
    if (series)
        k_screen_score_series<<<(unsigned)cdiv64((int64_t)R * d, 128), 128, 0, st>>>(f, R, d, o->n_base, S);
    else if (routine)
        k_screen_score_routine<<<(unsigned)cdiv64((int64_t)R * d, 128), 128, 0, st>>>(f, R, d, o->n_base, S);
    else
        k_screen_score_pairwise<<<(unsigned)cdiv64((int64_t)d * d, 128), 128, 0, st>>>(f, d, o->n_base, S, infl);
    GPBO_LAUNCH_CHECK(ctx);

    std::vector<double> hs((size_t)srows * d), hinfl(d);
    GPBO_CUDA_TRY(cudaMemcpyAsync(hs.data(), S, sizeof(double) * srows * d, cudaMemcpyDeviceToHost, st));
    if (!routine) GPBO_CUDA_TRY(cudaMemcpyAsync(hinfl.data(), infl, sizeof(double) * d, cudaMemcpyDeviceToHost, st));
    GPBO_CUDA_TRY(cudaStreamSynchronize(st));

    std::vector<int> label(d), fx(d);
    if (!routine) {
        DisjointSets ds(d);
        for (int i = 0; i < d; ++i)
            for (int j = i + 1; j < d; ++j)
                if (hs[(size_t)i * d + j] > o->cutoff) ds.join(i, j);
        for (int i = 0; i < d; ++i) label[i] = ds.root(i);
    } else {
        // a shared parameter belongs to the routine it influences most (ties: the first)
        for (int i = 0; i < d; ++i)
            if (owner[i] < 0) {
                int b = 0;
                for (int g = 1; g < R; ++g)
                    if (hs[(size_t)g * d + i] > hs[(size_t)b * d + i]) b = g;
                owner[i] = b;
            }
        DisjointSets rs(R);
        for (int i = 0; i < d; ++i) {
            hinfl[i] = 0.0;
            for (int g = 0; g < R; ++g) {
                const double s = hs[(size_t)g * d + i];
                hinfl[i] = std::max(hinfl[i], s);
                if (g != owner[i] && s > o->cutoff) rs.join(owner[i], g);
            }
        }
        // label = smallest parameter index owned by the merged routine set
        std::vector<int> first(R, -1);
        for (int i = 0; i < d; ++i) {
            int r = rs.root(owner[i]);
            if (first[r] < 0) first[r] = i;
            label[i] = first[r];
        }
    }
    int ng = 0;
    for (int i = 0; i < d; ++i) ng += label[i] == i;
    cap_groups(d, label.data(), hinfl.data(), o->max_dims, fx.data());

    if (score_out) std::copy(hs.begin(), hs.end(), score_out);
    if (infl_out) std::copy(hinfl.begin(), hinfl.end(), infl_out);
    std::copy(label.begin(), label.end(), group_of);
    *n_groups = ng;
    if (fixed_out) std::copy(fx.begin(), fx.end(), fixed_out);
    return GPBO_OK;
}

}  // namespace gpbo
