// The C ABI of libgpbo.so (declared in include/gpbo.h): argument checks, host/device
// marshalling, the context's workspace arena and error mapping.  All arithmetic of the
// method runs in the kernels of fit.cu, score.cu, score_tc.cu and screen.cu.
#include "gpbo_internal.cuh"

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

namespace gpbo {

void fit_set_smem_limits();
int probe_fma(gpbo_ctx *ctx, int kind, double *tflops);

void note_cuda_error(cudaError_t e, const char *what, const char *file, int line)
{
    if (getenv("GPBO_VERBOSE")) fprintf(stderr, "gpbo: %s failed at %s:%d: %s\n", what, file, line, cudaGetErrorString(e));
}

namespace {
std::mutex g_smem_mu;
std::map<std::pair<const void *, int>, int> g_smem_set;
}  // namespace

int ensure_smem(const void *fn, int device, int bytes)
{
    std::lock_guard<std::mutex> lk(g_smem_mu);
    int &have = g_smem_set[std::make_pair(fn, device)];
    if (have >= bytes) return GPBO_OK;
    GPBO_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    have = bytes;
    return GPBO_OK;
}

int ws_reserve(gpbo_ctx *ctx, size_t bytes, void **out)
{
    bytes = (bytes + 4095) & ~(size_t)4095;
    if (bytes > ctx->ws_size) {
        if ((int64_t)bytes > ctx->ws_limit + ((int64_t)64 << 20) && (int64_t)bytes > ((int64_t)256 << 20))
            return GPBO_ENOMEM;
        if (ctx->ws) {
            // stream-ordered users of the old arena must finish before it is released
            GPBO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
            if (ctx->side) GPBO_CUDA_TRY(cudaStreamSynchronize(ctx->side));
            if (ctx->side2) GPBO_CUDA_TRY(cudaStreamSynchronize(ctx->side2));
            if (ctx->side3) GPBO_CUDA_TRY(cudaStreamSynchronize(ctx->side3));
            if (ctx->mainf) GPBO_CUDA_TRY(cudaStreamSynchronize(ctx->mainf));
            GPBO_CUDA_TRY(cudaFree(ctx->ws));
            ctx->ws = nullptr;
            ctx->ws_size = 0;
        }
        GPBO_CUDA_TRY(cudaMalloc(&ctx->ws, bytes));
        ctx->ws_size = bytes;
    }
    *out = ctx->ws;
    return GPBO_OK;
}

int side_stream(gpbo_ctx *ctx, cudaStream_t *out)
{
    if (!ctx->side) {
        int lo = 0, hi = 0;
        GPBO_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        GPBO_CUDA_TRY(cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, hi));
        GPBO_CUDA_TRY(cudaStreamCreateWithPriority(&ctx->side2, cudaStreamNonBlocking, hi));
        GPBO_CUDA_TRY(cudaStreamCreateWithPriority(&ctx->side3, cudaStreamNonBlocking, lo));
        GPBO_CUDA_TRY(cudaStreamCreateWithPriority(&ctx->mainf, cudaStreamNonBlocking, (lo + hi) / 2));
        for (cudaEvent_t &e : ctx->side_ev) GPBO_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    *out = ctx->side;
    return GPBO_OK;
}

// Read and clear the device error word (synchronises the stream).
int take_device_status(gpbo_ctx *ctx, unsigned *bits_out)
{
    GPBO_CUDA_TRY(cudaMemcpyAsync(ctx->pinned, ctx->dev_status, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
    GPBO_CUDA_TRY(cudaMemsetAsync(ctx->dev_status, 0, sizeof(unsigned), ctx->stream));
    GPBO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    *bits_out = *(unsigned *)ctx->pinned;
    return GPBO_OK;
}

// Trace intervals may nest (the Cholesky updates inside the fit): begin takes the next
// record and pushes its index, end pops it.
int trace_begin(gpbo_ctx *ctx, int phase, double flops)
{
    if (!ctx->trace) return GPBO_OK;
    if (ctx->trace_depth >= (int)(sizeof(ctx->trace_stack) / sizeof(ctx->trace_stack[0]))) return GPBO_EINVAL;
    if (ctx->trace_n == ctx->trace_cap) {
        int cap = ctx->trace_cap ? ctx->trace_cap * 2 : 256;
        TraceRec *r = (TraceRec *)realloc(ctx->trace_recs, sizeof(TraceRec) * cap);
        if (!r) return GPBO_ENOMEM;
        for (int i = ctx->trace_cap; i < cap; ++i) {
            r[i].a = r[i].b = nullptr;
        }
        ctx->trace_recs = r;
        ctx->trace_cap = cap;
    }
    const int idx = ctx->trace_n++;
    TraceRec &t = ctx->trace_recs[idx];
    if (!t.a) GPBO_CUDA_TRY(cudaEventCreate(&t.a));
    if (!t.b) GPBO_CUDA_TRY(cudaEventCreate(&t.b));
    t.phase = phase;
    t.flops = flops;
    ctx->trace_stack[ctx->trace_depth++] = idx;
    GPBO_CUDA_TRY(cudaEventRecord(t.a, ctx->stream));
    return GPBO_OK;
}

int trace_end(gpbo_ctx *ctx)
{
    if (!ctx->trace) return GPBO_OK;
    if (ctx->trace_depth <= 0) return GPBO_EINVAL;
    const int idx = ctx->trace_stack[--ctx->trace_depth];
    GPBO_CUDA_TRY(cudaEventRecord(ctx->trace_recs[idx].b, ctx->stream));
    return GPBO_OK;
}

static int set_device(gpbo_ctx *ctx)
{
    GPBO_CUDA_TRY(cudaSetDevice(ctx->device));
    return GPBO_OK;
}

static bool finite_all(const double *a, int64_t n)
{
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

void model_free(gp_model *m)
{
    if (!m) return;
    void *ptrs[] = {m->X,       m->Xs64,    m->Xs32,   m->K,      m->L,      m->Dinv,
                    m->alpha64, m->alpha32, m->Linv64, m->Linv32, m->Linv16, m->Zsplit, m->nb32,
                    m->cslices, m->cexps, m->xmax};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete m;
}

template <typename T>
static int dalloc(T **p, size_t count)
{
    GPBO_CUDA_TRY(cudaMalloc((void **)p, sizeof(T) * count));
    return GPBO_OK;
}

static int alloc_model(gp_model *m)
{
    const size_t sq = (size_t)m->n_pad * m->n_pad;
    GPBO_TRY(dalloc(&m->X, (size_t)m->n_pad * m->d));  // room for any n with this n_pad
    GPBO_TRY(dalloc(&m->Xs64, (size_t)m->d * m->n_pad));
    GPBO_TRY(dalloc(&m->Xs32, (size_t)m->d * m->n_pad));
    GPBO_TRY(dalloc(&m->K, sq));
    GPBO_TRY(dalloc(&m->L, sq));
    GPBO_TRY(dalloc(&m->Dinv, (size_t)m->n_pad * NB));
    GPBO_TRY(dalloc(&m->alpha64, m->n_pad));
    GPBO_TRY(dalloc(&m->alpha32, m->n_pad));
    if (m->prec == GPBO_PREC_F64) GPBO_TRY(dalloc(&m->Linv64, sq));
    else GPBO_TRY(dalloc(&m->Linv32, sq));
    if (m->prec == GPBO_PREC_F16) GPBO_CUDA_TRY(cudaMalloc(&m->Linv16, sq * 2));
    if (m->prec == GPBO_PREC_BF16) GPBO_CUDA_TRY(cudaMalloc(&m->Linv16, sq * 4));  // hi then lo
    if (m->n_pad >= CHOL_TC_UPDATE_MIN_NPAD) {
        GPBO_CUDA_TRY(cudaMalloc(&m->cslices, chol_tc_slice_bytes(m->n_pad)));
        GPBO_TRY(dalloc(&m->cexps, m->n_pad));
    }
    if (m->n_pad >= CHOL_TC_MIN_NPAD) {
        GPBO_TRY(dalloc(&m->xmax, 1));
    }
    if ((m->prec == GPBO_PREC_BF16 || m->prec == GPBO_PREC_F16) && m->d <= 32) {
        GPBO_CUDA_TRY(cudaMalloc(&m->Zsplit, (size_t)m->n_pad * 128 * 2));
        GPBO_TRY(dalloc(&m->nb32, m->n_pad));
    }
    return GPBO_OK;
}

int model_n_pad(int n, int prec)
{
    return round_up(n, (prec == GPBO_PREC_BF16 || prec == GPBO_PREC_F16) ? TC_NCHUNK : NB);
}

int model_create(gpbo_ctx *ctx, int n, int d, int prec, gp_model **out)
{
    gp_model *m = new (std::nothrow) gp_model();
    if (!m) return GPBO_ENOMEM;
    m->ctx = ctx;
    m->n = n;
    m->d = d;
    m->prec = prec;
    m->n_pad = model_n_pad(n, prec);
    const int st = alloc_model(m);
    if (st != GPBO_OK) {
        model_free(m);
        return st;
    }
    *out = m;
    return GPBO_OK;
}

// Fit model m (allocated for this n, d, prec) with optional jitter escalation.  X and y are
// device pointers here.
static int fit_run(gpbo_ctx *ctx, gp_model *m, const double *X, const double *y, const gp_hyper *hyp, unsigned flags)
{
    const int n = m->n, d = m->d;
    int st = GPBO_OK;
    m->s2 = hyp->signal_var;
    m->sn2 = hyp->noise_var;
    for (int k = 0; k < d; ++k) m->ls[k] = hyp->lengthscale[k];
    const int tries = (flags & GPBO_JITTER) ? 4 : 1;
    for (int t = 0; st == GPBO_OK || st == GPBO_ENOTSPD; ++t) {
        if (t == tries) break;
        if (t > 0) m->sn2 = m->sn2 > 0 ? m->sn2 * 10.0 : 1e-10;  // jitter escalation
        const double nn = (double)n;
        st = trace_begin(ctx, PH_FIT, nn * nn * nn / 3.0);
        if (st != GPBO_OK) break;
        st = fit_model(ctx, m, X, y);
        if (st != GPBO_OK && st != GPBO_ENOTSPD) break;
        const int s2 = trace_end(ctx);
        if (s2 != GPBO_OK) { st = s2; break; }
        if (st == GPBO_OK) break;
    }
    if (st != GPBO_OK) cudaStreamSynchronize(ctx->stream);
    return st;
}

// Allocate and fit a new model.
static int fit_impl(gpbo_ctx *ctx, const double *X, const double *y, int n, int d, const gp_hyper *hyp, int prec,
                    unsigned flags, gp_model **out)
{
    gp_model *m = nullptr;
    int st = model_create(ctx, n, d, prec, &m);
    if (st != GPBO_OK) return st;
    st = fit_run(ctx, m, X, y, hyp, flags);
    if (st != GPBO_OK) {
        model_free(m);
        return st;
    }
    *out = m;
    return GPBO_OK;
}

int check_hyper(const gp_hyper *hyp, int d)
{
    if (!hyp || hyp->d != d || !hyp->lengthscale) return GPBO_EINVAL;
    for (int k = 0; k < d; ++k)
        if (!(hyp->lengthscale[k] > 0) || !std::isfinite(hyp->lengthscale[k])) return GPBO_EINVAL;
    if (!(hyp->signal_var > 0) || !(hyp->noise_var >= 0) || !std::isfinite(hyp->signal_var) ||
        !std::isfinite(hyp->noise_var))
        return GPBO_EINVAL;
    return GPBO_OK;
}

}  // namespace gpbo

using namespace gpbo;

extern "C" {

const char *gpbo_strerror(int s)
{
    switch (s) {
    case GPBO_OK: return "ok";
    case GPBO_EINVAL: return "invalid argument";
    case GPBO_ENOTSPD: return "kernel matrix not positive definite";
    case GPBO_ENAN: return "NaN or Inf in the inputs";
    case GPBO_ENOMEM: return "device allocation failed";
    case GPBO_ECUDA: return "CUDA runtime error";
    case GPBO_ETIMEOUT: return "bounded device wait timed out";
    case GPBO_ENOTSUP: return "unsupported device or feature";
    case GPBO_ESCRATCH: return "problem too large for the allocation-free scratch (4 MiB)";
    }
    return "unknown status";
}

int gpbo_create(gpbo_ctx **out, int device, void *stream)
{
    if (!out) return GPBO_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0 || device < 0 || device >= ndev) {
        cudaGetLastError();
        return GPBO_ENOTSUP;
    }
    cudaDeviceProp prop;
    GPBO_CUDA_TRY(cudaGetDeviceProperties(&prop, device));
    if (!(prop.major == 10 && prop.minor == 3)) return GPBO_ENOTSUP;
    gpbo_ctx *ctx = new (std::nothrow) gpbo_ctx();
    if (!ctx) return GPBO_ENOMEM;
    ctx->device = device;
    ctx->sm_count = prop.multiProcessorCount;
    GPBO_CUDA_TRY(cudaSetDevice(device));
    if (stream) {
        ctx->stream = (cudaStream_t)stream;
    } else {
        GPBO_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
        ctx->own_stream = true;
    }
    GPBO_CUDA_TRY(cudaMalloc(&ctx->dev_status, 64));
    GPBO_CUDA_TRY(cudaMemset(ctx->dev_status, 0, 64));
    GPBO_CUDA_TRY(cudaMallocHost(&ctx->pinned, 4096));
    fit_set_smem_limits();
    *out = ctx;
    return GPBO_OK;
}

int gpbo_destroy(gpbo_ctx *ctx)
{
    if (!ctx) return GPBO_EINVAL;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->batch_plan) batch_plan_free(ctx->batch_plan);
    if (ctx->step_model) model_free(ctx->step_model);
    if (ctx->step_buf) cudaFree(ctx->step_buf);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->dev_status) cudaFree(ctx->dev_status);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    if (ctx->side) {
        cudaStreamSynchronize(ctx->side);
        cudaStreamDestroy(ctx->side);
    }
    if (ctx->side2) {
        cudaStreamSynchronize(ctx->side2);
        cudaStreamDestroy(ctx->side2);
    }
    if (ctx->side3) {
        cudaStreamSynchronize(ctx->side3);
        cudaStreamDestroy(ctx->side3);
    }
    if (ctx->mainf) {
        cudaStreamSynchronize(ctx->mainf);
        cudaStreamDestroy(ctx->mainf);
    }
    for (cudaEvent_t e : ctx->side_ev)
        if (e) cudaEventDestroy(e);
    for (int i = 0; i < ctx->trace_cap; ++i) {
        if (ctx->trace_recs[i].a) cudaEventDestroy(ctx->trace_recs[i].a);
        if (ctx->trace_recs[i].b) cudaEventDestroy(ctx->trace_recs[i].b);
    }
    free(ctx->trace_recs);
    delete ctx;
    return GPBO_OK;
}

int gpbo_set_stream(gpbo_ctx *ctx, void *stream)
{
    if (!ctx) return GPBO_EINVAL;
    GPBO_TRY(set_device(ctx));
    if (stream) {
        if (ctx->own_stream) {
            cudaStreamSynchronize(ctx->stream);
            cudaStreamDestroy(ctx->stream);
            ctx->own_stream = false;
        }
        ctx->stream = (cudaStream_t)stream;
    } else if (!ctx->own_stream) {
        GPBO_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
        ctx->own_stream = true;
    }
    return GPBO_OK;
}

int64_t gpbo_launch_count(const gpbo_ctx *ctx) { return ctx ? ctx->launches : -1; }

int gpbo_trace_enable(gpbo_ctx *ctx, int on)
{
    if (!ctx) return GPBO_EINVAL;
    ctx->trace = on != 0;
    if (on) ctx->trace_n = 0;
    ctx->trace_depth = 0;
    return GPBO_OK;
}

int gpbo_trace_read(gpbo_ctx *ctx, int nphase, double *ms, int64_t *intervals, double *flops)
{
    if (!ctx || nphase < 0) return GPBO_EINVAL;
    GPBO_TRY(set_device(ctx));
    GPBO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    for (int p = 0; p < nphase; ++p) {
        if (ms) ms[p] = 0.0;
        if (intervals) intervals[p] = 0;
        if (flops) flops[p] = 0.0;
    }
    for (int i = 0; i < ctx->trace_n; ++i) {
        const TraceRec &t = ctx->trace_recs[i];
        if (t.phase >= nphase) continue;
        float e = 0.f;
        GPBO_CUDA_TRY(cudaEventElapsedTime(&e, t.a, t.b));
        if (ms) ms[t.phase] += e;
        if (intervals) intervals[t.phase] += 1;
        if (flops) flops[t.phase] += t.flops;
    }
    return GPBO_OK;
}

int gpbo_probe_fma(gpbo_ctx *ctx, int kind, double *tflops)
{
    if (!ctx || !tflops || (kind != 0 && kind != 1)) return GPBO_EINVAL;
    GPBO_TRY(set_device(ctx));
    return probe_fma(ctx, kind, tflops);
}

int gpbo_set_wait_limit(gpbo_ctx *ctx, int64_t cycles)
{
    if (!ctx || cycles < 0) return GPBO_EINVAL;
    GPBO_TRY(set_device(ctx));
    const long long v = (long long)cycles;
    GPBO_CUDA_TRY(cudaMemcpyAsync((char *)ctx->dev_status + 8, &v, sizeof(v), cudaMemcpyHostToDevice, ctx->stream));
    GPBO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return GPBO_OK;
}

int gpbo_inject_wait_stall(gpbo_ctx *ctx, int stall)
{
    if (!ctx || (stall != 0 && stall != 1)) return GPBO_EINVAL;
    GPBO_TRY(set_device(ctx));
    const unsigned v = (unsigned)stall;
    GPBO_CUDA_TRY(cudaMemcpyAsync((char *)ctx->dev_status + 4, &v, sizeof(v), cudaMemcpyHostToDevice, ctx->stream));
    GPBO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return GPBO_OK;
}

int gpbo_set_workspace_limit(gpbo_ctx *ctx, int64_t bytes)
{
    if (!ctx || bytes < ((int64_t)1 << 20)) return GPBO_EINVAL;
    ctx->ws_limit = bytes;
    return GPBO_OK;
}

int gp_fit(gpbo_ctx *ctx, const double *X, const double *y, int n, int d, const gp_hyper *hyp, gpbo_prec prec,
           unsigned flags, gp_model **out)
{
    if (!ctx || !X || !y || !out || n < 1 || n > GPBO_MAX_N || d < 1 || d > GPBO_MAX_D) return GPBO_EINVAL;
    if (prec < GPBO_PREC_F64 || prec > GPBO_PREC_F16) return GPBO_EINVAL;
    GPBO_TRY(check_hyper(hyp, d));
    GPBO_TRY(set_device(ctx));
    const double *Xd = X, *yd = y;
    if (flags & GPBO_HOST_PTRS) {
        if (!finite_all(X, (int64_t)n * d) || !finite_all(y, n)) return GPBO_ENAN;
        // the fit reserves more workspace later, so stage the inputs in their own buffer
        double *stage = nullptr;
        GPBO_CUDA_TRY(cudaMalloc(&stage, sizeof(double) * ((size_t)n * d + n)));
        GPBO_CUDA_TRY(cudaMemcpyAsync(stage, X, sizeof(double) * n * d, cudaMemcpyHostToDevice, ctx->stream));
        GPBO_CUDA_TRY(cudaMemcpyAsync(stage + (size_t)n * d, y, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
        int st = fit_impl(ctx, stage, stage + (size_t)n * d, n, d, hyp, prec, flags, out);
        cudaStreamSynchronize(ctx->stream);
        cudaFree(stage);
        return st;
    }
    return fit_impl(ctx, Xd, yd, n, d, hyp, prec, flags, out);
}

int gp_model_free(gp_model *m)
{
    if (!m) return GPBO_EINVAL;
    cudaSetDevice(m->ctx->device);
    cudaStreamSynchronize(m->ctx->stream);
    model_free(m);
    return GPBO_OK;
}

int gp_model_info(const gp_model *m, int *n, int *d, int *prec, double *sn2)
{
    if (!m) return GPBO_EINVAL;
    if (n) *n = m->n;
    if (d) *d = m->d;
    if (prec) *prec = m->prec;
    if (sn2) *sn2 = m->sn2;
    return GPBO_OK;
}

int gp_model_read(const gp_model *m, double *L_host, double *alpha_host)
{
    if (!m) return GPBO_EINVAL;
    gpbo_ctx *ctx = m->ctx;
    GPBO_TRY(set_device(ctx));
    if (L_host)
        GPBO_CUDA_TRY(cudaMemcpy2DAsync(L_host, sizeof(double) * m->n, m->L, sizeof(double) * m->n_pad,
                                        sizeof(double) * m->n, m->n, cudaMemcpyDeviceToHost, ctx->stream));
    if (alpha_host)
        GPBO_CUDA_TRY(cudaMemcpyAsync(alpha_host, m->alpha64, sizeof(double) * m->n, cudaMemcpyDeviceToHost, ctx->stream));
    GPBO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return GPBO_OK;
}

int gpbo_gen_candidates(gpbo_ctx *ctx, uint64_t seed, int64_t first, int64_t M, int d, float *out)
{
    if (!ctx || !out || M < 1 || first < 0 || d < 1 || d > GPBO_MAX_D) return GPBO_EINVAL;
    GPBO_TRY(set_device(ctx));
    return gen_candidates(ctx, seed, first, M, d, out);
}

static int posterior_impl(gpbo_ctx *ctx, const gp_model *m, const float *Xc, int64_t M, uint64_t seed, double y_best,
                          const double *tau_dev, double xi, unsigned flags, void *mu, void *sigma, void *ei,
                          int64_t *argmax, double *ei_max)
{
    const size_t esz = m->prec == GPBO_PREC_F64 ? 8 : 4;
    if (!(flags & GPBO_HOST_PTRS))
        return score_model(ctx, m, Xc, M, seed, y_best, tau_dev, xi, mu, sigma, ei, argmax, ei_max);
    // host buffers: stage through device memory of our own (the workspace is used by scoring)
    float *dXc = nullptr;
    void *dmu = nullptr, *dsg = nullptr, *dei = nullptr;
    int st = GPBO_OK;
    auto cleanup = [&]() {
        cudaStreamSynchronize(ctx->stream);
        if (dXc) cudaFree(dXc);
        if (dmu) cudaFree(dmu);
        if (dsg) cudaFree(dsg);
        if (dei) cudaFree(dei);
    };
    if (Xc) {
        if (cudaMalloc(&dXc, sizeof(float) * M * m->d) != cudaSuccess) { cleanup(); return GPBO_ENOMEM; }
        cudaMemcpyAsync(dXc, Xc, sizeof(float) * M * m->d, cudaMemcpyHostToDevice, ctx->stream);
    }
    if (mu && cudaMalloc(&dmu, esz * M) != cudaSuccess) { cleanup(); return GPBO_ENOMEM; }
    if (sigma && cudaMalloc(&dsg, esz * M) != cudaSuccess) { cleanup(); return GPBO_ENOMEM; }
    if (ei && cudaMalloc(&dei, esz * M) != cudaSuccess) { cleanup(); return GPBO_ENOMEM; }
    st = score_model(ctx, m, dXc, M, seed, y_best, tau_dev, xi, dmu, dsg, dei, argmax, ei_max);
    if (st == GPBO_OK) {
        if (mu) cudaMemcpyAsync(mu, dmu, esz * M, cudaMemcpyDeviceToHost, ctx->stream);
        if (sigma) cudaMemcpyAsync(sigma, dsg, esz * M, cudaMemcpyDeviceToHost, ctx->stream);
        if (ei) cudaMemcpyAsync(ei, dei, esz * M, cudaMemcpyDeviceToHost, ctx->stream);
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) st = GPBO_ECUDA;
    }
    cleanup();
    return st;
}

int gp_posterior_ei(gpbo_ctx *ctx, const gp_model *m, const float *Xc, int64_t M, uint64_t seed, double y_best,
                    double xi, unsigned flags, void *mu, void *sigma, void *ei, int64_t *argmax, double *ei_max)
{
    if (!ctx || !m || !argmax || !ei_max || M < 1 || M > 0x7fffffffll) return GPBO_EINVAL;
    if (!std::isfinite(y_best) || !std::isfinite(xi)) return GPBO_EINVAL;
    GPBO_TRY(set_device(ctx));
    int64_t am = -1;
    double em = 0.0;
    GPBO_TRY(posterior_impl(ctx, m, Xc, M, seed, y_best, nullptr, xi, flags, mu, sigma, ei, &am, &em));
    *argmax = am;
    *ei_max = em;
    return GPBO_OK;
}

int interdep_screen(gpbo_ctx *ctx, const gpbo_objective *obj, int d, const screen_opts *o, double *score,
                    double *influence, int *group_of, int *n_groups, int *fixed)
{
    if (!ctx || !obj || !o || !group_of || !n_groups || d < 1 || d > GPBO_MAX_D) return GPBO_EINVAL;
    if (o->mode != GPBO_SCREEN_PAIRWISE && o->mode != GPBO_SCREEN_ROUTINE && o->mode != GPBO_SCREEN_ROUTINE_SERIES)
        return GPBO_EINVAL;
    if (o->n_base < 1 || !std::isfinite(o->cutoff)) return GPBO_EINVAL;
    if (o->mode == GPBO_SCREEN_ROUTINE_SERIES) {
        if (!(o->growth > 0.0) || !std::isfinite(o->growth) || (int64_t)o->n_base * d > (1 << 24)) return GPBO_EINVAL;
        if (obj->fn && o->lo && o->hi)
            for (int i = 0; i < d; ++i)
                if (!(o->lo[i] < o->hi[i]) || !std::isfinite(o->lo[i]) || !std::isfinite(o->hi[i])) return GPBO_EINVAL;
    } else if (!(o->h > 0.0) || !(o->h < 0.5)) {
        return GPBO_EINVAL;
    }
    if (!(obj->noise_sd >= 0.0)) return GPBO_EINVAL;
    GPBO_TRY(set_device(ctx));
    GPBO_TRY(trace_begin(ctx, PH_SCREEN, 0.0));
    int st = screen_run(ctx, obj, d, o, score, influence, group_of, n_groups, fixed);
    int s2 = trace_end(ctx);
    return st != GPBO_OK ? st : s2;
}

int search_step(gpbo_ctx *ctx, const double *X, const double *y, int n, int d, const gp_hyper *hyp, const float *Xc,
                int64_t M, uint64_t seed, double xi, gpbo_prec prec, unsigned flags, double *x_next, double *ei_max,
                int64_t *argmax)
{
    if (!ctx || !X || !y || !x_next || !ei_max || n < 1 || n > GPBO_MAX_N || d < 1 || d > GPBO_MAX_D || M < 1 ||
        M > 0x7fffffffll)
        return GPBO_EINVAL;
    if (prec < GPBO_PREC_F64 || prec > GPBO_PREC_F16) return GPBO_EINVAL;
    GPBO_TRY(check_hyper(hyp, d));
    GPBO_TRY(set_device(ctx));
    // private device staging: X, y, standardised y, tau, and (host) candidates
    const bool host = flags & GPBO_HOST_PTRS;
    if (host && (!finite_all(X, (int64_t)n * d) || !finite_all(y, n))) return GPBO_ENAN;
    // the staging buffer and the model stay with the context for the next call of this shape
    float *dXc = nullptr;
    const size_t nd = (size_t)n * d;
    const size_t buf_bytes = sizeof(double) * (nd + 2 * (size_t)n + 2 + GPBO_MAX_D);
    if (ctx->step_buf_bytes < buf_bytes) {
        GPBO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        if (ctx->step_buf) GPBO_CUDA_TRY(cudaFree(ctx->step_buf));
        ctx->step_buf = nullptr;
        ctx->step_buf_bytes = 0;
        GPBO_CUDA_TRY(cudaMalloc(&ctx->step_buf, buf_bytes));
        ctx->step_buf_bytes = buf_bytes;
    }
    double *buf = (double *)ctx->step_buf;
    double *dX = buf, *dy = buf + nd, *ys = dy + n, *tau = ys + n;
    float *xsel = (float *)(tau + 2);
    int st = GPBO_OK;
    gp_model *m = nullptr;
    if (host) {
        cudaMemcpyAsync(dX, X, sizeof(double) * nd, cudaMemcpyHostToDevice, ctx->stream);
        cudaMemcpyAsync(dy, y, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream);
        if (Xc) {
            if (cudaMalloc(&dXc, sizeof(float) * M * d) != cudaSuccess) st = GPBO_ENOMEM;
            else cudaMemcpyAsync(dXc, Xc, sizeof(float) * M * d, cudaMemcpyHostToDevice, ctx->stream);
        }
    } else {
        cudaMemcpyAsync(dX, X, sizeof(double) * nd, cudaMemcpyDeviceToDevice, ctx->stream);
        cudaMemcpyAsync(dy, y, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream);
        dXc = const_cast<float *>(Xc);
    }
    if (st == GPBO_OK) st = standardize_dev(ctx, dy, n, ys, tau);
    m = ctx->step_model;
    if (st == GPBO_OK && m && m->d == d && m->prec == prec && m->n_pad == model_n_pad(n, prec)) {
        m->n = n;  // same buffers: every n-dependent part of the fit is recomputed
    } else if (st == GPBO_OK) {
        cudaStreamSynchronize(ctx->stream);
        if (m) model_free(m);
        m = ctx->step_model = nullptr;
        st = model_create(ctx, n, d, prec, &m);
        if (st == GPBO_OK) ctx->step_model = m;
    }
    if (st == GPBO_OK) st = fit_run(ctx, m, dX, ys, hyp, flags & ~GPBO_HOST_PTRS);
    int64_t am = -1;
    double em = 0.0;
    if (st == GPBO_OK) st = score_model(ctx, m, dXc, M, seed, 0.0, tau, xi, nullptr, nullptr, nullptr, &am, &em);
    if (st == GPBO_OK) {
        // x_next is the argmax candidate: gather it from Xc, or redraw that one point
        std::vector<float> xn(d);
        const float *src = dXc ? dXc + am * d : xsel;
        if (!dXc) st = gen_candidates(ctx, seed, am, 1, d, xsel);
        if (st == GPBO_OK && cudaMemcpyAsync(xn.data(), src, sizeof(float) * d, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
            st = GPBO_ECUDA;
        if (st == GPBO_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) st = GPBO_ECUDA;
        for (int k = 0; k < d; ++k) x_next[k] = (double)xn[k];
        *ei_max = em;
        if (argmax) *argmax = am;
    }
    cudaStreamSynchronize(ctx->stream);
    if (host && dXc) cudaFree(dXc);
    return st;
}

}  // extern "C"
