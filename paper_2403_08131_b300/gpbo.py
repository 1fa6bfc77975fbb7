"""Python binding of libgpbo.so (include/gpbo.h): argument marshalling only.

Every computation runs in the library's CUDA kernels.  PyTorch provides device
buffers and the stream; numpy arrays are passed as host buffers with GPBO_HOST_PTRS.
Importing this module fails loudly when the library has not been built: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgpbo.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2403_08131_b300.build`")

_lib = C.CDLL(LIB_PATH)

GPBO_OK, GPBO_EINVAL, GPBO_ENOTSPD, GPBO_ENAN, GPBO_ENOMEM, GPBO_ECUDA, GPBO_ETIMEOUT, GPBO_ENOTSUP, GPBO_ESCRATCH = \
    range(9)
PREC = {"f64": 0, "f32": 1, "bf16": 2, "f16": 3}
HOST_PTRS = 0x1
JITTER = 0x2
SCREEN_PAIRWISE, SCREEN_ROUTINE, SCREEN_ROUTINE_SERIES = 0, 1, 2

_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_L = C.POINTER(C.c_int64)


class GpHyper(C.Structure):
    _fields_ = [("d", C.c_int), ("lengthscale", _D), ("signal_var", C.c_double), ("noise_var", C.c_double)]


HOST_FN = C.CFUNCTYPE(C.c_int, _D, C.c_int, _D, _D, C.c_void_p)
EVAL_FN = C.CFUNCTYPE(C.c_int, _D, C.c_int, _D, C.c_void_p)


class BoOpts(C.Structure):
    _fields_ = [("budget", C.c_int), ("n_init", C.c_int), ("x_init", _D), ("M", C.c_int64), ("seed", C.c_uint64),
                ("prec", C.c_int), ("refit", C.c_int), ("hyp", GpHyper), ("xi", C.c_double), ("mle_iters", C.c_int)]


class GpboObjective(C.Structure):
    _fields_ = [("n_blocks", C.c_int), ("block_dim", _I), ("block_fn", _I), ("noise_sd", C.c_double),
                ("seed", C.c_uint64), ("fn", HOST_FN), ("n_routines", C.c_int), ("param_owner", _I),
                ("user", C.c_void_p)]


class ScreenOpts(C.Structure):
    _fields_ = [("mode", C.c_int), ("n_base", C.c_int), ("h", C.c_double), ("cutoff", C.c_double),
                ("max_dims", C.c_int), ("seed", C.c_uint64), ("growth", C.c_double), ("lo", _D), ("hi", _D)]


def _sig(name, restype, argtypes):
    f = getattr(_lib, name)
    f.restype = restype
    f.argtypes = argtypes
    return f


_create = _sig("gpbo_create", C.c_int, [C.POINTER(_P), C.c_int, _P])
_destroy = _sig("gpbo_destroy", C.c_int, [_P])
_set_stream = _sig("gpbo_set_stream", C.c_int, [_P, _P])
_strerror = _sig("gpbo_strerror", C.c_char_p, [C.c_int])
_launches = _sig("gpbo_launch_count", C.c_int64, [_P])
_ws_limit = _sig("gpbo_set_workspace_limit", C.c_int, [_P, C.c_int64])
_trace_en = _sig("gpbo_trace_enable", C.c_int, [_P, C.c_int])
_trace_rd = _sig("gpbo_trace_read", C.c_int, [_P, C.c_int, _D, _L, _D])
PHASES = ("fit", "xkern", "variance", "screen", "chol_update", "lml", "factor", "inverse")
_probe = _sig("gpbo_probe_fma", C.c_int, [_P, C.c_int, _D])
_wait_limit = _sig("gpbo_set_wait_limit", C.c_int, [_P, C.c_int64])
_inject_stall = _sig("gpbo_inject_wait_stall", C.c_int, [_P, C.c_int])
_fit = _sig("gp_fit", C.c_int, [_P, _P, _P, C.c_int, C.c_int, C.POINTER(GpHyper), C.c_int, C.c_uint,
                                 C.POINTER(_P)])
_model_free = _sig("gp_model_free", C.c_int, [_P])
_model_info = _sig("gp_model_info", C.c_int, [_P, _I, _I, _I, _D])
_model_read = _sig("gp_model_read", C.c_int, [_P, _P, _P])
_posterior = _sig("gp_posterior_ei", C.c_int, [_P, _P, _P, C.c_int64, C.c_uint64, C.c_double, C.c_double, C.c_uint,
                                               _P, _P, _P, _L, _D])
_step_batched = _sig("search_step_batched", C.c_int, [_P, C.c_int, C.POINTER(_P), C.POINTER(_P), _I, _I,
                                                     C.POINTER(GpHyper), _L, C.POINTER(C.c_uint64), C.c_double,
                                                     C.c_int, C.c_uint, _D, _D, _L])
_batched_tile = _sig("search_step_batched_tile", C.c_int, [_P, C.c_int])
_batched_tuning = _sig("search_step_batched_tuning", C.c_int, [_P, _I, C.POINTER(C.c_float), _I])
_posterior_noalloc = _sig("gp_posterior_ei_noalloc", C.c_int, [_P, _P, _P, C.c_int64, C.c_uint64, C.c_double,
                                                               C.c_double, _P, _P, _P, _L, _D])
_mlp_create = _sig("mlp_create", C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_uint64, C.POINTER(_P)])
_mlp_free = _sig("mlp_free", C.c_int, [_P])
_mlp_params = _sig("mlp_params", C.c_int, [_P, _P, _P])
_mlp_forward = _sig("mlp_forward", C.c_int, [_P, _P, _P, C.c_int, _P])
_mlp_grads = _sig("mlp_gradients", C.c_int, [_P, _P, _P, _P, C.c_int, _P, _P])
_mlp_train = _sig("mlp_train", C.c_int, [_P, _P, _P, _P, _P, C.c_int64, C.c_int, C.c_int, C.c_float, C.c_uint64,
                                         C.POINTER(C.c_float)])
_mlp_norm = _sig("mlp_norm", C.c_int, [_P, _D])
_mlp_score = _sig("mlp_score", C.c_int, [_P, _P, _P, C.c_int64, C.c_uint64, C.c_double, C.c_double, C.c_int, _P,
                                          _P, _P])
_screen_sur = _sig("surrogate_screen", C.c_int, [_P, _P, _P, C.c_int64, C.c_uint64, C.c_int, C.c_double, C.c_double,
                                                 _P, _P, _L, _D])
_lml = _sig("gp_lml", C.c_int, [_P, _P, _P, C.c_int, C.c_int, C.POINTER(GpHyper), C.c_uint, _D, _D])
_fit_mle = _sig("gp_fit_mle", C.c_int, [_P, _P, _P, C.c_int, C.c_int, C.c_int, _D, _D, _D, C.c_int, C.c_double,
                                         C.c_uint, _D, _D, _L])
_bo = _sig("bo_search", C.c_int, [_P, C.c_int, EVAL_FN, C.c_void_p, C.POINTER(BoOpts), _D, _D, _I])
_gen = _sig("gpbo_gen_candidates", C.c_int, [_P, C.c_uint64, C.c_int64, C.c_int64, C.c_int, _P])
_screen = _sig("interdep_screen", C.c_int, [_P, C.POINTER(GpboObjective), C.c_int, C.POINTER(ScreenOpts), _P, _P,
                                             _P, _I, _P])
_step = _sig("search_step", C.c_int, [_P, _P, _P, C.c_int, C.c_int, C.POINTER(GpHyper), _P, C.c_int64, C.c_uint64,
                                       C.c_double, C.c_int, C.c_uint, _P, _D, _L])


class GpboError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        super().__init__(f"{where}: {_strerror(code).decode()} ({code})")


def check(code, where=""):
    if code != GPBO_OK:
        raise GpboError(code, where)


def strerror(code):
    return _strerror(code).decode()


def _ptr(a):
    """Device or host address of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


def _is_host(a):
    return a is None or isinstance(a, np.ndarray)


def _hyper(lengthscale, signal_var, noise_var):
    ls = np.ascontiguousarray(lengthscale, dtype=np.float64)
    h = GpHyper(len(ls), ls.ctypes.data_as(_D), float(signal_var), float(noise_var))
    return h, ls


class Context:
    """A gpbo_ctx on one device, ordered on `stream` (a torch.cuda.Stream, a raw
    cudaStream_t as int, or None for a stream the library owns)."""

    def __init__(self, device: int = 0, stream=None):
        self._h = _P()
        self._models = weakref.WeakSet()
        check(_create(C.byref(self._h), device, _stream_handle(stream)), "gpbo_create")
        self.device = device

    def close(self):
        """Free every live model of this context, then the context itself."""
        if self._h:
            for m in list(self._models):
                m.free()
            _destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        check(_set_stream(self._h, _stream_handle(stream)), "gpbo_set_stream")

    def set_workspace_limit(self, nbytes: int):
        check(_ws_limit(self._h, int(nbytes)), "gpbo_set_workspace_limit")

    @property
    def launches(self) -> int:
        return int(_launches(self._h))

    def trace(self, on: bool):
        """Start (clearing) or stop per-phase CUDA-event timing on the context's stream."""
        check(_trace_en(self._h, 1 if on else 0), "gpbo_trace_enable")

    def probe_fma(self, kind: str) -> float:
        """Measured FMA throughput in TFLOP/s: kind "f64" (DFMA) or "f32" (FFMA)."""
        v = C.c_double(0.0)
        check(_probe(self._h, 0 if kind == "f64" else 1, C.byref(v)), "gpbo_probe_fma")
        return float(v.value)

    def set_wait_limit(self, cycles: int):
        """Limit, in SM clock cycles, of the library's bounded device waits (0 = default)."""
        check(_wait_limit(self._h, int(cycles)), "gpbo_set_wait_limit")

    def inject_wait_stall(self, on):
        """Failure injection for tests: the tensor-core variance epilogue waits on a barrier
        that nothing arrives at, so the scoring call returns GPBO_ETIMEOUT."""
        check(_inject_stall(self._h, int(on)), "gpbo_inject_wait_stall")

    def trace_read(self):
        n = len(PHASES)
        ms = (C.c_double * n)()
        cnt = (C.c_int64 * n)()
        fl = (C.c_double * n)()
        check(_trace_rd(self._h, n, ms, cnt, fl), "gpbo_trace_read")
        return {p: {"ms": ms[i], "intervals": int(cnt[i]), "flops": fl[i]} for i, p in enumerate(PHASES)}

    # ------------------------------------------------------------ fit / score
    def fit(self, X, y, lengthscale, signal_var, noise_var, prec="f64", jitter=False):
        """X (n x d) and y (n): both torch float64 CUDA tensors, or both numpy arrays."""
        host = _is_host(X)
        if host:
            X = np.ascontiguousarray(X, dtype=np.float64)
            y = np.ascontiguousarray(y, dtype=np.float64)
        n, d = X.shape
        h, keep = _hyper(lengthscale, signal_var, noise_var)
        flags = (HOST_PTRS if host else 0) | (JITTER if jitter else 0)
        out = _P()
        check(_fit(self._h, _ptr(X), _ptr(y), n, d, C.byref(h), PREC[prec], flags, C.byref(out)), "gp_fit")
        m = Model(self, out, prec)
        self._models.add(m)
        return m

    # ------------------------------------------------------------ a BO search
    def bo_search(self, fn, x_init, budget, M, seed, lengthscale, signal_var, noise_var, prec="f64", refit=False,
                  xi=0.0, mle_iters=0):
        """fn(u) -> float for u (k,) in the unit cube (called on the host); x_init (n_init x k).
        Returns (X (budget x k), y (budget,), index of the best y)."""
        x_init = np.ascontiguousarray(np.atleast_2d(x_init), dtype=np.float64)
        n_init, k = x_init.shape
        err = []

        def tramp(up, kk, fp, user):
            try:
                fp[0] = float(fn(np.ctypeslib.as_array(up, shape=(kk,)).copy()))
                return 0
            except Exception as e:  # reported after the call returns
                err.append(e)
                return 1

        cb = EVAL_FN(tramp)
        ls = np.ascontiguousarray(np.broadcast_to(np.asarray(lengthscale, dtype=np.float64), (k,)))
        o = BoOpts(int(budget), n_init, x_init.ctypes.data_as(_D), int(M), int(seed), PREC[prec], int(bool(refit)),
                   GpHyper(k, ls.ctypes.data_as(_D), float(signal_var), float(noise_var)), float(xi), int(mle_iters))
        X = np.empty((budget, k))
        y = np.empty(budget)
        best = C.c_int(-1)
        code = _bo(self._h, k, cb, None, C.byref(o), X.ctypes.data_as(_D), y.ctypes.data_as(_D), C.byref(best))
        if err:
            raise err[0]
        check(code, "bo_search")
        return X, y, int(best.value)

    # ------------------------------------------------------------ hyperparameters
    def lml(self, X, y, lengthscale, signal_var, noise_var):
        """Log marginal likelihood and its gradient over (log l_1..l_d, log signal_var,
        log noise_var).  X, y: torch float64 CUDA tensors or numpy arrays."""
        host = _is_host(X)
        if host:
            X = np.ascontiguousarray(X, dtype=np.float64)
            y = np.ascontiguousarray(y, dtype=np.float64)
        n, d = X.shape
        h, keep = _hyper(lengthscale, signal_var, noise_var)
        v = C.c_double()
        g = np.empty(d + 2)
        check(_lml(self._h, _ptr(X), _ptr(y), n, d, C.byref(h), HOST_PTRS if host else 0, C.byref(v),
                   g.ctypes.data_as(_D)), "gp_lml")
        return v.value, g

    def fit_mle(self, X, y, theta0, lo, hi, max_iter=200, gtol=1e-6):
        """Maximise the LML over the box [lo, hi] of log parameters from each row of theta0
        (n_starts x (d + 2)).  Returns (theta, lml, evaluations)."""
        host = _is_host(X)
        if host:
            X = np.ascontiguousarray(X, dtype=np.float64)
            y = np.ascontiguousarray(y, dtype=np.float64)
        n, d = X.shape
        t0 = np.ascontiguousarray(np.atleast_2d(theta0), dtype=np.float64)
        lo = np.ascontiguousarray(np.broadcast_to(np.asarray(lo, dtype=np.float64), (d + 2,)))
        hi = np.ascontiguousarray(np.broadcast_to(np.asarray(hi, dtype=np.float64), (d + 2,)))
        assert t0.shape[1] == d + 2
        th = np.empty(d + 2)
        v = C.c_double()
        ev = C.c_int64()
        check(_fit_mle(self._h, _ptr(X), _ptr(y), n, d, t0.shape[0], t0.ctypes.data_as(_D), lo.ctypes.data_as(_D),
                       hi.ctypes.data_as(_D), int(max_iter), float(gtol), HOST_PTRS if host else 0,
                       th.ctypes.data_as(_D), C.byref(v), C.byref(ev)), "gp_fit_mle")
        return th, v.value, int(ev.value)

    def posterior_ei(self, model, Xc=None, M=None, seed=0, y_best=0.0, xi=0.0, mu=None, sigma=None, ei=None):
        """Xc: M x d float32 torch CUDA tensor / numpy array, or None with M and seed.
        mu/sigma/ei: preallocated outputs of the same kind (or None).  Returns (argmax, ei_max)."""
        host = Xc is not None and _is_host(Xc) or any(isinstance(a, np.ndarray) for a in (mu, sigma, ei))
        if Xc is not None:
            if isinstance(Xc, np.ndarray):
                Xc = np.ascontiguousarray(Xc, dtype=np.float32)
            M = Xc.shape[0]
        am = C.c_int64(-1)
        em = C.c_double(0.0)
        check(_posterior(self._h, model._h, _ptr(Xc), int(M), int(seed), float(y_best), float(xi),
                         HOST_PTRS if host else 0, _ptr(mu), _ptr(sigma), _ptr(ei), C.byref(am), C.byref(em)),
              "gp_posterior_ei")
        return int(am.value), float(em.value)

    def posterior_ei_noalloc(self, model, Xc=None, M=None, seed=0, y_best=0.0, xi=0.0, mu=None, sigma=None,
                             ei=None):
        """Allocation-free scoring of an FP32/FP64 model: the library allocates nothing
        during the call.  Every array is a device tensor the caller already owns."""
        if Xc is not None:
            M = Xc.shape[0]
        am = C.c_int64(-1)
        em = C.c_double(0.0)
        check(_posterior_noalloc(self._h, model._h, _ptr(Xc), int(M), int(seed), float(y_best), float(xi), _ptr(mu),
                                 _ptr(sigma), _ptr(ei), C.byref(am), C.byref(em)), "gp_posterior_ei_noalloc")
        return int(am.value), float(em.value)

    def gen_candidates(self, out, seed, first=0):
        M, d = out.shape
        check(_gen(self._h, int(seed), int(first), int(M), int(d), _ptr(out)), "gpbo_gen_candidates")
        return out

    def search_step(self, X, y, lengthscale, signal_var, noise_var, Xc=None, M=None, seed=0, xi=0.0, prec="f64",
                    jitter=False):
        host = _is_host(X)
        if host:
            X = np.ascontiguousarray(X, dtype=np.float64)
            y = np.ascontiguousarray(y, dtype=np.float64)
            if Xc is not None:
                Xc = np.ascontiguousarray(Xc, dtype=np.float32)
        n, d = X.shape
        if Xc is not None:
            M = Xc.shape[0]
        h, keep = _hyper(lengthscale, signal_var, noise_var)
        x_next = np.empty(d)
        em = C.c_double(0.0)
        am = C.c_int64(-1)
        flags = (HOST_PTRS if host else 0) | (JITTER if jitter else 0)
        check(_step(self._h, _ptr(X), _ptr(y), n, d, C.byref(h), _ptr(Xc), int(M), int(seed), float(xi), PREC[prec],
                    flags, x_next.ctypes.data, C.byref(em), C.byref(am)), "search_step")
        return {"x_next": x_next, "ei_max": float(em.value), "argmax": int(am.value)}

    def search_step_batched(self, problems, xi=0.0, prec="f32"):
        """problems: list of dicts with X (n x d), y (n), lengthscale, signal_var, noise_var, M, seed.
        X and y are all numpy arrays (host) or all torch CUDA tensors (device)."""
        G = len(problems)
        host = isinstance(problems[0]["X"], np.ndarray)
        keep = []
        Xp = (_P * G)()
        yp = (_P * G)()
        ns = np.zeros(G, dtype=np.int32)
        ds = np.zeros(G, dtype=np.int32)
        Ms = np.zeros(G, dtype=np.int64)
        seeds = (C.c_uint64 * G)()
        hyps = (GpHyper * G)()
        for g, pb in enumerate(problems):
            X, y = pb["X"], pb["y"]
            if host:
                X = np.ascontiguousarray(X, dtype=np.float64)
                y = np.ascontiguousarray(y, dtype=np.float64)
            keep += [X, y]
            Xp[g] = _ptr(X)
            yp[g] = _ptr(y)
            ns[g], ds[g] = X.shape
            Ms[g] = int(pb["M"])
            seeds[g] = int(pb["seed"])
            h, ls = _hyper(pb["lengthscale"], pb["signal_var"], pb["noise_var"])
            keep.append(ls)
            hyps[g] = h
        x_next = np.zeros((G, 64))
        ei_max = np.zeros(G)
        am = np.zeros(G, dtype=np.int64)
        self._batched_G = G
        check(_step_batched(self._h, G, Xp, yp, ns.ctypes.data_as(_I), ds.ctypes.data_as(_I), hyps,
                            Ms.ctypes.data_as(_L), seeds, float(xi), PREC[prec], HOST_PTRS if host else 0,
                            x_next.ctypes.data_as(_D), ei_max.ctypes.data_as(_D), am.ctypes.data_as(_L)),
              "search_step_batched")
        return {"x_next": [x_next[g, :ds[g]] for g in range(G)], "ei_max": ei_max, "argmax": am}

    def batched_tile(self, tile=0):
        """Variance tile of the batched step (64, 128, 256), or 0 for the autotuner."""
        check(_batched_tile(self._h, int(tile)), "search_step_batched_tile")

    def batched_tuning(self, members=False):
        """(tile in use, {tile: autotuner ms per launch}) of the batched plan that holds the
        largest problems of the last call; with members=True also a boolean array over that
        call's problems marking the ones in that plan."""
        t = C.c_int(0)
        ms = (C.c_float * 3)()
        mem = np.zeros(max(getattr(self, "_batched_G", 0), 1), dtype=np.int32)
        check(_batched_tuning(self._h, C.byref(t), ms, mem.ctypes.data_as(_I)), "search_step_batched_tuning")
        out = (t.value, {k: float(v) for k, v in zip((64, 128, 256), ms) if v >= 0})
        return out + (mem[:getattr(self, "_batched_G", 0)].astype(bool),) if members else out

    # ------------------------------------------------------------ screen
    def screen(self, block_dim=None, block_fn=None, noise_sd=0.0, seed=0, n_base=32, h=0.1, cutoff=0.25,
               max_dims=10, mode=SCREEN_PAIRWISE, host_fn=None, d=None, n_routines=0, param_owner=None,
               growth=0.1, lo=None, hi=None):
        """Built-in block objective (block_dim, block_fn) or a host black box
        host_fn(x: np.ndarray) -> (f_total, routines) with d / n_routines / param_owner
        (-1 for a shared parameter).  mode SCREEN_ROUTINE_SERIES: n_base variations per
        parameter, each `growth` above the last, in the ranges lo / hi of a host black box."""
        keep = []
        if host_fn is None:
            bd = np.ascontiguousarray(block_dim, dtype=np.int32)
            bf = np.ascontiguousarray(block_fn, dtype=np.int32)
            keep += [bd, bf]
            d = int(bd.sum())
            obj = GpboObjective(len(bd), bd.ctypes.data_as(_I), bf.ctypes.data_as(_I), float(noise_sd), int(seed),
                                HOST_FN(), 0, C.cast(None, _I), None)
            R = len(bd)
        else:
            def tramp(xp, dd, ft, fr, user):
                try:
                    x = np.ctypeslib.as_array(xp, shape=(dd,)).copy()
                    tot, rout = host_fn(x)
                    ft[0] = float(tot)
                    for g in range(n_routines):
                        fr[g] = float(rout[g])
                    return 0
                except Exception:
                    return 1
            cb = HOST_FN(tramp)
            keep.append(cb)
            ow = np.ascontiguousarray(param_owner if param_owner is not None else np.zeros(d), dtype=np.int32)
            keep.append(ow)
            obj = GpboObjective(0, C.cast(None, _I), C.cast(None, _I), 0.0, int(seed), cb, int(n_routines),
                                ow.ctypes.data_as(_I), None)
            R = n_routines
        lo_a = None if lo is None else np.ascontiguousarray(np.broadcast_to(np.asarray(lo, dtype=np.float64), (d,)))
        hi_a = None if hi is None else np.ascontiguousarray(np.broadcast_to(np.asarray(hi, dtype=np.float64), (d,)))
        keep += [lo_a, hi_a]
        opts = ScreenOpts(int(mode), int(n_base), float(h), float(cutoff), int(max_dims), int(seed), float(growth),
                          C.cast(None, _D) if lo_a is None else lo_a.ctypes.data_as(_D),
                          C.cast(None, _D) if hi_a is None else hi_a.ctypes.data_as(_D))
        rows = d if mode == SCREEN_PAIRWISE else R
        score = np.zeros((rows, d))
        infl = np.zeros(d)
        group = np.zeros(d, dtype=np.int32)
        fixed = np.zeros(d, dtype=np.int32)
        ng = C.c_int(0)
        check(_screen(self._h, C.byref(obj), d, C.byref(opts), score.ctypes.data, infl.ctypes.data,
                      group.ctypes.data, C.byref(ng), fixed.ctypes.data), "interdep_screen")
        return {"score": score, "influence": infl, "group_of": group, "n_groups": int(ng.value), "fixed": fixed}


class Surrogate:
    """Ensemble pre-screen network (learned form of candidate scoring)."""

    def __init__(self, ctx, E=8, d=20, H=256, seed=5):
        self.ctx = ctx
        self.E, self.d, self.H = E, d, H
        self.P = d * H + H + H * H + H + 2 * H + 2
        self._h = _P()
        check(_mlp_create(ctx._h, E, d, H, int(seed), C.byref(self._h)), "mlp_create")
        ctx._models.add(self)   # freed before the context

    def free(self):
        if self._h:
            _mlp_free(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def params(self, new=None):
        out = np.empty((self.E, self.P), dtype=np.float32)
        inp = None if new is None else np.ascontiguousarray(new, dtype=np.float32)
        check(_mlp_params(self._h, out.ctypes.data, None if inp is None else inp.ctypes.data), "mlp_params")
        return out

    def forward(self, X, out):
        check(_mlp_forward(self.ctx._h, self._h, _ptr(X), int(X.shape[0]), _ptr(out)), "mlp_forward")
        return out

    def gradients(self, X, T):
        g = np.empty((self.E, self.P), dtype=np.float32)
        loss = np.empty(self.E, dtype=np.float32)
        check(_mlp_grads(self.ctx._h, self._h, _ptr(X), _ptr(T), int(X.shape[0]), g.ctypes.data, loss.ctypes.data),
              "mlp_gradients")
        return loss, g

    def train(self, X, mu, sigma, steps, batch=1024, lr=1e-3, seed=7):
        fl = C.c_float(0.0)
        check(_mlp_train(self.ctx._h, self._h, _ptr(X), _ptr(mu), _ptr(sigma), int(X.shape[0]), int(steps),
                         int(batch), float(lr), int(seed), C.byref(fl)), "mlp_train")
        return float(fl.value)

    def norm(self):
        v = np.empty(4)
        check(_mlp_norm(self._h, v.ctypes.data_as(_D)), "mlp_norm")
        return v

    def score(self, ei, X=None, M=None, seed=0, y_best=0.0, xi=0.0, prec="f16", mu=None, sigma=None):
        """Ensemble (EI, mu_bar, sigma_bar) of rows of X (device) or of M seeded candidates.
        prec "f16": tensor-core kernel (FP16 operands); "f32": CUDA-core forward."""
        if X is not None:
            M = X.shape[0]
        check(_mlp_score(self.ctx._h, self._h, _ptr(X), int(M), int(seed), float(y_best), float(xi), PREC[prec],
                         _ptr(ei), _ptr(mu), _ptr(sigma)), "mlp_score")
        return ei

    def screen(self, model, M, seed, k, y_best, xi=0.0, ei_pool=None, want_top=False):
        am = C.c_int64(-1)
        em = C.c_double(0.0)
        top = np.empty(k, dtype=np.int64) if want_top else None
        check(_screen_sur(self.ctx._h, model._h, self._h, int(M), int(seed), int(k), float(y_best), float(xi),
                          _ptr(ei_pool), None if top is None else top.ctypes.data, C.byref(am), C.byref(em)),
              "surrogate_screen")
        return int(am.value), float(em.value), top


class Model:
    def __init__(self, ctx, handle, prec):
        self.ctx = ctx
        self._h = handle
        self.prec = prec

    def free(self):
        if self._h:
            _model_free(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def info(self):
        n, d, p = C.c_int(), C.c_int(), C.c_int()
        sn2 = C.c_double()
        check(_model_info(self._h, C.byref(n), C.byref(d), C.byref(p), C.byref(sn2)), "gp_model_info")
        return {"n": n.value, "d": d.value, "prec": p.value, "noise_var": sn2.value}

    def read(self):
        inf = self.info()
        n = inf["n"]
        Lm = np.empty((n, n))
        alpha = np.empty(n)
        check(_model_read(self._h, Lm.ctypes.data, alpha.ctypes.data), "gp_model_read")
        return Lm, alpha


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream
