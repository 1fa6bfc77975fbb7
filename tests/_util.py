"""Shared helpers of the GPU parity tests.

Error metric (a reading of "rel 1e-4 / 2e-3" that survives the cancellation in
sigma^2 = s2 - |v|^2 near observations): err(q) = max_c |q_gpu - q_ref| / (|q_ref| + S_q)
with S = sqrt(signal_var) for mu and sigma and S = max EI_ref for EI.
Bars: FP64 1e-9, FP32 1e-4, BF16/FP16 tensor tiles 2e-3.

Argmax agreement: bit-exact when the oracle's relative margin between its best and
second-best EI exceeds the bar; otherwise the GPU's pick must have oracle EI within
the bar of the oracle's maximum."""
import numpy as np

BAR = {"f64": 1e-9, "f32": 1e-4, "bf16": 2e-3, "f16": 2e-3}


def scaled_err(q, ref, S):
    q = np.asarray(q, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(q - ref) / (np.abs(ref) + S)))


def check_argmax(idx_gpu, ei_ref, bar):
    order = np.argsort(-ei_ref, kind="stable")
    best, second = ei_ref[order[0]], ei_ref[order[1]] if len(order) > 1 else 0.0
    margin = (best - second) / best if best > 0 else 0.0
    if margin > bar:
        assert idx_gpu == int(np.argmax(ei_ref)), (idx_gpu, int(np.argmax(ei_ref)), margin)
        return "exact"
    assert ei_ref[idx_gpu] >= best * (1 - bar), (idx_gpu, ei_ref[idx_gpu], best)
    return "near-tie"


def to_dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


# ---------------------------------------------------------------- FP16 ensemble forward tolerance
U_F16 = 2.0 ** -11  # unit roundoff of FP16 (11-bit significand)


def _gelu(z):
    import scipy.special
    return 0.5 * z * scipy.special.erfc(-z / np.sqrt(2.0))


def _gelu_slope(z):
    import scipy.special
    return 0.5 * scipy.special.erfc(-z / np.sqrt(2.0)) + z * np.exp(-0.5 * z * z) / np.sqrt(2 * np.pi)


def _gelu_tanh(z):
    return 0.5 * z * (1 + np.tanh(np.sqrt(2 / np.pi) * (z + 0.044715 * z ** 3)))


def f16_round(a):
    """Round to FP32, then to the nearest FP16 value (ties to even), as the kernel's FP32 ->
    FP16 conversions do; returned as float64."""
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float16).astype(np.float64)


def f16_ensemble_tol(orc, thetas, X, d, H, nm, tau, lam=6.0):
    """Tolerances (mu_bar, sigma_bar, ei) of the FP16 tensor-core ensemble against the FP64
    oracle, per candidate, derived from the kernel's arithmetic in two parts.
    (1) Deterministic: x, W1, b1, W2 (halved, exactly) and H1 rounded to FP16, GELU in the
        tanh form.  A float64 emulation with exactly these roundings gives
        |emulation - oracle|.
    (2) What the emulation cannot reproduce: tanh.approx.f32's relative error (2^-11) on
        each tanh, the FP32 accumulation, and the H1 roundings that this moves across an
        FP16 rounding boundary (one ulp, 2u|h1|, with probability about delta / (2u|h1|), so
        expected square delta * 2u|h1|).  These vary in sign from element to
        element, so they are propagated as a root sum of squares through the next layer's
        weights (the sqrt(n) growth of Higham & Mary, SIAM J. Sci. Comput. 2019); lam is the
        number of standard deviations allowed."""
    from scipy.stats import norm
    u = U_F16
    X = np.asarray(X, dtype=np.float64)
    Xq = f16_round(X)
    mus, emus, dmus, ss, ess, dss = [], [], [], [], [], []
    for th in np.asarray(thetas, dtype=np.float64):
        W1, b1, W2, b2, W3, b3 = [p.reshape(s) for p, (_, s) in zip(orc.mlp_split(th, d, H), orc.mlp_sizes(d, H))]
        # reference (exact GELU, FP64) and emulation of the kernel's roundings
        o = _gelu(_gelu(X @ W1 + b1) @ W2 + b2) @ W3 + b3
        z1 = Xq @ f16_round(W1) + f16_round(b1)
        h1 = f16_round(_gelu_tanh(z1))           # the kernel stores fp16(2 gelu) = 2 fp16(gelu)
        z2 = h1 @ (2.0 * f16_round(0.5 * W2)) + b2
        h2 = _gelu_tanh(z2)
        oe = h2 @ W3 + b3
        # residual, per element: tanh.approx.f32 (2^-11 relative, times |z|/2) and the FP32
        # accumulation of z1
        t1 = np.abs(z1) * 2.0 ** -12 + 1e-7 * (np.abs(Xq) @ np.abs(W1) + 1)
        dh1 = np.sqrt(t1 ** 2 + t1 * 2 * u * np.abs(h1))
        dz2 = np.sqrt((dh1 ** 2) @ (W2 ** 2)) + 1e-7 * (np.abs(h1) @ np.abs(W2) + 1)
        dh2 = np.sqrt((_gelu_slope(z2) * dz2) ** 2 + (np.abs(z2) * 2.0 ** -12) ** 2)
        do = np.sqrt((dh2 ** 2) @ (W3 ** 2)) + 1e-7 * (np.abs(h2) @ np.abs(W3) + 1)
        for out, oo in ((mus, o), (emus, oe)):
            out.append(oo[:, 0] * nm[1] + nm[0])
        ss.append(np.exp(o[:, 1] * nm[3] + nm[2]))
        ess.append(np.exp(oe[:, 1] * nm[3] + nm[2]))
        dmus.append(nm[1] * do[:, 0])
        dss.append(ess[-1] * nm[3] * do[:, 1])
    mus, emus, dmus, ss, ess, dss = map(np.array, (mus, emus, dmus, ss, ess, dss))
    E = mus.shape[0]

    def combine(m, s):
        mb = m.mean(0)
        return mb, np.sqrt((s ** 2).mean(0) + ((m - mb) ** 2).mean(0))

    mbar, sbar = combine(mus, ss)
    embar, esbar = combine(emus, ess)
    dm = np.sqrt((dmus ** 2).sum(0)) / E
    dvar = np.sqrt(((2 * ess * dss) ** 2 + (2 * (emus - embar) * dmus) ** 2).sum(0)) / E
    ds = dvar / (2 * esbar)
    z = (tau - mbar) / sbar
    ez = (tau - embar) / esbar
    ei = (tau - mbar) * norm.cdf(z) + sbar * norm.pdf(z)
    eei = (tau - embar) * norm.cdf(ez) + esbar * norm.pdf(ez)
    dei = np.sqrt((norm.cdf(ez) * dm) ** 2 + (norm.pdf(ez) * ds) ** 2)
    return (np.abs(embar - mbar) + lam * dm + 1e-6 * (np.abs(mbar) + 1),
            np.abs(esbar - sbar) + lam * ds + 1e-6 * sbar,
            np.abs(eei - ei) + lam * dei + 1e-6 * sbar)
