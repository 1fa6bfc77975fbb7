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


# ---------------------------------------------------------------- BF16 ensemble forward tolerance
U_BF16 = 2.0 ** -8  # unit roundoff of BF16 (8-bit significand)


def _gelu(z):
    import scipy.special
    return 0.5 * z * scipy.special.erfc(-z / np.sqrt(2.0))


def _gelu_slope(z):
    import scipy.special
    return 0.5 * scipy.special.erfc(-z / np.sqrt(2.0)) + z * np.exp(-0.5 * z * z) / np.sqrt(2 * np.pi)


def _gelu_tanh_gap(z):
    """|tanh-form GELU - z Phi(z)| plus tanh.approx's relative error (2^-11) times |z|/2."""
    t = 0.5 * z * (1 + np.tanh(np.sqrt(2 / np.pi) * (z + 0.044715 * z ** 3)))
    return np.abs(t - _gelu(z)) + np.abs(z) * 2.0 ** -12


def bf16_ensemble_tol(orc, thetas, X, d, H, nm, tau, lam=6.0):
    """Tolerances (mu_bar, sigma_bar, ei) of the BF16 tensor-core ensemble against the FP64
    oracle, per candidate.  x, W1, b1, W2 and H1 are rounded to BF16 (unit roundoff u); b2,
    W3, b3 and H2 stay FP32; GELU is the tanh form.  Rounding errors of an n-term sum grow
    like sqrt(n) u with high probability (Higham & Mary, SIAM J. Sci. Comput. 2019), so each
    layer's error is propagated as a root sum of squares through the next layer's weights;
    lam is the number of standard deviations allowed."""
    from scipy.stats import norm
    u = U_BF16
    mus, dmus, ss, dss = [], [], [], []
    for th in np.asarray(thetas, dtype=np.float64):
        W1, b1, W2, b2, W3, b3 = [p.reshape(s) for p, (_, s) in zip(orc.mlp_split(th, d, H), orc.mlp_sizes(d, H))]
        z1 = X @ W1 + b1
        dz1 = u * np.sqrt(2 * (X ** 2) @ (W1 ** 2) + b1 ** 2) + 1e-7
        h1 = _gelu(z1)
        dh1 = np.sqrt((_gelu_slope(z1) * dz1) ** 2 + _gelu_tanh_gap(z1) ** 2 + (u * h1) ** 2)
        z2 = h1 @ W2 + b2
        dz2 = np.sqrt((dh1 ** 2 + (u * h1) ** 2) @ (W2 ** 2)) + 1e-7
        h2 = _gelu(z2)
        dh2 = np.sqrt((_gelu_slope(z2) * dz2) ** 2 + _gelu_tanh_gap(z2) ** 2)
        o = h2 @ W3 + b3
        do = np.sqrt((dh2 ** 2) @ (W3 ** 2)) + 1e-7
        mu, s = o[:, 0] * nm[1] + nm[0], np.exp(o[:, 1] * nm[3] + nm[2])
        mus.append(mu)
        dmus.append(nm[1] * do[:, 0])
        ss.append(s)
        dss.append(s * nm[3] * do[:, 1])
    mus, dmus, ss, dss = map(np.array, (mus, dmus, ss, dss))
    E = mus.shape[0]
    mbar = mus.mean(0)
    sbar = np.sqrt((ss ** 2).mean(0) + ((mus - mbar) ** 2).mean(0))
    dm = np.sqrt((dmus ** 2).sum(0)) / E
    dvar = np.sqrt(((2 * ss * dss) ** 2 + (2 * (mus - mbar) * dmus) ** 2).sum(0)) / E
    ds = dvar / (2 * sbar)
    z = (tau - mbar) / sbar
    dei = np.sqrt((norm.cdf(z) * dm) ** 2 + (norm.pdf(z) * ds) ** 2)
    return (lam * dm + 1e-6 * (np.abs(mbar) + 1), lam * ds + 1e-6 * sbar, lam * dei + 1e-6 * sbar)
