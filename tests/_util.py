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
