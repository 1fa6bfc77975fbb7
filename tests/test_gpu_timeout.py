"""The bounded-wait error path (GPBO_ETIMEOUT), run without a fault: a short wait limit and
an injected wait on a barrier that nothing arrives at make the tensor-core variance
kernel's wait run out.  Every role of the kernel then leaves its loop, drains its own
copies and MMAs, frees its tensor memory and exits; the call reports GPBO_ETIMEOUT and the
context keeps working."""
import numpy as np
import pytest

from paper_2403_08131_b300 import workloads as W
from tests._util import to_dev

pytestmark = pytest.mark.gpu


def _score(ctx, m, Xc, tau):
    import torch
    M = Xc.shape[0]
    out = [torch.empty(M, dtype=torch.float32, device="cuda") for _ in range(3)]
    am, em = ctx.posterior_ei(m, Xc, y_best=tau, mu=out[0], sigma=out[1], ei=out[2])
    return am, em, [t.cpu().numpy() for t in out]


def test_wait_timeout_reports_and_context_recovers(ctx):
    from paper_2403_08131_b300 import gpbo
    w = W.make_gp_workload("t", 2405, 512, W.five_block_objective(2405), 4096, "f16")
    ys = (w.y - w.y.mean()) / w.y.std()
    tau = float(ys.min())
    m = ctx.fit(to_dev(w.X), to_dev(ys), w.lengthscale, 1.0, w.noise_var, prec="f16")
    Xc = to_dev(w.candidates())
    ref = _score(ctx, m, Xc, tau)
    ctx.set_wait_limit(200_000)           # about 0.1 ms of SM clock
    ctx.inject_wait_stall(True)
    try:
        with pytest.raises(gpbo.GpboError) as e:
            _score(ctx, m, Xc, tau)
        assert e.value.code == gpbo.GPBO_ETIMEOUT
        # the error bit is read and cleared by the failing call: it does not leak into the next
        ctx.inject_wait_stall(False)
        ctx.set_wait_limit(0)
    finally:
        ctx.inject_wait_stall(False)
        ctx.set_wait_limit(0)
    # every CTA released its tensor memory, so the same kernel runs again on every SM,
    # with the same results as before the failure
    for _ in range(2):
        am, em, outs = _score(ctx, m, Xc, tau)
        assert am == ref[0] and em == ref[1]
        assert all(np.array_equal(a, b) for a, b in zip(outs, ref[2]))
    m.free()


def test_wait_controls_reject_bad_arguments(ctx):
    from paper_2403_08131_b300 import gpbo
    with pytest.raises(gpbo.GpboError) as e:
        ctx.set_wait_limit(-1)
    assert e.value.code == gpbo.GPBO_EINVAL
    with pytest.raises(gpbo.GpboError) as e:
        ctx.inject_wait_stall(2)
    assert e.value.code == gpbo.GPBO_EINVAL
