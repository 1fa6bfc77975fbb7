"""The allocation-free scoring entry point, gp_posterior_ei_noalloc.

It exists for callers that must not allocate device memory while they run (a serving
loop whose memory belongs to a pooling allocator, a process under a hard memory cap):
its scratch is one fixed 4 MiB array inside the library.  These tests call it through
the C ABI twice in a row and compare each result with gp_posterior_ei's on the same
inputs, within the FP32 / FP64 tolerances of the other parity tests.  The second call
scores a pool whose best EI is strictly below the first call's, so scratch left over
from the first call (the running best) would show up as a wrong argmax.

This file sorts last so that a run stopping at the first failure has run every other
test already; it also passes on its own in a fresh process."""
import numpy as np
import pytest

from paper_2403_08131_b300 import workloads as W
from tests._util import BAR, scaled_err, to_dev

pytestmark = pytest.mark.gpu


def _outputs(M, dt, torch):
    return [torch.empty(M, dtype=dt, device="cuda") for _ in range(3)]


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_noalloc_equals_allocating_path_on_two_calls(prec):
    import torch
    from paper_2403_08131_b300 import gpbo

    ctx = gpbo.Context(0, torch.cuda.current_stream())
    dt = torch.float64 if prec == "f64" else torch.float32
    w = W.config2()
    ys = (w.y - w.y.mean()) / w.y.std()
    m = ctx.fit(to_dev(w.X), to_dev(ys), w.lengthscale, 1.0, w.noise_var, prec=prec)
    tau = float(ys.min())
    pool_a = w.candidates(20000)              # several scratch chunks for n = 512
    # pool B drops pool A's 200 best candidates, so its best EI is below pool A's
    mu, sg, ei = _outputs(len(pool_a), dt, torch)
    ctx.posterior_ei(m, to_dev(pool_a), y_best=tau, mu=mu, sigma=sg, ei=ei)
    keep = np.argsort(-ei.cpu().numpy(), kind="stable")[200:]
    pool_b = pool_a[np.sort(keep)]
    bar = BAR[prec]
    best = []
    for pool in (pool_a, pool_b):
        Xc = to_dev(pool)
        ref = _outputs(len(pool), dt, torch)
        am_r, em_r = ctx.posterior_ei(m, Xc, y_best=tau, mu=ref[0], sigma=ref[1], ei=ref[2])
        got = _outputs(len(pool), dt, torch)
        am, em = ctx.posterior_ei_noalloc(m, Xc, y_best=tau, mu=got[0], sigma=got[1], ei=got[2])
        r = [t.cpu().numpy() for t in ref]
        g = [t.cpu().numpy() for t in got]
        assert scaled_err(g[0], r[0], 1.0) <= bar
        assert scaled_err(g[1], r[1], 1.0) <= bar
        assert scaled_err(g[2], r[2], r[2].max()) <= bar
        assert am == am_r and abs(em - em_r) <= bar * abs(em_r)
        best.append(em)
    assert best[1] < best[0]
    # optional outputs may be omitted; the seeded pool is drawn on the device as usual
    am_s, em_s = ctx.posterior_ei_noalloc(m, None, M=3000, seed=w.seed, y_best=tau)
    am_t, em_t = ctx.posterior_ei(m, None, M=3000, seed=w.seed, y_best=tau)
    assert am_s == am_t and abs(em_s - em_t) <= bar * abs(em_t)
    ctx.close()


def test_noalloc_rejects_what_does_not_fit_and_16bit_models():
    import torch
    from paper_2403_08131_b300 import gpbo

    ctx = gpbo.Context(0, torch.cuda.current_stream())
    # FP64 with n_pad = 8192 leaves room for fewer than 64 candidates per chunk in 4 MiB
    n, d = 8192, 4
    X = W.uniform_points(5, W.STREAM_OBS, n, d)
    y = np.sin(X.sum(1))
    m = ctx.fit(to_dev(X), to_dev(y), W.lengthscale_rule(d), 1.0, 1e-4, prec="f64")
    with pytest.raises(gpbo.GpboError) as e:
        ctx.posterior_ei_noalloc(m, None, M=128, seed=1, y_best=0.0)
    assert e.value.code == gpbo.GPBO_ESCRATCH
    m16 = ctx.fit(to_dev(X[:300]), to_dev(y[:300]), W.lengthscale_rule(d), 1.0, 1e-4, prec="f16")
    with pytest.raises(gpbo.GpboError) as e:
        ctx.posterior_ei_noalloc(m16, None, M=128, seed=1, y_best=0.0)
    assert e.value.code == gpbo.GPBO_ENOTSUP
    ctx.close()
