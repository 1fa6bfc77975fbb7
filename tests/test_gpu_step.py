"""One BO iteration (standardise, fit, score, argmax, gather) against the oracle."""
import numpy as np
import pytest

from paper_2403_08131_b300 import workloads as W
from tests._util import BAR, check_argmax, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("host", [True, False])
def test_step_rosenbrock_f64(ctx, orc, host):
    w = W.config1()
    Xc = w.candidates()
    ref = orc.search_step(w.X, w.y, w.lengthscale, 1.0, w.noise_var, Xc=Xc.astype(np.float64), want_arrays=True)
    X, y, C = (w.X, w.y, Xc) if host else (to_dev(w.X), to_dev(w.y), to_dev(Xc))
    got = ctx.search_step(X, y, w.lengthscale, 1.0, w.noise_var, Xc=C, prec="f64")
    assert check_argmax(got["argmax"], ref["ei"], BAR["f64"]) == "exact"
    assert np.array_equal(got["x_next"], ref["x_next"])
    assert abs(got["ei_max"] - ref["ei_max"]) <= 1e-9 * ref["ei_max"]


@pytest.mark.parametrize("prec", ["f32", "bf16", "f16"])
def test_step_fiveblock_seeded(ctx, orc, prec):
    w = W.config2()
    M = 16384
    ref = orc.search_step(w.X, w.y, w.lengthscale, 1.0, w.noise_var, M=M, seed=w.seed, want_arrays=True)
    got = ctx.search_step(w.X, w.y, w.lengthscale, 1.0, w.noise_var, M=M, seed=w.seed, prec=prec)
    check_argmax(got["argmax"], ref["ei"], BAR[prec])
    assert np.array_equal(got["x_next"], w.candidates(M)[got["argmax"]].astype(np.float64))
    assert abs(got["ei_max"] - ref["ei_max"]) <= BAR[prec] * ref["ei_max"] * 2


def test_step_rejects_nan_and_bad_sizes(ctx):
    from paper_2403_08131_b300 import gpbo
    w = W.config1()
    y = w.y.copy()
    y[5] = np.inf
    with pytest.raises(gpbo.GpboError) as e:
        ctx.search_step(w.X, y, w.lengthscale, 1.0, w.noise_var, M=16, seed=1)
    assert e.value.code == gpbo.GPBO_ENAN
    with pytest.raises(gpbo.GpboError) as e:
        ctx.search_step(w.X, w.y, w.lengthscale, 1.0, w.noise_var, M=0, seed=1)
    assert e.value.code == gpbo.GPBO_EINVAL


def test_step_reuses_model_across_calls_and_shapes(ctx):
    """The context keeps search_step's model for the next call of the same shape: repeated
    calls give identical results, and calls of other shapes and precisions in between (which
    replace the kept model) change nothing."""
    w = W.config2()
    M = 8192
    args = (w.X, w.y, w.lengthscale, 1.0, w.noise_var)
    a = ctx.search_step(*args, M=M, seed=w.seed, prec="f16")
    b = ctx.search_step(*args, M=M, seed=w.seed, prec="f16")
    small = W.config1()
    ctx.search_step(small.X, small.y, small.lengthscale, 1.0, small.noise_var, M=1024, seed=3, prec="f64")
    ctx.search_step(w.X[:300], w.y[:300], w.lengthscale, 1.0, w.noise_var, M=M, seed=w.seed, prec="f16")
    ctx.search_step(*args, M=M, seed=w.seed, prec="f32")
    c = ctx.search_step(*args, M=M, seed=w.seed, prec="f16")
    for r in (b, c):
        assert r["argmax"] == a["argmax"] and r["ei_max"] == a["ei_max"]
        assert np.array_equal(r["x_next"], a["x_next"])
