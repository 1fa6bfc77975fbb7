"""GPU fit (kernel matrix, FP64 Cholesky, refined alpha) against the FP64 oracle."""
import numpy as np
import pytest

from paper_2403_08131_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _obs(n, d, seed):
    X = W.uniform_points(seed, W.STREAM_OBS, n, d)
    obj = W.Objective([d], [W.FN_ACKLEY], 0.0, seed)
    y = obj(X)
    return X, (y - y.mean()) / (y.std() or 1.0)


@pytest.mark.parametrize("n,d", [(1, 3), (3, 2), (64, 4), (100, 20), (257, 7), (513, 20)])
@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
def test_fit_factor_and_alpha_match_oracle(ctx, orc, n, d, prec):
    from tests._util import to_dev
    X, y = _obs(n, d, 1000 + n)
    ls = W.lengthscale_rule(d)
    m = ctx.fit(to_dev(X), to_dev(y), ls, 1.0, 1e-4, prec=prec)
    Lg, ag = m.read()
    _, Lo, ao = orc.gp_fit(X, y, ls, 1.0, 1e-4)
    assert np.abs(Lg - Lo).max() <= 1e-11 * np.abs(Lo).max()
    assert np.abs(ag - ao).max() <= 1e-9 * (np.abs(ao).max() + 1)
    assert np.all(np.triu(Lg, 1) == 0)
    m.free()


@pytest.mark.parametrize("n,d,prec", [(1536, 20, "f64"), (2000, 8, "f16"), (2113, 20, "f32")])
def test_fit_tensor_core_update_matches_oracle(ctx, orc, n, d, prec):
    """n_pad >= 1536: the trailing updates run on the tensor cores (exact 8-bit slice
    products); L and alpha keep the FP64 bars."""
    from tests._util import to_dev
    X, y = _obs(n, d, 1100 + n)
    ls = W.lengthscale_rule(d)
    m = ctx.fit(to_dev(X), to_dev(y), ls, 1.0, 1e-4, prec=prec)
    Lg, ag = m.read()
    _, Lo, ao = orc.gp_fit(X, y, ls, 1.0, 1e-4)
    assert np.abs(Lg - Lo).max() <= 1e-11 * np.abs(Lo).max()
    assert np.abs(ag - ao).max() <= 1e-9 * (np.abs(ao).max() + 1)
    assert np.all(np.triu(Lg, 1) == 0)
    m.free()


@pytest.mark.parametrize("prec", ["f16", "bf16", "f32", "f64"])
def test_fit_full_size_matches_oracle(ctx, full_size, prec):
    """The bench's fit (n = 4096, d = 20, 64 block columns, the lookahead chain and every
    tensor-core update level) in each scoring precision: L and alpha against the textbook
    FP64 Cholesky and solves at the same bars as the smaller fits."""
    from tests._util import to_dev
    w, ys, Lo, ao = full_size
    m = ctx.fit(to_dev(w.X), to_dev(ys), w.lengthscale, 1.0, w.noise_var, prec=prec)
    Lg, ag = m.read()
    m.free()
    assert np.abs(Lg - Lo).max() <= 1e-11 * np.abs(Lo).max(), np.abs(Lg - Lo).max()
    assert np.abs(ag - ao).max() <= 1e-9 * (np.abs(ao).max() + 1), np.abs(ag - ao).max()
    assert not np.triu(Lg, 1).any()


def test_fit_host_pointers_equal_device(ctx):
    from tests._util import to_dev
    X, y = _obs(200, 5, 7)
    ls = W.lengthscale_rule(5)
    a = ctx.fit(X, y, ls, 1.0, 1e-6).read()
    b = ctx.fit(to_dev(X), to_dev(y), ls, 1.0, 1e-6).read()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_fit_not_spd_and_jitter(ctx, orc):
    from paper_2403_08131_b300 import gpbo
    X = np.array([[0.1, 0.2], [0.1, 0.2], [0.7, 0.4]])
    y = np.array([1.0, 1.0, -1.0])
    with pytest.raises(gpbo.GpboError) as e:
        ctx.fit(X, y, [0.3, 0.3], 1.0, 0.0)
    assert e.value.code == gpbo.GPBO_ENOTSPD
    with pytest.raises(orc.OracleError) as e2:
        orc.gp_fit(X, y, 0.3, 1.0, 0.0)
    assert e2.value.code == 2
    m = ctx.fit(X, y, [0.3, 0.3], 1.0, 0.0, jitter=True)
    assert m.info()["noise_var"] > 0


def test_fit_rejects_bad_arguments(ctx):
    from paper_2403_08131_b300 import gpbo
    X, y = _obs(10, 3, 1)
    for ls in ([0.3, -1.0, 0.3], [0.3, 0.3]):
        with pytest.raises(gpbo.GpboError) as e:
            ctx.fit(X, y, ls, 1.0, 1e-6)
        assert e.value.code == gpbo.GPBO_EINVAL
    Xn = X.copy()
    Xn[3, 1] = np.nan
    with pytest.raises(gpbo.GpboError) as e:
        ctx.fit(Xn, y, [0.3] * 3, 1.0, 1e-6)
    assert e.value.code == gpbo.GPBO_ENAN


def test_trace_phases_nest(ctx):
    """The Cholesky-update intervals nest inside the factorisation, which with the inverse
    splits the fit interval; all are recorded."""
    import torch
    w = W.config2()
    ys = (w.y - w.y.mean()) / w.y.std()
    ctx.trace(True)
    m = ctx.fit(w.X, ys, w.lengthscale, 1.0, w.noise_var, prec="f16")
    ctx.posterior_ei(m, None, M=4096, seed=1, y_best=float(ys.min()))
    tr = ctx.trace_read()
    ctx.trace(False)
    assert tr["fit"]["intervals"] == 1 and tr["fit"]["ms"] > 0
    assert tr["chol_update"]["intervals"] == 512 // 64 - 2   # steps with tiles beyond the lookahead column
    assert 0 < tr["chol_update"]["ms"] < tr["fit"]["ms"]
    assert tr["variance"]["intervals"] >= 1 and tr["xkern"]["intervals"] >= 1
    assert tr["chol_update"]["flops"] == sum(T * (T - 1) // 2 for T in range(2, 8)) * 2 * 64 ** 3
    # the factorisation and the inverse split the fit, in that order, inside its interval
    assert tr["factor"]["intervals"] == 1 and tr["inverse"]["intervals"] == 1
    assert tr["chol_update"]["ms"] < tr["factor"]["ms"]
    assert tr["factor"]["ms"] + tr["inverse"]["ms"] <= tr["fit"]["ms"] * 1.001


@pytest.mark.parametrize("n", [100, 1600])
def test_fit_nan_in_device_inputs_fails_the_same_way(ctx, n):
    """A NaN coordinate in device-resident X makes K NaN and the factorisation fail, with the
    same error whether the distances are FP64 (n = 100) or exact integers (n = 1600)."""
    from paper_2403_08131_b300 import gpbo
    from tests._util import to_dev
    X, y = _obs(n, 6, 4000 + n)
    X[n // 2, 3] = np.nan
    with pytest.raises(gpbo.GpboError) as e:
        ctx.fit(to_dev(X), to_dev(y), W.lengthscale_rule(6), 1.0, 1e-4, prec="f32")
    assert e.value.code == gpbo.GPBO_ENOTSPD
