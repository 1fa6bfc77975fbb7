"""GPU posterior mean / std / EI / argmax against the FP64 oracle, per scoring precision."""
import numpy as np
import pytest

from paper_2403_08131_b300 import workloads as W
from tests._util import BAR, check_argmax, scaled_err, to_dev

pytestmark = pytest.mark.gpu


def _score(ctx, model, Xc, prec, y_best, seed=None, M=None):
    import torch
    dt = torch.float64 if prec == "f64" else torch.float32
    M = Xc.shape[0] if Xc is not None else M
    mu, sg, ei = (torch.empty(M, dtype=dt, device="cuda") for _ in range(3))
    am, em = ctx.posterior_ei(model, to_dev(Xc) if Xc is not None else None, M=M, seed=seed or 0, y_best=y_best,
                              mu=mu, sigma=sg, ei=ei)
    return am, em, mu.cpu().numpy(), sg.cpu().numpy(), ei.cpu().numpy()


def _oracle(orc, w, ys, Xc, tau):
    _, Lo, ao = orc.gp_fit(w.X, ys, w.lengthscale, 1.0, w.noise_var)
    mu, sg = orc.posterior(w.X, w.lengthscale, 1.0, Lo, ao, Xc.astype(np.float64))
    return mu, sg, orc.ei_batch(mu, sg, tau)


def _check(prec, got, ref, Xc=None):
    am, em, mu, sg, ei = got
    rmu, rsg, rei = ref
    bar = BAR[prec]
    assert scaled_err(mu, rmu, 1.0) <= bar, scaled_err(mu, rmu, 1.0)
    assert scaled_err(sg, rsg, 1.0) <= bar, scaled_err(sg, rsg, 1.0)
    assert scaled_err(ei, rei, rei.max()) <= bar, scaled_err(ei, rei, rei.max())
    assert ei[am] == ei.max() and abs(em - ei[am]) <= 1e-6 * abs(ei[am])
    return check_argmax(am, rei, bar)


@pytest.mark.parametrize("n", [600, 1100])
def test_f64_parity_with_tensor_core_inverse(ctx, orc, n):
    """n_pad >= 512: the large levels of the FP64 L^-1 run on the tensor cores (slice
    products at FP64 accuracy); FP64 scoring keeps the FP64 bar."""
    w = W.config4(n=n, M=3000, prec="f64")
    ys = (w.y - w.y.mean()) / w.y.std()
    m = ctx.fit(to_dev(w.X), to_dev(ys), w.lengthscale, 1.0, w.noise_var, prec="f64")
    Xc = w.candidates(3000)
    got = _score(ctx, m, Xc, "f64", ys.min())
    _check("f64", got, _oracle(orc, w, ys, Xc, ys.min()))
    m.free()


def test_f64_rosenbrock_n64_full_parity(ctx, orc):
    w = W.config1()
    ys = (w.y - w.y.mean()) / w.y.std()
    Xc = w.candidates()
    m = ctx.fit(to_dev(w.X), to_dev(ys), w.lengthscale, 1.0, w.noise_var, prec="f64")
    tau = ys.min()
    got = _score(ctx, m, Xc, "f64", tau)
    assert _check("f64", got, _oracle(orc, w, ys, Xc, tau)) == "exact"


@pytest.mark.parametrize("prec", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("n,M", [(512, 8192), (300, 1000), (64, 1), (1, 33)])
def test_fiveblock_parity(ctx, orc, prec, n, M):
    w = W.make_gp_workload("t", 2405, n, W.five_block_objective(2405), M, prec)
    ys = (w.y - w.y.mean()) / (w.y.std() or 1.0)
    Xc = w.candidates()
    m = ctx.fit(to_dev(w.X), to_dev(ys), w.lengthscale, 1.0, w.noise_var, prec=prec)
    tau = ys.min()
    got = _score(ctx, m, Xc, prec, tau)
    _check(prec, got, _oracle(orc, w, ys, Xc, tau))


def test_seeded_candidates_equal_explicit(ctx):
    import torch
    w = W.config2()
    ys = (w.y - w.y.mean()) / w.y.std()
    m = ctx.fit(to_dev(w.X), to_dev(ys), w.lengthscale, 1.0, w.noise_var, prec="f32")
    a = _score(ctx, m, None, "f32", ys.min(), seed=w.seed, M=5000)
    b = _score(ctx, m, w.candidates(5000), "f32", ys.min())
    assert a[0] == b[0] and all(np.array_equal(x, y) for x, y in zip(a[2:], b[2:]))
    out = torch.empty((777, 20), dtype=torch.float32, device="cuda")
    ctx.gen_candidates(out, w.seed, first=123)
    assert np.array_equal(out.cpu().numpy(), w.candidates(777, first=123))


def test_host_pointer_outputs_equal_device(ctx):
    w = W.config1()
    ys = (w.y - w.y.mean()) / w.y.std()
    m = ctx.fit(w.X, ys, w.lengthscale, 1.0, w.noise_var, prec="f64")
    Xc = w.candidates(3000)
    mu, sg, ei = np.empty(3000), np.empty(3000), np.empty(3000)
    am, em = ctx.posterior_ei(m, Xc, y_best=ys.min(), mu=mu, sigma=sg, ei=ei)
    got = _score(ctx, m, Xc, "f64", ys.min())
    assert am == got[0] and np.array_equal(mu, got[2]) and np.array_equal(sg, got[3]) and np.array_equal(ei, got[4])


def test_chunked_pool_equals_single_pass(ctx):
    """A workspace bound that forces many chunks gives bit-identical results."""
    from paper_2403_08131_b300 import gpbo
    import torch
    w = W.make_gp_workload("t", 2405, 512, W.five_block_objective(2405), 20000, "bf16")
    ys = (w.y - w.y.mean()) / w.y.std()
    Xc = w.candidates()
    c2 = gpbo.Context(0, torch.cuda.current_stream())
    for prec in ("f32", "bf16"):
        m1 = ctx.fit(to_dev(w.X), to_dev(ys), w.lengthscale, 1.0, w.noise_var, prec=prec)
        m2 = c2.fit(to_dev(w.X), to_dev(ys), w.lengthscale, 1.0, w.noise_var, prec=prec)
        c2.set_workspace_limit(4 << 20)   # ~2 MiB of K* per chunk
        a = _score(ctx, m1, Xc, prec, ys.min())
        b = _score(c2, m2, Xc, prec, ys.min())
        assert a[0] == b[0] and all(np.array_equal(x, y) for x, y in zip(a[2:], b[2:]))
        c2.set_workspace_limit(2 << 30)
    c2.close()


@pytest.mark.parametrize("prec", ["f16", "bf16"])
def test_full_size_sampled_parity(ctx, orc, full_size, prec):
    w, ys, Lo, ao = full_size
    m = ctx.fit(to_dev(w.X), to_dev(ys), w.lengthscale, 1.0, w.noise_var, prec=prec)
    tau = ys.min()
    am, em, mu, sg, ei = _score(ctx, m, None, prec, tau, seed=w.seed, M=w.M)
    # the oracle on a sample: random indices, the GPU's top 64, the first and last candidate
    rng = np.random.default_rng(0)
    top = np.argsort(-ei)[:64]
    idx = np.unique(np.concatenate([rng.choice(w.M, 384, replace=False), top, [w.M - 1, 0]]))
    cnt = idx.astype(np.uint64)[:, None] * np.uint64(w.d) + np.arange(w.d, dtype=np.uint64)[None, :]
    Xs = W.uniform24(w.seed, W.STREAM_CAND, cnt)
    rmu, rsg = orc.posterior(w.X, w.lengthscale, 1.0, Lo, ao, Xs)
    rei = orc.ei_batch(rmu, rsg, tau)
    bar = BAR[prec]
    assert scaled_err(mu[idx], rmu, 1.0) <= 1e-4          # the mean comes from FP32 K*
    assert scaled_err(sg[idx], rsg, 1.0) <= bar
    assert scaled_err(ei[idx], rei, rei.max()) <= bar
    # argmax: the GPU's pick is within the bar of the best oracle EI among the GPU's top 64
    pos = {int(i): k for k, i in enumerate(idx)}
    best_ref = max(rei[pos[int(i)]] for i in top)
    assert rei[pos[am]] >= best_ref * (1 - bar)
    m.free()


@pytest.fixture(scope="module")
def full_pool(ctx, orc, full_size):
    """Every scoring path on the bench's whole pool (n = 4096, M = 2^20): each path's pick and
    its top 1024 by EI, and the oracle's EI on the union of those sets and 512 random pool
    indices.  The FP64 path's top 1024 is within the FP64 bar of the oracle's ranking, so the
    union holds the oracle's best candidates of the whole pool."""
    w, ys, Lo, ao = full_size
    tau = float(ys.min())
    picks, tops = {}, {}
    for prec in ("f16", "bf16", "f32", "f64"):
        m = ctx.fit(to_dev(w.X), to_dev(ys), w.lengthscale, 1.0, w.noise_var, prec=prec)
        am, em, _, _, ei = _score(ctx, m, None, prec, tau, seed=w.seed, M=w.M)
        m.free()
        picks[prec] = am
        tops[prec] = np.argsort(-ei, kind="stable")[:1024]
        assert tops[prec][0] == am or ei[tops[prec][0]] == ei[am]
    rng = np.random.default_rng(1)
    union = np.unique(np.concatenate(list(tops.values()) + [rng.choice(w.M, 512, replace=False)]))
    cnt = union.astype(np.uint64)[:, None] * np.uint64(w.d) + np.arange(w.d, dtype=np.uint64)[None, :]
    Xs = W.uniform24(w.seed, W.STREAM_CAND, cnt)
    rmu, rsg = orc.posterior(w.X, w.lengthscale, 1.0, Lo, ao, Xs)
    return picks, tops, union, orc.ei_batch(rmu, rsg, tau)


@pytest.mark.parametrize("prec", ["f16", "bf16", "f32", "f64"])
def test_full_pool_argmax_against_oracle(full_pool, prec):
    """The pick over all 2^20 candidates obeys the argmax rule against the oracle's best over
    the union (exact when the oracle's margin exceeds the path's bar), and no oracle-scored
    candidate that the path ranked outside its top 1024 beats the pick."""
    picks, tops, union, rei = full_pool
    pos = {int(i): k for k, i in enumerate(union)}
    bar = BAR[prec]
    am = picks[prec]
    rule = check_argmax(pos[am], rei, bar)
    outside = ~np.isin(union, tops[prec])
    assert rei[outside].max() <= rei[pos[am]] * (1 + bar), (prec, float(rei[outside].max()), float(rei[pos[am]]))
    order = np.argsort(-rei, kind="stable")
    print(f"{prec}: pick {am}, oracle best {int(union[order[0]])}, margin "
          f"{(rei[order[0]] - rei[order[1]]) / rei[order[0]]:.3g}, rule {rule}")
