"""Learned pre-screen on the GPU: forward and gradients against the FP64 oracle, training,
radix top-k, and what the screen gains over an unscreened subset of the same size."""
import numpy as np
import pytest

from paper_2403_08131_b300 import workloads as W
from tests._util import to_dev

pytestmark = pytest.mark.gpu


def _net(ctx, E, d, H, seed=5):
    from paper_2403_08131_b300 import gpbo
    return gpbo.Surrogate(ctx, E=E, d=d, H=H, seed=seed)


def test_init_layout(ctx, orc):
    d, H = 6, 32
    net = _net(ctx, 3, d, H)
    th = net.params()
    for e in range(3):
        W1, b1, W2, b2, W3, b3 = orc.mlp_split(th[e].astype(np.float64), d, H)
        assert not b1.any() and not b2.any() and not b3.any()
        assert np.abs(W1).max() <= np.sqrt(6 / (d + H)) and np.abs(W2).max() <= np.sqrt(6 / (2 * H))
        assert W1.std() > 0.5 * np.sqrt(6 / (d + H)) / np.sqrt(3)
    assert not np.array_equal(th[0], th[1])


def test_forward_matches_oracle(ctx, orc):
    import torch
    E, d, H, B = 3, 5, 48, 70
    net = _net(ctx, E, d, H)
    th = net.params()
    X = np.random.default_rng(0).random((B, d)).astype(np.float32)
    out = torch.empty((E, B, 2), dtype=torch.float32, device="cuda")
    net.forward(to_dev(X), out)
    got = out.cpu().numpy()
    for e in range(E):
        ref = orc.mlp_forward(th[e].astype(np.float64), X.astype(np.float64), d, H)
        assert np.allclose(got[e], ref, rtol=1e-4, atol=1e-5 * np.abs(ref).max())


def test_gradients_match_oracle(ctx, orc):
    E, d, H, B = 2, 4, 40, 37
    net = _net(ctx, E, d, H, seed=9)
    th = net.params()
    rng = np.random.default_rng(1)
    X = rng.random((B, d)).astype(np.float32)
    T = rng.normal(size=(B, 2)).astype(np.float32)
    loss, g = net.gradients(to_dev(X), to_dev(T))
    for e in range(E):
        rl, rg = orc.mlp_grad(th[e].astype(np.float64), X.astype(np.float64), T.astype(np.float64), d, H)
        assert loss[e] == pytest.approx(rl, rel=1e-5)
        assert np.max(np.abs(g[e] - rg)) <= 1e-4 * np.abs(rg).max()


@pytest.fixture(scope="module")
def trained(ctx):
    """Exact GP (n=512, d=20, FP16 tiles) and an 8-network ensemble trained on 65536 of its
    posterior samples."""
    import torch
    w = W.config2()
    ys = (w.y - w.y.mean()) / w.y.std()
    model = ctx.fit(to_dev(w.X), to_dev(ys), w.lengthscale, 1.0, w.noise_var, prec="f16")
    N = 65536
    Xt = torch.empty((N, 20), dtype=torch.float32, device="cuda")
    ctx.gen_candidates(Xt, seed=99)
    mu = torch.empty(N, dtype=torch.float32, device="cuda")
    sg = torch.empty(N, dtype=torch.float32, device="cuda")
    ctx.posterior_ei(model, Xt, y_best=float(ys.min()), mu=mu, sigma=sg)
    net = _net(ctx, 8, 20, 256)
    l0 = net.train(Xt, mu, sg, steps=1, batch=1024, lr=1e-3)
    l1 = net.train(Xt, mu, sg, steps=1500, batch=1024, lr=1e-3)
    return w, ys, model, net, l0, l1


def test_training_reduces_loss(trained):
    w, ys, model, net, l0, l1 = trained
    print(f"loss first step {l0:.4f}, after 1500 steps {l1:.4f}")
    assert l1 < 0.25 * l0


def test_topk_is_the_k_largest(ctx, trained):
    import torch
    w, ys, model, net, _, _ = trained
    M, k = 200_000, 4096
    ei = torch.empty(M, dtype=torch.float32, device="cuda")
    am, em, top = net.screen(model, M, 321, k, float(ys.min()), ei_pool=ei, want_top=True)
    v = ei.cpu().numpy()
    assert len(set(top.tolist())) == k
    thr = np.sort(v)[::-1][k - 1]
    assert np.all(v[top] >= thr)
    assert set(np.nonzero(v > thr)[0].tolist()) <= set(top.tolist())
    assert 0 <= am < M


def test_screen_gains_over_unscreened_subset(ctx, trained):
    """The exact EI of the screened pick against (a) the exact argmax of the whole pool and
    (b) the best of a random subset of the same size k."""
    import torch
    w, ys, model, net, _, _ = trained
    M, k, seed = 1 << 20, 4096, 4242
    tau = float(ys.min())
    am, em, top = net.screen(model, M, seed, k, tau, want_top=True)
    ei = torch.empty(M, dtype=torch.float32, device="cuda")
    gam, gem = ctx.posterior_ei(model, None, M=M, seed=seed, y_best=tau, ei=ei)
    e = ei.cpu().numpy()
    rand = np.random.default_rng(0).choice(M, k, replace=False)
    best_rand = e[rand].max()
    recall = gam in set(top.tolist())
    print(f"screened pick EI {em:.5g}, global max {gem:.5g} (ratio {em / gem:.4f}), "
          f"random-subset best {best_rand:.5g}, exact argmax in top-k: {recall}")
    assert em > best_rand
    # agreement with the exact argmax of the whole pool within the 16-bit bar (same scoring path)
    assert em >= gem * (1 - 2e-3)


# ------------------------------------------------------------------ tensor-core (BF16) forward
def _rand_biases(net, d, H, seed):
    th = net.params()
    rng = np.random.default_rng(seed)
    o_b1, o_b2, o_b3 = d * H, d * H + H + H * H, d * H + H + H * H + H + 2 * H
    for e in range(th.shape[0]):
        th[e, o_b1:o_b1 + H] = rng.normal(0, 0.2, H)
        th[e, o_b2:o_b2 + H] = rng.normal(0, 0.2, H)
        th[e, o_b3:o_b3 + 2] = rng.normal(0, 0.2, 2)
    net.params(th)
    return th


def _check_tc(orc, th, X, ei, mu, sg, nm, tau, d, H):
    """Tensor-core (mu_bar, sigma_bar, EI) against the FP64 oracle within the FP16 tolerance;
    returns the worst error / tolerance of each."""
    from tests._util import f16_ensemble_tol
    th = np.asarray(th, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    rm, rs, re = orc.mlp_ensemble(th, X, d, H, nm, tau)
    tm, ts, te = f16_ensemble_tol(orc, th, X, d, H, nm, tau)
    gm, gs, ge = (a.cpu().numpy().astype(np.float64) for a in (mu, sg, ei))
    r = (np.max(np.abs(gm - rm) / tm), np.max(np.abs(gs - rs) / ts), np.max(np.abs(ge - re) / te))
    assert max(r) <= 1.0, f"worst error / tolerance (mu_bar, sigma_bar, ei) = {r}"
    return r


@pytest.mark.parametrize("M", [1, 127, 129, 1000])
def test_tc_forward_matches_oracle_within_f16_tolerance(ctx, orc, M):
    """Random-init ensemble (E = 3, random biases) on M explicit rows: the tensor-core
    mu_bar, sigma_bar and EI against the FP64 oracle within the FP16 tolerance; the FP32
    path within 1e-4 of it."""
    import torch
    d, H = 20, 256
    net = _net(ctx, 3, d, H, seed=11)
    th = _rand_biases(net, d, H, 12)
    X = np.random.default_rng(M).random((M, d)).astype(np.float32)
    outs = {p: [torch.empty(M, dtype=torch.float32, device="cuda") for _ in range(3)] for p in ("f16", "f32")}
    for p, (ei, mu, sg) in outs.items():
        net.score(ei, X=to_dev(X), y_best=0.1, prec=p, mu=mu, sigma=sg)
    rm, rs, _ = orc.mlp_ensemble(th.astype(np.float64), X.astype(np.float64), d, H, (0, 1, 0, 1), 0.1)
    r = _check_tc(orc, th, X, *outs["f16"], (0.0, 1.0, 0.0, 1.0), 0.1, d, H)
    print(f"M={M}: worst error / tolerance (mu_bar, sigma_bar, ei) = {r[0]:.3f}, {r[1]:.3f}, {r[2]:.3f}")
    fm, fs = outs["f32"][1].cpu().numpy(), outs["f32"][2].cpu().numpy()
    assert np.max(np.abs(fm - rm) / (np.abs(rm) + 1)) <= 1e-4 and np.max(np.abs(fs - rs) / rs) <= 1e-4


@pytest.mark.parametrize("E,d,M", [(1, 7, 60013), (3, 31, 57000), (5, 20, 40129)])
def test_tc_forward_many_tiles_per_cta(ctx, orc, E, d, M):
    """Several tiles per CTA pair (M / 256 pair tiles over at most 74 pairs), so that the
    per-network TMEM regions, the barrier phases and the one-network-behind layer 2 cross tile
    boundaries: a single network, odd ensembles, a one-step (d = 7) and a full (d = 31) layer-1
    K width, ragged tails.  The tensor-core outputs against the FP64 oracle within the FP16
    tolerance."""
    import torch
    H = 256
    net = _net(ctx, E, d, H, seed=20 + E)
    th = _rand_biases(net, d, H, 30 + E)
    X = np.random.default_rng(M).random((M, d)).astype(np.float32)
    ei, mu, sg = (torch.empty(M, dtype=torch.float32, device="cuda") for _ in range(3))
    net.score(ei, X=to_dev(X), y_best=0.1, prec="f16", mu=mu, sigma=sg)
    r = _check_tc(orc, th, X, ei, mu, sg, (0.0, 1.0, 0.0, 1.0), 0.1, d, H)
    print(f"E={E} d={d} M={M}: worst error / tolerance (mu_bar, sigma_bar, ei) = {r[0]:.3f}, {r[1]:.3f}, {r[2]:.3f}")


def test_tc_trained_ensemble_seeded_equals_explicit(ctx, orc, trained):
    """Trained 8-member ensemble: seeded candidates equal the same rows passed explicitly
    (bit for bit), and both agree with the oracle within the FP16 tolerance."""
    import torch
    w, ys, model, net, _, _ = trained
    d, H, M, seed = 20, 256, 777, 31
    X = torch.empty((M, d), dtype=torch.float32, device="cuda")
    ctx.gen_candidates(X, seed=seed)
    a = [torch.empty(M, dtype=torch.float32, device="cuda") for _ in range(3)]
    b = [torch.empty(M, dtype=torch.float32, device="cuda") for _ in range(3)]
    tau = float(ys.min())
    net.score(a[0], X=X, y_best=tau, mu=a[1], sigma=a[2])
    net.score(b[0], M=M, seed=seed, y_best=tau, mu=b[1], sigma=b[2])
    for u, v in zip(a, b):
        assert torch.equal(u, v)
    nm = tuple(net.norm())
    r = _check_tc(orc, net.params(), X.cpu().numpy(), *a, nm, tau, d, H)
    print(f"trained: worst error / tolerance (mu_bar, sigma_bar, ei) = {r[0]:.3f}, {r[1]:.3f}, {r[2]:.3f}")


def test_tc_full_size_sampled(ctx, orc, trained):
    """2^22 seeded candidates in one launch: 64 sampled candidates against the oracle."""
    import torch
    w, ys, model, net, _, _ = trained
    d, H, M, seed = 20, 256, 1 << 22, 4243
    tau = float(ys.min())
    ei, mu, sg = (torch.empty(M, dtype=torch.float32, device="cuda") for _ in range(3))
    net.score(ei, M=M, seed=seed, y_best=tau, mu=mu, sigma=sg)
    idx = np.sort(np.random.default_rng(3).choice(M, 64, replace=False))
    idx[-1] = M - 1
    X = np.concatenate([W.uniform_points(seed, W.STREAM_CAND, 1, d, first=int(i)) for i in idx])
    sel = torch.from_numpy(idx).cuda()
    r = _check_tc(orc, net.params(), X, ei[sel], mu[sel], sg[sel], tuple(net.norm()), tau, d, H)
    print(f"2^22 sampled: worst error / tolerance = {r[0]:.3f}, {r[1]:.3f}, {r[2]:.3f}")
    assert torch.isfinite(ei).all() and (ei >= 0).all()


def test_tc_rejects_unsupported_shapes(ctx):
    import torch
    from paper_2403_08131_b300 import gpbo
    net = _net(ctx, 2, 20, 128)
    ei = torch.empty(10, dtype=torch.float32, device="cuda")
    with pytest.raises(gpbo.GpboError) as e:
        net.score(ei, M=10, seed=1, prec="f16")
    assert e.value.code == gpbo.GPBO_ENOTSUP
    net.score(ei, M=10, seed=1, prec="f32")
    net2 = _net(ctx, 2, 20, 256)
    with pytest.raises(gpbo.GpboError) as e:   # the tensor-core forward has FP16 operands only
        net2.score(ei, M=10, seed=1, prec="bf16")
    assert e.value.code == gpbo.GPBO_ENOTSUP
