"""Batched step (many independent sub-searches in one graph launch) against the
single-problem path, bit for bit, and against the oracle on two problems."""
import numpy as np
import pytest

from paper_2403_08131_b300 import workloads as W
from tests._util import BAR, check_argmax

pytestmark = pytest.mark.gpu


def _problems(G=12, M=2048, seed_shift=0):
    subs = W.batched_config3(G=G, M=M)
    return subs, [dict(X=w.X, y=w.y, lengthscale=w.lengthscale, signal_var=1.0, noise_var=w.noise_var, M=M,
                       seed=w.seed + seed_shift) for w in subs]


@pytest.mark.parametrize("seed_shift", [0, 7])
def test_batched_equals_single_calls(ctx, seed_shift):
    subs, probs = _problems(seed_shift=seed_shift)
    out = ctx.search_step_batched(probs)
    for g, pb in enumerate(probs):
        one = ctx.search_step(pb["X"], pb["y"], pb["lengthscale"], 1.0, pb["noise_var"], M=pb["M"], seed=pb["seed"],
                              prec="f32")
        assert out["argmax"][g] == one["argmax"], g
        assert out["ei_max"][g] == one["ei_max"], g
        assert np.array_equal(out["x_next"][g], one["x_next"]), g


def test_batched_against_oracle(ctx, orc):
    subs, probs = _problems()
    out = ctx.search_step_batched(probs)
    for g in (0, 5):
        w, pb = subs[g], probs[g]
        ref = orc.search_step(w.X, w.y, w.lengthscale, 1.0, w.noise_var, M=pb["M"], seed=pb["seed"], want_arrays=True)
        check_argmax(int(out["argmax"][g]), ref["ei"], BAR["f32"])
        assert abs(out["ei_max"][g] - ref["ei_max"]) <= 1e-4 * max(ref["ei_max"], 1e-12) + 1e-6


def test_batched_shapes_are_uneven(ctx):
    subs, probs = _problems()
    ns = {w.n for w in subs}
    ds = {w.d for w in subs}
    assert len(ns) > 5 and len(ds) > 3
    assert min(w.d for w in subs) >= 2 and max(w.d for w in subs) <= 12
    assert min(w.n for w in subs) >= 32 and max(w.n for w in subs) <= 1024


def test_autotuned_tile_is_the_fastest_measured_and_tiles_agree(ctx):
    """The autotuner times the 64/128/256-candidate variance tiles on the plan and keeps the
    fastest; every forced tile gives the same results bit for bit (each candidate's sums run
    in the same order)."""
    subs, probs = _problems(seed_shift=3)
    ctx.batched_tile(0)
    auto = ctx.search_step_batched(probs)
    tile, ms = ctx.batched_tuning()
    assert set(ms) == {64, 128, 256} and all(v > 0 for v in ms.values())
    assert tile == min(ms, key=ms.get)
    print(f"autotuner: {ms} -> {tile}")
    for t in (64, 128, 256):
        ctx.batched_tile(t)
        out = ctx.search_step_batched(probs)
        assert ctx.batched_tuning()[0] == t
        assert np.array_equal(out["argmax"], auto["argmax"]) and np.array_equal(out["ei_max"], auto["ei_max"])
    ctx.batched_tile(0)
    with pytest.raises(Exception):
        ctx.batched_tile(48)


def test_full_config_sampled_against_oracle(ctx, orc):
    """The bench's batched workload at full size (64 GPs, M = 16384 each, autotuned tile):
    for four problems (the largest n, the largest d, two others) the GPU's pick is checked
    against the FP64 oracle -- its EI matches the oracle's EI at that candidate within the
    FP32 bar, it is at least as good as every one of 256 sampled candidates, and x_next is
    that candidate."""
    from tests._util import BAR
    subs, probs = _problems(G=64, M=16384)
    ctx.batched_tile(0)
    out = ctx.search_step_batched(probs)
    ns = [w.n for w in subs]
    ds = [w.d for w in subs]
    picks = sorted({int(np.argmax(ns)), int(np.argmax(ds)), 0, 37})
    rng = np.random.default_rng(5)
    for g in picks:
        w, pb = subs[g], probs[g]
        ys, _, _ = orc.standardize(w.y)
        _, Lo, ao = orc.gp_fit(w.X, ys, w.lengthscale, 1.0, w.noise_var)
        am = int(out["argmax"][g])
        idx = np.unique(np.concatenate([rng.choice(pb["M"], 256, replace=False), [am]]))
        Xc = np.concatenate([W.uniform_points(pb["seed"], W.STREAM_CAND, 1, w.d, first=int(i)) for i in idx])
        mu, sg = orc.posterior(w.X, w.lengthscale, 1.0, Lo, ao, Xc)
        ei = orc.ei_batch(mu, sg, float(ys.min()))
        e_am = ei[int(np.nonzero(idx == am)[0][0])]
        assert abs(out["ei_max"][g] - e_am) <= BAR["f32"] * (abs(e_am) + ei.max()), (g, out["ei_max"][g], e_am)
        assert e_am >= ei.max() * (1 - BAR["f32"]), (g, e_am, ei.max())
        assert np.allclose(out["x_next"][g], Xc[int(np.nonzero(idx == am)[0][0])], rtol=0, atol=1e-7)


@pytest.mark.parametrize("shapes", [[(1, 1)], [(1, 3), (2, 1), (65, 12), (700, 5)]])
def test_batched_edge_shapes_equal_single_calls(ctx, shapes):
    """Degenerate and uneven shapes (n = 1, n = 2, d = 1, a single problem, a block tail):
    the batched step still equals the single-problem calls bit for bit."""
    probs = []
    for g, (n, d) in enumerate(shapes):
        X = W.uniform_points(9000 + g, W.STREAM_OBS, n, d)
        y = W.Objective([d], [W.FN_ACKLEY], 0.0, 9000 + g)(X)
        probs.append(dict(X=X, y=y, lengthscale=W.lengthscale_rule(d), signal_var=1.0, noise_var=1e-4,
                          M=777 + 13 * g, seed=500 + g))
    out = ctx.search_step_batched(probs)
    for g, pb in enumerate(probs):
        one = ctx.search_step(pb["X"], pb["y"], pb["lengthscale"], 1.0, pb["noise_var"], M=pb["M"], seed=pb["seed"],
                              prec="f32")
        assert out["argmax"][g] == one["argmax"] and out["ei_max"][g] == one["ei_max"], (g, shapes[g])
        assert np.array_equal(out["x_next"][g], one["x_next"])


def test_batched_large_problem_within_bars_small_one_bit_for_bit(ctx):
    """Beside a small problem, one that pads to at least 1536 rows: search_step factors it with
    the tensor-core Cholesky updates and L^-1 levels, the batched step on the CUDA cores, so
    the large problem agrees within the FP32 bars (its pick's EI, rescored by the
    single-problem path, within the bar of that path's maximum) while the small one stays
    bit for bit."""
    from paper_2403_08131_b300 import gpbo
    from tests._util import to_dev
    probs = []
    for g, (n, d) in enumerate([(300, 6), (1600, 8)]):
        X = W.uniform_points(7100 + g, W.STREAM_OBS, n, d)
        y = W.Objective([d], [W.FN_ACKLEY], 0.0, 7100 + g)(X)
        probs.append(dict(X=X, y=y, lengthscale=W.lengthscale_rule(d), signal_var=1.0, noise_var=1e-4, M=4096,
                          seed=800 + g))
    out = ctx.search_step_batched(probs)
    small, large = probs
    one = ctx.search_step(small["X"], small["y"], small["lengthscale"], 1.0, 1e-4, M=small["M"], seed=small["seed"],
                          prec="f32")
    assert out["argmax"][0] == one["argmax"] and out["ei_max"][0] == one["ei_max"]
    one = ctx.search_step(large["X"], large["y"], large["lengthscale"], 1.0, 1e-4, M=large["M"], seed=large["seed"],
                          prec="f32")
    ys = (large["y"] - large["y"].mean()) / (large["y"].std() or 1.0)
    m = ctx.fit(to_dev(large["X"]), to_dev(ys), large["lengthscale"], 1.0, 1e-4, prec="f32")
    import torch
    ei = torch.empty(large["M"], dtype=torch.float32, device="cuda")
    ctx.posterior_ei(m, None, M=large["M"], seed=large["seed"], y_best=float(ys.min()), ei=ei)
    ei = ei.cpu().numpy().astype(np.float64)
    check_argmax(int(out["argmax"][1]), ei, BAR["f32"])
    assert abs(out["ei_max"][1] - one["ei_max"]) <= BAR["f32"] * one["ei_max"]
    m.free()


def test_batched_device_inputs_equal_host_inputs(ctx):
    """Device inputs (read by the graph's first kernel) and host inputs (copied by the host
    before the graph) give the same step bit for bit, on one plan, in either order."""
    import torch

    def dev(ps):
        return [dict(pb, X=torch.from_numpy(pb["X"]).cuda(), y=torch.from_numpy(pb["y"]).cuda()) for pb in ps]

    def same(a, b):
        return (np.array_equal(a["argmax"], b["argmax"]) and np.array_equal(a["ei_max"], b["ei_max"])
                and all(np.array_equal(x, z) for x, z in zip(a["x_next"], b["x_next"])))

    _, probs_a = _problems(G=9, M=1536)
    probs_b = [dict(pb, y=pb["y"][::-1].copy()) for pb in probs_a]   # same shapes, other values
    host_a = ctx.search_step_batched(probs_a)
    assert same(host_a, ctx.search_step_batched(dev(probs_a)))
    host_b = ctx.search_step_batched(probs_b)
    assert not same(host_a, host_b)
    assert same(host_b, ctx.search_step_batched(dev(probs_b)))
    assert same(host_a, ctx.search_step_batched(probs_a))


def test_batched_plan_members(ctx):
    """The tuning report covers the plan of the largest problems: those that pad to more than
    512 rows (the small ones run as a second, concurrent plan), or all of them if none do."""
    subs, probs = _problems()
    ctx.search_step_batched(probs)
    tile, ms, big = ctx.batched_tuning(members=True)
    npad = np.array([(w.n + 63) // 64 * 64 for w in subs])
    expect = npad > 512 if (npad > 512).any() else np.ones(len(subs), dtype=bool)
    assert np.array_equal(big, expect) and tile in ms
    small = [pb for pb, w in zip(probs, subs) if (w.n + 63) // 64 * 64 <= 512][:3]
    ctx.search_step_batched(small)
    assert ctx.batched_tuning(members=True)[2].all()
