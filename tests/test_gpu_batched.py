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
