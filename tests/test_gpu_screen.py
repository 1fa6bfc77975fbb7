"""GPU interdependence screen against the oracle: scores to rounding, partitions bit-exact."""
import numpy as np
import pytest

from paper_2403_08131_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _planted(noise):
    sw = W.screen_config2(noise_sd=noise)
    return sw, sw.objective


@pytest.mark.parametrize("noise", [0.0, 0.01])
def test_pairwise_matches_oracle(ctx, orc, noise):
    sw, o = _planted(noise)
    g = ctx.screen(o.block_dim, o.block_fn, noise, sw.seed, sw.n_base, sw.h, sw.cutoff, sw.max_dims)
    score, sens = orc.screen_pairwise(o.block_dim, o.block_fn, noise, sw.seed, sw.n_base, sw.h)
    lab, ng, fixed = orc.partition_pairwise(score, sw.cutoff, sw.max_dims, sens)
    assert np.allclose(g["score"], score, rtol=1e-9, atol=1e-12)
    assert np.allclose(g["influence"], sens, rtol=1e-9, atol=1e-12)
    assert np.array_equal(g["group_of"], lab) and g["n_groups"] == ng and np.array_equal(g["fixed"], fixed)
    want = np.arange(20)
    for b in (0, 2, 4):
        want[4 * b:4 * b + 4] = 4 * b
    assert np.array_equal(g["group_of"], want)


@pytest.mark.parametrize("noise", [0.0, 0.01])
def test_routine_matches_oracle_and_recovers_blocks(ctx, orc, noise):
    from paper_2403_08131_b300 import gpbo
    sw, o = _planted(noise)
    g = ctx.screen(o.block_dim, o.block_fn, noise, sw.seed, sw.n_base, sw.h, sw.cutoff_routine, sw.max_dims,
                   mode=gpbo.SCREEN_ROUTINE)
    S = orc.screen_routine(o.block_dim, o.block_fn, noise, sw.seed, sw.n_base, sw.h)
    owner = orc.block_owner(o.block_dim)
    lab, ng, fixed = orc.partition_routine(S, owner, sw.cutoff_routine, sw.max_dims)
    assert np.allclose(g["score"], S, rtol=1e-9, atol=1e-12)
    assert np.array_equal(g["group_of"], lab) and g["n_groups"] == ng == 5
    assert np.array_equal(g["group_of"], 4 * owner)


def test_cap_on_a_merged_search(ctx, orc):
    """A chained 12-D Rosenbrock block is one group at a 5% cut-off; the cap keeps its 10
    most influential parameters."""
    g = ctx.screen([12, 3], [W.FN_ROSENBROCK, W.FN_RASTRIGIN], 0.0, 11, 32, 0.1, 0.05, 10)
    score, sens = orc.screen_pairwise([12, 3], [W.FN_ROSENBROCK, W.FN_RASTRIGIN], 0.0, 11, 32, 0.1)
    lab, ng, fixed = orc.partition_pairwise(score, 0.05, 10, sens)
    assert list(lab[:12]) == [0] * 12
    assert np.array_equal(g["group_of"], lab) and np.array_equal(g["fixed"], fixed)
    assert fixed[:12].sum() == 2 and fixed[12:].sum() == 0


def test_host_black_box_equals_builtin(ctx):
    from paper_2403_08131_b300 import gpbo
    sw, o = _planted(0.0)

    def black_box(x):
        r = o.routines(x[None, :])[0]
        return r.sum(), r

    a = ctx.screen(o.block_dim, o.block_fn, 0.0, sw.seed, sw.n_base, sw.h, sw.cutoff, sw.max_dims)
    b = ctx.screen(host_fn=black_box, d=20, seed=sw.seed, n_base=sw.n_base, h=sw.h, cutoff=sw.cutoff,
                   max_dims=sw.max_dims)
    assert np.array_equal(a["group_of"], b["group_of"])
    assert np.allclose(a["score"], b["score"], rtol=1e-9, atol=1e-12)
    owner = np.repeat(np.arange(5), 4)
    c = ctx.screen(host_fn=black_box, d=20, seed=sw.seed, n_base=sw.n_base, h=sw.h, cutoff=sw.cutoff_routine,
                   max_dims=sw.max_dims, mode=gpbo.SCREEN_ROUTINE, n_routines=5, param_owner=owner)
    assert np.array_equal(c["group_of"], 4 * owner)


# ---------------------------------------------------------------- the paper's series schedule
def _series_orc(orc, fn, d, R, V, seed, lo, hi, owner, cutoff):
    return orc.screen_routine_series(fn, d, R, V, 0.1, seed, lo, hi, owner, cutoff, 10)


@pytest.mark.parametrize("case", [1, 3, 5])
def test_series_screen_host_black_box_matches_oracle(ctx, orc, case):
    from paper_2403_08131_b300 import gpbo
    f = W.PaperSynthetic(case)
    owner = np.repeat(np.arange(4), 5)
    r = ctx.screen(host_fn=lambda u: (0.0, f.group_values(u)), d=20, n_routines=4, param_owner=owner, n_base=100,
                   cutoff=0.25, seed=1, mode=gpbo.SCREEN_ROUTINE_SERIES, growth=0.1, lo=-50.0, hi=50.0)
    S, grp, ng, fx, own = _series_orc(orc, f.group_values, 20, 4, 100, 1, -50.0, 50.0, owner, 0.25)
    assert np.allclose(r["score"], S, rtol=1e-13, atol=0)
    assert np.array_equal(r["group_of"], grp) and r["n_groups"] == ng and np.array_equal(r["fixed"], fx)
    assert r["n_groups"] == (4 if case == 1 else 3)


def test_series_screen_builtin_blocks_match_oracle(ctx, orc):
    from paper_2403_08131_b300 import gpbo
    bd, bf = [4, 3, 5], [W.FN_ACKLEY, W.FN_RASTRIGIN, W.FN_ROSENBROCK]
    d = sum(bd)
    r = ctx.screen(block_dim=bd, block_fn=bf, n_base=40, cutoff=0.05, seed=9, mode=gpbo.SCREEN_ROUTINE_SERIES,
                   growth=0.1)
    lo = np.concatenate([np.full(m, -w) for m, w in zip(bd, (32.768, 5.12, 2.0))])
    owner = orc.block_owner(bd)

    def fn(u):
        o, out = 0, []
        for m, code in zip(bd, bf):
            out.append(orc.block_value(code, u[o:o + m]))
            o += m
        return np.array(out)

    S, grp, ng, fx, own = _series_orc(orc, fn, d, 3, 40, 9, lo, -lo, owner, 0.05)
    assert np.allclose(r["score"], S, rtol=1e-11, atol=1e-14)
    assert np.all(r["score"][owner, np.arange(d)] > 0) and np.array_equal(r["group_of"], grp)
    # additive blocks: no cross-block influence at all
    for g in range(3):
        assert np.all(r["score"][g][owner != g] == 0.0)


def test_series_screen_shared_parameter(ctx, orc):
    from paper_2403_08131_b300 import gpbo

    def fn(u):
        return np.array([1.0 + u[0] + 0.1 * u[2], 1.0 + u[1] + 2.0 * u[2]])

    owner = np.array([0, 1, -1])
    r = ctx.screen(host_fn=lambda u: (0.0, fn(u)), d=3, n_routines=2, param_owner=owner, n_base=10, cutoff=10.0,
                   seed=5, mode=gpbo.SCREEN_ROUTINE_SERIES, growth=0.1)
    S, grp, ng, fx, own = _series_orc(orc, fn, 3, 2, 10, 5, 0.0, 1.0, owner, 10.0)
    assert np.array_equal(r["group_of"], grp) and list(grp) == [0, 1, 1]
