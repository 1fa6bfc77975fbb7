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
