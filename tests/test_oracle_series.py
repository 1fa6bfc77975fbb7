"""Pins of the oracle's routine sensitivity on the paper's schedule (§IV-B, §IV-C) and of the
decisions it reaches on the paper's synthetic Cases 1-5."""
import numpy as np
import pytest

from paper_2403_08131_b300 import workloads as W


def test_series_points_grow_by_ten_percent_and_clamp(orc):
    u0 = np.array([0.7, 0.5, 0.2])   # x = 20, 0, -30 in [-50, 50]
    p = orc.series_points(u0, 0, 12, 0.1, -50.0, 50.0)
    x = -50 + 100 * p[:, 0]
    expect = np.minimum(20.0 * 1.1 ** np.arange(1, 13), 50.0)
    assert np.allclose(x, expect, rtol=1e-13, atol=1e-12)
    assert np.all(p[:, 1:] == u0[1:])                       # the others stay at the baseline
    assert np.all(orc.series_points(u0, 1, 5, 0.1, -50.0, 50.0)[:, 1] == 0.5)   # 0 stays 0
    x2 = -50 + 100 * orc.series_points(u0, 2, 30, 0.1, -50.0, 50.0)[:, 2]
    assert x2[0] == pytest.approx(-33.0, rel=1e-13) and x2.min() == -50.0    # grows toward -50


def test_series_score_closed_form(orc):
    """Two routines, f_0 = 2 + x_0 (own x_0), f_1 = 3 + 0.5 x_0 + x_1 (own x_1), on [0, 1]: the
    scores are the mean relative changes along each parameter's series, computed here by hand."""
    def fn(u):
        return np.array([2.0 + u[0], 3.0 + 0.5 * u[0] + u[1]])

    V, g = 8, 0.1
    S, grp, ng, fx, own = orc.screen_routine_series(fn, 2, 2, V, g, 11, 0.0, 1.0, [0, 1], 0.01, 10)
    u0 = orc.uniform_points(11, 3, 1, 2)[0]
    f0 = fn(u0)
    for i in range(2):
        x = np.minimum(u0[i] * (1 + g) ** np.arange(1, V + 1), 1.0)
        dx = x - u0[i]
        coef = np.array([[1.0, 0.0], [0.5, 1.0]])[:, i]
        assert np.allclose(S[:, i], np.abs(coef * dx[:, None] / f0).mean(0).ravel(), rtol=1e-12, atol=1e-15)
    assert S[0, 1] == 0.0
    # x_0 moves routine 1 by more than the cut-off: the two routines merge
    assert S[1, 0] > 0.01 and ng == 1 and np.all(grp == 0)


def test_series_separable_routines_stay_apart(orc):
    def fn(u):
        return np.array([1.0 + u[0] ** 2 + u[1], 5.0 + np.cos(3 * u[2]) + u[3] ** 3])

    S, grp, ng, fx, own = orc.screen_routine_series(fn, 4, 2, 20, 0.1, 3, 0.0, 1.0, [0, 0, 1, 1], 0.0, 10)
    assert np.all(S[0, 2:] == 0.0) and np.all(S[1, :2] == 0.0)
    assert ng == 2 and list(grp) == [0, 0, 2, 2]


def test_series_shared_parameter_goes_to_its_strongest_routine(orc):
    def fn(u):
        return np.array([1.0 + u[0] + 0.1 * u[2], 1.0 + u[1] + 2.0 * u[2]])

    S, grp, ng, fx, own = orc.screen_routine_series(fn, 3, 2, 10, 0.1, 5, 0.0, 1.0, [0, 1, -1], 10.0, 10)
    assert list(own) == [0, 1, 1] and S[1, 2] > S[0, 2]


def _group_values(case):
    f = W.PaperSynthetic(case)
    return lambda u: f.group_values(u)


@pytest.mark.parametrize("case,merged", [(1, False), (2, False), (3, True), (4, True), (5, True)])
def test_series_reaches_the_papers_decisions(orc, case, merged):
    """§IV-D: with a 25% cut-off, Groups 3 and 4 are merged for Cases 3, 4 and 5 and searched
    apart for Cases 1 and 2; Groups 1 and 2 are always searched alone.  Routine outputs are
    the raw group values (the routines' 'runtimes', before the logarithm); baseline from seed 1;
    100 variations of 10%; x in [-50, 50]."""
    S, grp, ng, fx, own = orc.screen_routine_series(_group_values(case), 20, 4, 100, 0.1, 1, -50.0, 50.0,
                                                    np.repeat(np.arange(4), 5), 0.25, 10)
    assert grp[0] == 0 and np.all(grp[:5] == 0) and np.all(grp[5:10] == 5)
    if merged:
        assert ng == 3 and np.all(grp[10:20] == 10) and fx.sum() == 0   # ten dimensions: no cap
    else:
        assert ng == 4 and np.all(grp[10:15] == 10) and np.all(grp[15:20] == 15)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_series_group4_influence_rises_with_the_case(orc, seed):
    """Table `tab:sensitSynth`: Group 4's influence on Group 3 is very low / low in Cases 1-2,
    medium in Case 3 and high in Cases 4-5 (the exact percentages depend on the paper's
    unstated baseline)."""
    ext = []
    for case in range(1, 6):
        S, *_ = orc.screen_routine_series(_group_values(case), 20, 4, 100, 0.1, seed, -50.0, 50.0,
                                          np.repeat(np.arange(4), 5), 0.25, 10)
        ext.append(S[2, 15:20].max())
    assert max(ext[0], ext[1]) < ext[2] < min(ext[3], ext[4])
