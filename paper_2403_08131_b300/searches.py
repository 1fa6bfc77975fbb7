"""Search strategies over an objective made of routines (§IV-D, Table `BO-synth`).

A strategy is a list of searches; each search tunes the variables of its routines (a merged
search several routines' variables) and minimises the sum of those routines' outputs, with
every other variable at its default.  The searches run one after another here (the paper
runs them in parallel; they share nothing), each with 5 initial random configurations and
10 x (its number of variables) evaluations in all.  The strategy's result is the objective,
without noise, at the combination of the searches' best configurations.  Random search
evaluates the same total budget at uniform points.

Host composition only: every search is one bo_search call of the library.
"""
from __future__ import annotations

import time

import numpy as np

from . import workloads as W

# routine lists per search (routines 0..3 = Groups 1..4)
STRATEGIES = {
    "joint": [[0, 1, 2, 3]],            # G1+G2+G3+G4
    "g1_g2_g34": [[0], [1], [2, 3]],    # G1, G2, G3+G4 (the screen's choice for Cases 3-5)
    "independent": [[0], [1], [2], [3]],  # G1, G2, G3, G4
}


def search_vars(objective, routines):
    return np.concatenate([np.arange(*objective.GROUPS[r]) for r in routines])


def run_strategy(ctx, objective, searches, seed, M=16384, n_init=5, per_dim=10, prec="f32", refit=True,
                 u_default=0.75, noise_var=1e-4, mle_iters=20):
    """Runs the searches of one strategy; returns a dict with the combined best configuration
    (unit cube), its noise-free objective value, each search's best value and the time."""
    d = objective.d
    best_u = np.full(d, u_default)
    per = []
    t0 = time.perf_counter()
    for s, routines in enumerate(searches):
        vars_ = search_vars(objective, routines)
        k = len(vars_)
        counter = [0]
        base = np.full(d, u_default)  # defaults for the variables this search does not tune

        def f(u, vars_=vars_, routines=routines, base=base, s=s):
            x = base.copy()
            x[vars_] = u
            c = counter[0]
            counter[0] += 1
            return float(objective.routines(x[None, :], noise_counter0=(s + 1) * 1_000_000 + c)[0, routines].sum())

        x_init = W.uniform_points(seed * 100 + s, W.STREAM_BO_INIT, n_init, k)
        X, y, b = ctx.bo_search(f, x_init, per_dim * k, M, seed * 100_000 + s * 10_000, W.lengthscale_rule(k), 1.0,
                                noise_var, prec=prec, refit=refit, mle_iters=mle_iters)
        best_u[vars_] = X[b]
        per.append({"routines": routines, "k": int(k), "evaluations": int(per_dim * k), "best": float(y[b])})
    elapsed = time.perf_counter() - t0
    clean = W.PaperSynthetic(objective.case, 0.0) if isinstance(objective, W.PaperSynthetic) else objective
    return {"value": float(clean(best_u[None, :])[0]), "x_best": best_u, "searches": per, "seconds": elapsed}


def random_search(objective, budget, seed):
    """Best of `budget` uniform configurations (noise-free value at the best noisy pick)."""
    U = W.uniform_points(seed, W.STREAM_BO_INIT, budget, objective.d, first=1_000_000)
    f = objective(U, noise_counter0=9_000_000)
    b = int(np.argmin(f))
    clean = W.PaperSynthetic(objective.case, 0.0) if isinstance(objective, W.PaperSynthetic) else objective
    return {"value": float(clean(U[b:b + 1])[0]), "x_best": U[b]}
