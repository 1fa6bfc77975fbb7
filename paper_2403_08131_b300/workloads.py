"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and the bench.

This module holds no arithmetic of the GP-BO method itself.  It draws the
observation sets (X, y) that a tuning search would have collected, and states the
fixed hyperparameters each workload uses.  The objectives below are the black
boxes being tuned (§III-C of the paper uses additive blocks of classic test
functions for the same purpose); they are evaluated here only to fill ``y``.
The library and the oracle each evaluate their own copy of the objectives where
the method itself calls them (the interdependence screen).

Random numbers come from SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) used as
a counter-based generator: the value at (seed, stream, counter) is the
``counter``-th output of a SplitMix64 generator seeded with
``seed XOR (stream * 0x9E3779B97F4A7C15)``.  Uniforms keep the top 24 bits, so
every coordinate is exact in float32 and float64 on both sides.

Streams: 1 observations, 2 candidates, 3 screen base points, 4 noise,
5 network init, 6 batched-workload shapes, 7 surrogate training points.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
_MASK = (1 << 64) - 1

STREAM_OBS = 1
STREAM_CAND = 2
STREAM_BASE = 3
STREAM_NOISE = 4
STREAM_INIT = 5
STREAM_SHAPES = 6
STREAM_TRAIN = 7
STREAM_MLE_STARTS = 8
STREAM_BO_INIT = 9

# Objective block codes (same numbering as the C ABI's gpbo_fn).
FN_ACKLEY = 0
FN_RASTRIGIN = 1
FN_ROSENBROCK = 2

# Affine map of the unit box onto each function's customary domain.
DOMAIN = {
    FN_ACKLEY: (-32.768, 32.768),
    FN_RASTRIGIN: (-5.12, 5.12),
    FN_ROSENBROCK: (-2.0, 2.0),
}


def splitmix64(seed: int, stream: int, counter) -> np.ndarray:
    """Counter-th output (0-based) of SplitMix64 seeded with seed ^ stream*GAMMA."""
    s0 = np.uint64((int(seed) ^ ((int(stream) * GAMMA) & _MASK)) & _MASK)
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = s0 + (c + np.uint64(1)) * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform24(seed: int, stream: int, counter) -> np.ndarray:
    """Uniform in [0, 1) on the 2^-24 grid (exact in float32)."""
    bits = splitmix64(seed, stream, counter) >> np.uint64(40)
    return bits.astype(np.float64) * (1.0 / (1 << 24))


def normal(seed: int, stream: int, counter) -> np.ndarray:
    """Standard normal by Box-Muller from the draws at 2c and 2c+1."""
    c = np.asarray(counter, dtype=np.uint64)
    b1 = splitmix64(seed, stream, c * np.uint64(2)) >> np.uint64(11)
    b2 = splitmix64(seed, stream, c * np.uint64(2) + np.uint64(1)) >> np.uint64(11)
    u1 = (b1.astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = b2.astype(np.float64) * 2.0 ** -53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def uniform_points(seed: int, stream: int, count: int, d: int, first: int = 0) -> np.ndarray:
    """count x d points; point p, coordinate k uses counter (first + p) * d + k."""
    idx = (np.arange(count, dtype=np.uint64)[:, None] + np.uint64(first)) * np.uint64(d) \
        + np.arange(d, dtype=np.uint64)[None, :]
    return uniform24(seed, stream, idx)


# ---------------------------------------------------------------- black boxes
def _block_value(fn: int, x01: np.ndarray) -> np.ndarray:
    lo, hi = DOMAIN[fn]
    z = lo + (hi - lo) * x01
    m = z.shape[-1]
    if fn == FN_ACKLEY:
        a = np.sqrt(np.sum(z * z, axis=-1) / m)
        b = np.sum(np.cos(2.0 * math.pi * z), axis=-1) / m
        return -20.0 * np.exp(-0.2 * a) - np.exp(b) + 20.0 + math.e
    if fn == FN_RASTRIGIN:
        return 10.0 * m + np.sum(z * z - 10.0 * np.cos(2.0 * math.pi * z), axis=-1)
    if fn == FN_ROSENBROCK:
        z0, z1 = z[..., :-1], z[..., 1:]
        return np.sum(100.0 * (z1 - z0 * z0) ** 2 + (1.0 - z0) ** 2, axis=-1)
    raise ValueError(fn)


@dataclass
class Objective:
    """Additive sum of blocks; block b owns a contiguous run of block_dim[b] inputs."""
    block_dim: list
    block_fn: list
    noise_sd: float = 0.0
    seed: int = 0

    @property
    def d(self) -> int:
        return int(sum(self.block_dim))

    def routines(self, X: np.ndarray) -> np.ndarray:
        out, o = [], 0
        for m, fn in zip(self.block_dim, self.block_fn):
            out.append(_block_value(fn, X[..., o:o + m]))
            o += m
        return np.stack(out, axis=-1)

    def __call__(self, X: np.ndarray, noise_counter0: int = 0) -> np.ndarray:
        f = self.routines(X).sum(axis=-1)
        if self.noise_sd > 0:
            cnt = np.arange(f.shape[0], dtype=np.uint64) + np.uint64(noise_counter0)
            f = f + self.noise_sd * normal(self.seed, STREAM_NOISE, cnt)
        return f


class PaperSynthetic:
    """The 20-dimensional synthetic function of the paper's evaluation (§III, Fig. `equation`
    and Table `group3_defs`), a black box: four groups (routines) of five variables each,
    x = -50 + 100 u for u in the unit cube, and each group's value entering the total as
    log|G_g|.  With A_i = 10 cos(2 pi (x_i - 1)) + eps:
      G1 = sum_{i=0..3} (x_i - x_{i+1})^2 + sum_{i=0..4} A_i
      G2 = sum_{k=5..8} (x_k - x_{k+1})^4 + sum_{k=5..9} A_k
      G3 = Case 1: sum x_u + sum cos(2 pi x_v) + eps     Case 2: sum x_u^2 + sum x_v + eps
           Case 3: sum x_u^2 + sum x_v^2 + eps           Case 4: sum (x_u x_{u+5}^4)^2 + eps
           Case 5: sum (x_u x_{u+5}^8)^2 + eps           (u = 10..14, v = 15..19)
      G4 = sum_{v=15..19} 1 / x_v + eps
    Readings of the garbled or unstated points: G2's A_j runs over G2's own indices; Cases 4-5
    pair u with v = u + 5; |x_v| below 1e-3 is moved out to 1e-3 (keeping its sign) in 1/x_v;
    log|G| is floored at log(1e-12); every eps is its own N(0, noise_sd^2) draw, twelve per
    evaluation, from counters 12 e .. 12 e + 11 of the noise stream (e the evaluation index)."""

    d = 20
    n_routines = 4
    GROUPS = ((0, 5), (5, 10), (10, 15), (15, 20))

    def __init__(self, case: int, noise_sd: float = 0.0, seed: int = 0):
        assert case in (1, 2, 3, 4, 5)
        self.case, self.noise_sd, self.seed = case, float(noise_sd), int(seed)

    def group_values(self, U: np.ndarray, noise_counter0: int = 0) -> np.ndarray:
        """(..., 4) raw group values G1..G4 (before the logarithm)."""
        U = np.asarray(U, dtype=np.float64)
        x = -50.0 + 100.0 * U
        lead = x.shape[:-1]
        if self.noise_sd > 0:
            n = int(np.prod(lead)) if lead else 1
            cnt = (np.arange(n, dtype=np.uint64)[:, None] + np.uint64(noise_counter0)) * np.uint64(12) \
                + np.arange(12, dtype=np.uint64)[None, :]
            eps = (self.noise_sd * normal(self.seed, STREAM_NOISE, cnt)).reshape(lead + (12,))
        else:
            eps = np.zeros(lead + (12,))
        A = 10.0 * np.cos(2.0 * math.pi * (x[..., 0:10] - 1.0)) + eps[..., 0:10]
        g1 = np.sum((x[..., 0:4] - x[..., 1:5]) ** 2, axis=-1) + np.sum(A[..., 0:5], axis=-1)
        g2 = np.sum((x[..., 5:9] - x[..., 6:10]) ** 4, axis=-1) + np.sum(A[..., 5:10], axis=-1)
        xu, xv = x[..., 10:15], x[..., 15:20]
        if self.case == 1:
            g3 = np.sum(xu, axis=-1) + np.sum(np.cos(2.0 * math.pi * xv), axis=-1)
        elif self.case == 2:
            g3 = np.sum(xu ** 2, axis=-1) + np.sum(xv, axis=-1)
        elif self.case == 3:
            g3 = np.sum(xu ** 2, axis=-1) + np.sum(xv ** 2, axis=-1)
        elif self.case == 4:
            g3 = np.sum((xu * xv ** 4) ** 2, axis=-1)
        else:
            g3 = np.sum((xu * xv ** 8) ** 2, axis=-1)
        g3 = g3 + eps[..., 10]
        xs = np.where(np.abs(xv) < 1e-3, np.where(xv < 0, -1e-3, 1e-3), xv)
        g4 = np.sum(1.0 / xs, axis=-1) + eps[..., 11]
        return np.stack([g1, g2, g3, g4], axis=-1)

    def routines(self, U: np.ndarray, noise_counter0: int = 0) -> np.ndarray:
        """(..., 4) routine outputs log|G_g|."""
        return np.log(np.maximum(np.abs(self.group_values(U, noise_counter0)), 1e-12))

    def __call__(self, U: np.ndarray, noise_counter0: int = 0) -> np.ndarray:
        return self.routines(U, noise_counter0).sum(axis=-1)


def five_block_objective(seed: int, noise_sd: float = 0.01) -> Objective:
    """d=20: five planted blocks of four inputs, Ackley on even blocks, Rastrigin on odd."""
    return Objective([4] * 5, [FN_ACKLEY, FN_RASTRIGIN] * 2 + [FN_ACKLEY], noise_sd, seed)


# ---------------------------------------------------------------- workloads
@dataclass
class GPWorkload:
    name: str
    seed: int
    n: int
    d: int
    M: int
    objective: Objective
    prec: str                       # "f64" | "f32" | "bf16"
    X: np.ndarray = field(repr=False, default=None)
    y: np.ndarray = field(repr=False, default=None)
    lengthscale: np.ndarray = field(repr=False, default=None)
    signal_var: float = 1.0
    noise_var: float = 1e-6

    def candidates(self, M: int | None = None, first: int = 0) -> np.ndarray:
        """The seeded candidate pool as float32 (exact: 24-bit grid)."""
        M = self.M if M is None else M
        return uniform_points(self.seed, STREAM_CAND, M, self.d, first).astype(np.float32)


def lengthscale_rule(d: int) -> np.ndarray:
    """0.3 * sqrt(d/4) per dimension: keeps the typical scaled distance fixed as d grows."""
    return np.full(d, 0.3 * math.sqrt(d / 4.0))


def make_gp_workload(name: str, seed: int, n: int, objective: Objective, M: int, prec: str,
                     noise_floor: float = 1e-6, obs_noise_sd: float | None = None) -> GPWorkload:
    d = objective.d
    X = uniform_points(seed, STREAM_OBS, n, d)
    y = objective(X)
    sd = float(np.std(y)) or 1.0
    obs = objective.noise_sd if obs_noise_sd is None else obs_noise_sd
    noise_var = max(noise_floor, (obs / sd) ** 2)
    return GPWorkload(name, seed, n, d, M, objective, prec, X, y, lengthscale_rule(d), 1.0, noise_var)


def config1() -> GPWorkload:
    """n=64, d=4 Rosenbrock(x0,x1)+Rosenbrock(x2,x3), noise-free, M=4096, FP64 scoring."""
    obj = Objective([2, 2], [FN_ROSENBROCK, FN_ROSENBROCK], 0.0, 2404)
    return make_gp_workload("rosenbrock2x2_n64_d4_m4096_f64", 2404, 64, obj, 4096, "f64")


def config2() -> GPWorkload:
    """n=512, d=20 five-block Ackley/Rastrigin + N(0, 0.01^2), M=65536, FP32 scoring."""
    obj = five_block_objective(2405)
    return make_gp_workload("fiveblock_n512_d20_m65536_f32", 2405, 512, obj, 65536, "f32")


def config4(n: int = 4096, M: int = 1 << 20, prec: str = "bf16") -> GPWorkload:
    """n=4096, d=20 five-block function, M=2^20 candidates, BF16 variance tiles."""
    obj = five_block_objective(2407)
    return make_gp_workload(f"fiveblock_n{n}_d20_m{M}_{prec}", 2407, n, obj, M, prec)


@dataclass
class ScreenWorkload:
    """Screen settings.  The routine-mode cut-off is the paper's 25% for its synthetic
    functions (§IV-D); the pairwise interaction ratio uses the paper's other cut-off,
    10% (§VIII), because its separable and cross-block values sit at noise level
    (< 0.03) while planted interacting pairs stay above 0.12."""
    objective: Objective
    n_base: int = 32
    h: float = 0.1
    cutoff: float = 0.10
    cutoff_routine: float = 0.25
    max_dims: int = 10
    seed: int = 2405


def screen_config2(noise_sd: float = 0.01) -> ScreenWorkload:
    """190 pairs of the d=20 five-block function, 32 base points, h=0.1, cut-off 25%."""
    return ScreenWorkload(five_block_objective(2405, noise_sd))


def batched_config3(seed: int = 2406, G: int = 64, M: int = 16384):
    """G independent sub-searches: d_g in U{2..12}, n_g in U{32..1024}, block fn cycling
    Ackley, Rastrigin, Rosenbrock (chained for d_g > 2)."""
    u = uniform24(seed, STREAM_SHAPES, np.arange(2 * G, dtype=np.uint64))
    ds = (2 + np.floor(u[:G] * 11)).astype(int)
    ns = (32 + np.floor(u[G:] * 993)).astype(int)
    fns = [FN_ACKLEY, FN_RASTRIGIN, FN_ROSENBROCK]
    out = []
    for g in range(G):
        obj = Objective([int(ds[g])], [fns[g % 3]], 0.01, seed * 1000 + g)
        out.append(make_gp_workload(f"sub{g}", seed * 1000 + g, int(ns[g]), obj, M, "f32"))
    return out


def mle_box(d: int):
    """Bounds on theta = (log l_1..l_d, log signal_var, log noise_var) for standardised y in
    the unit cube: lengthscales 0.01..100, signal variance e^-3..e^3, noise variance
    e^-14..1."""
    lo = np.concatenate([np.full(d, math.log(0.01)), [-3.0, -14.0]])
    hi = np.concatenate([np.full(d, math.log(100.0)), [3.0, 0.0]])
    return lo, hi


def mle_starts(seed: int, count: int, d: int) -> np.ndarray:
    """Starting points of the multi-start hyperparameter fit: the rule's point
    (lengthscale_rule, signal 1, noise 1e-3) first, then draws uniform in the log box
    narrowed to lengthscales 0.05..5, signal e^-1..e^1, noise e^-10..e^-2 (stream 8)."""
    base = np.concatenate([np.log(lengthscale_rule(d)), [0.0, math.log(1e-3)]])
    if count <= 1:
        return np.repeat(base[None, :], count, axis=0)
    u = uniform_points(seed, STREAM_MLE_STARTS, count - 1, d + 2)
    lo = np.concatenate([np.full(d, math.log(0.05)), [-1.0, -10.0]])
    hi = np.concatenate([np.full(d, math.log(5.0)), [1.0, -2.0]])
    return np.vstack([base, lo + u * (hi - lo)])
