"""Seeded synthetic inputs for NSGA-III environmental selection.

This module produces the *inputs* of the selection path and nothing else:
merged populations ``F`` (float32, row-major ``[2N][M]``), reference
directions ``R`` (float32, ``[n_r][M]``) and the batch descriptors of the
many-population workload. It contains none of the selection arithmetic, so
both the CUDA path and the CPU oracle consume exactly the same float32
arrays.

Shapes follow the paper's workloads (Section VI, Table S.II): DTLZ-style
populations with a linear front (sum f = 0.5) or a spherical front
(||f|| = 1). The DTLZ definitions themselves are not reproduced; the
geometric stand-in below has the same front shapes and a convergence gap
``(1 + g) >= 1`` driven by the tail decision variables:

* decision vectors ``x`` uniform in ``[0, 1)^D`` (float32 draws);
* position part: the first ``M - 1`` coordinates;
* linear shape: ``s`` = stick-breaking point of the unit simplex,
  ``f = 0.5 (1 + 100 g) s``;
* sphere shape: ``s`` = hyperspherical unit vector with angles
  ``x_i * pi / 2``, ``f = (1 + g) s``;
* ``g = sum_{i >= M} (x_i - 0.5)^2``;
* computed in float64, rounded once to float32.

Das-Dennis directions (the paper's reference tensor R, Section III-B) are
all compositions of ``H`` into ``M`` non-negative parts, in lexicographic
order, with values ``k / H`` (float64, rounded to float32). The two-layer
set appends an inner layer ``0.5 * (k / H2) + 0.5 / M``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 0x250320286


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    """Counter-based Philox stream from numpy (independent of the method)."""
    return np.random.Generator(np.random.Philox(key=[seed & 0xFFFFFFFFFFFFFFFF, stream]))


def decision_vectors(n: int, d: int, seed: int, stream: int = 0) -> np.ndarray:
    """``n x d`` decision vectors uniform in [0, 1) (float32 values)."""
    return _rng(seed, stream).random((n, d), dtype=np.float32)


def _simplex_point(x: np.ndarray, m: int) -> np.ndarray:
    """Stick-breaking map [0,1)^(m-1) -> unit simplex (float64)."""
    n = x.shape[0]
    s = np.empty((n, m), dtype=np.float64)
    rest = np.ones(n, dtype=np.float64)
    for k in range(m - 1):
        s[:, k] = rest * x[:, k]
        rest = rest * (1.0 - x[:, k])
    s[:, m - 1] = rest
    return s


def _sphere_point(x: np.ndarray, m: int) -> np.ndarray:
    """Hyperspherical unit vector in the positive orthant (float64)."""
    n = x.shape[0]
    ang = x[:, : m - 1].astype(np.float64) * (math.pi / 2.0)
    s = np.empty((n, m), dtype=np.float64)
    prod = np.ones(n, dtype=np.float64)
    for k in range(m - 1):
        s[:, m - 1 - k] = prod * np.sin(ang[:, k])
        prod = prod * np.cos(ang[:, k])
    s[:, 0] = prod
    return s


def objectives_from_decisions(x: np.ndarray, m: int, shape: str) -> np.ndarray:
    """Stand-in objective values for decision vectors ``x`` (float32 out)."""
    xd = x.astype(np.float64)
    g = np.sum((xd[:, m - 1:] - 0.5) ** 2, axis=1)
    if shape == "linear":
        f = 0.5 * (1.0 + 100.0 * g)[:, None] * _simplex_point(xd, m)
    elif shape == "sphere":
        f = (1.0 + g)[:, None] * _sphere_point(xd, m)
    else:
        raise ValueError(f"unknown front shape {shape!r}")
    return f.astype(np.float32)


def population(n2: int, m: int, d: int, shape: str, seed: int, stream: int = 0,
               quantize: float | None = None) -> np.ndarray:
    """Merged population objectives ``F`` of ``n2`` points (float32 [n2][m]).

    ``quantize=q`` rounds every objective to the grid ``1/q`` (half-even),
    which creates duplicated points and ties in single objectives.
    """
    x = decision_vectors(n2, d, seed, stream)
    f = objectives_from_decisions(x, m, shape)
    if quantize:
        f = (np.round(f.astype(np.float64) * quantize) / quantize).astype(np.float32)
    return np.ascontiguousarray(f)


def front_points(n: int, m: int, shape: str, seed: int, stream: int = 7) -> np.ndarray:
    """Points exactly on the front (g = 0): sum f = 0.5 or ||f|| = 1."""
    x = decision_vectors(n, m - 1, seed, stream)
    xd = x.astype(np.float64)
    s = _simplex_point(xd, m) if shape == "linear" else _sphere_point(xd, m)
    scale = 0.5 if shape == "linear" else 1.0
    return (scale * s).astype(np.float32)


def das_dennis(h: int, m: int) -> np.ndarray:
    """All compositions of ``h`` into ``m`` parts, lexicographic, / h (float32)."""
    out: list[tuple[int, ...]] = []

    def rec(prefix: list[int], left: int, slots: int) -> None:
        if slots == 1:
            out.append(tuple(prefix + [left]))
            return
        for k in range(left + 1):
            rec(prefix + [k], left - k, slots - 1)

    rec([], h, m)
    a = np.asarray(out, dtype=np.float64) / float(h)
    return a.astype(np.float32)


def das_dennis_two_layer(h1: int, h2: int, m: int) -> np.ndarray:
    """Outer layer ``H1`` plus inner layer ``H2`` shrunk towards the centre."""
    outer = das_dennis(h1, m).astype(np.float64)
    inner = das_dennis(h2, m).astype(np.float64) * 0.5 + 0.5 / m
    return np.concatenate([outer, inner.astype(np.float32).astype(np.float64)]).astype(np.float32)


def reference_front(h: int, m: int, shape: str) -> np.ndarray:
    """Points of the true front for IGD: Das-Dennis directions scaled onto
    the linear front (sum f = 0.5) or projected onto the unit sphere."""
    w = das_dennis(h, m).astype(np.float64)
    if shape == "linear":
        f = 0.5 * w
    elif shape == "sphere":
        f = w / np.linalg.norm(w, axis=1, keepdims=True)
    else:
        raise ValueError(f"unknown front shape {shape!r}")
    return f.astype(np.float32)


def moead_neighbours(W: np.ndarray, t: int) -> np.ndarray:
    """Indices of the ``t`` weight vectors closest to each one (Euclidean,
    FP64, ties by index; every vector is its own first neighbour)."""
    Wd = np.asarray(W, dtype=np.float64)
    n = Wd.shape[0]
    out = np.empty((n, t), dtype=np.int32)
    for i in range(n):
        d2 = np.sum((Wd - Wd[i]) ** 2, axis=1)
        out[i] = np.lexsort((np.arange(n), d2))[:t]
    return out


def moead_neighbours_fast(W: np.ndarray, t: int, extra: int = 16) -> np.ndarray:
    """``moead_neighbours`` for large weight sets: k-d tree candidates, then
    the same (distance, index) order. A row whose t-th distance ties the
    last candidate's is recomputed exhaustively, so the result equals the
    exhaustive definition."""
    from scipy.spatial import cKDTree
    Wd = np.asarray(W, dtype=np.float64)
    n = Wd.shape[0]
    k = min(n, t + extra)
    _, cand = cKDTree(Wd).query(Wd, k=k)
    cand = np.asarray(cand, dtype=np.int64).reshape(n, k)
    d2 = np.sum((Wd[cand] - Wd[:, None, :]) ** 2, axis=2)
    out = np.empty((n, t), dtype=np.int32)
    for i in range(n):
        order = np.lexsort((cand[i], d2[i]))
        if k < n and d2[i, order[t - 1]] >= d2[i, order[k - 1]]:
            full = np.sum((Wd - Wd[i]) ** 2, axis=1)
            out[i] = np.lexsort((np.arange(n), full))[:t]
        else:
            out[i] = cand[i, order[:t]]
    return out


def das_dennis_count(h: int, m: int) -> int:
    return math.comb(h + m - 1, m - 1)


def h_for_count(target: int, m: int) -> int:
    """Smallest-distance ``H`` with ``C(H+M-1, M-1)`` closest to ``target``."""
    best_h, best = 1, None
    h = 1
    while True:
        c = das_dennis_count(h, m)
        dist = abs(c - target)
        if best is None or dist < best:
            best, best_h = dist, h
        if c > target:
            break
        h += 1
    return best_h


@dataclass
class Problem:
    """One selection problem: objectives, directions and the survivor count."""
    name: str
    F: np.ndarray
    R: np.ndarray
    n_keep: int
    seed: int
    generation: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n2(self) -> int:
        return int(self.F.shape[0])

    @property
    def m(self) -> int:
        return int(self.F.shape[1])

    @property
    def n_r(self) -> int:
        return int(self.R.shape[0])


def ideal_corner_case(F: np.ndarray, delta: float = 2.0 ** -20) -> np.ndarray:
    """Replace point 0 by ``min(F) + (delta, delta, 0, ...)``.

    That point minimises the achievement scalarising function of at least the
    first two axes, so two rows of the extreme-point matrix coincide and the
    hyperplane solve is singular (the nadir fallback of Algorithm S.5).
    """
    G = F.copy()
    p = F.min(axis=0).astype(np.float64)
    p[0] += delta
    p[1] += delta
    G[0] = p.astype(np.float32)
    return G


def config(idx: int, seed: int | None = None) -> Problem | list[Problem]:
    """The five workloads, by index.

    0: 2N=184, M=3, D=7, linear front, H=12 (91 directions).
    1: 2N=20000, M=3, D=12, sphere front, H=140 (10011 directions).
    2: 2N=100000, M=8, D=17, sphere front quantised to 1/64,
       two-layer directions H1=3, H2=2 (156).
    3: 64 populations, 2N log-uniform in [1000, 40000] (even), M in {2,3,5},
       linear/sphere alternating, D=M+9, H giving ~N directions.
    4: 2N=400000, M=3, D=12, sphere front, H=631 (200028 directions).
    """
    s = BASE_SEED + idx if seed is None else seed
    if idx == 0:
        return Problem("2N=184 M=3 linear H=12", population(184, 3, 7, "linear", s),
                       das_dennis(12, 3), 92, s)
    if idx == 1:
        return Problem("2N=20000 M=3 sphere H=140", population(20000, 3, 12, "sphere", s),
                       das_dennis(140, 3), 10000, s)
    if idx == 2:
        return Problem("2N=100000 M=8 sphere q=1/64 H1=3,H2=2",
                       population(100000, 8, 17, "sphere", s, quantize=64.0),
                       das_dennis_two_layer(3, 2, 8), 50000, s)
    if idx == 3:
        return batch_problems(64, s)
    if idx == 4:
        return Problem("2N=400000 M=3 sphere H=631", population(400000, 3, 12, "sphere", s),
                       das_dennis(631, 3), 200000, s)
    raise ValueError(idx)


def batch_problems(count: int, seed: int, lo: float = 1000.0, hi: float = 40000.0,
                   ms=(2, 3, 5)) -> list[Problem]:
    """Independent populations of uneven size and objective count."""
    rng = _rng(seed, 0xB7)
    probs: list[Problem] = []
    for b in range(count):
        n2 = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi))) / 2.0)) * 2
        m = int(ms[int(rng.integers(0, len(ms)))])
        shape = "linear" if b % 2 == 0 else "sphere"
        d = m + 9
        h = h_for_count(n2 // 2, m)
        probs.append(Problem(f"pop{b} 2N={n2} M={m} {shape} H={h}",
                             population(n2, m, d, shape, seed, stream=1000 + b),
                             das_dennis(h, m), n2 // 2, seed, generation=b,
                             meta={"shape": shape, "H": h}))
    return probs
