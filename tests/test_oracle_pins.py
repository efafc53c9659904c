"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each check is chosen so that a plausible slip in the oracle (a dropped
strictness test, a swapped operand, a row sum instead of a column sum, an
off-by-one in l, a wrong Philox constant, a wrong pivot rule...) fails here:

* Philox-4x32-10 against the library implementation shipped with Triton
  (run in its CPU interpreter).
* Dominance on the full grid {0..q-1}^m against the closed-form pair count
  (q(q+1)/2)^m - q^m and the per-point count prod_k (q - a_k) - 1.
* Ranks on the full grid equal sum_k a_k (longest chain from the origin);
  Deb's sort (Algorithm S.2), the peel (Algorithm S.3) and a longest-chain
  dynamic programme agree on random inputs with ties.
* Front points with sum f = 0.5 or ||f|| = 1 form one front.
* Intercepts equal alpha for corner points z + alpha_k e_k; the linear front
  gives a = 0.5; a doubled extreme point forces the nadir fallback.
* A point s R_j associates to j with distance 0; adding delta u with u
  orthogonal to R_j gives distance delta ||u||.
* Niching equals a literal one-pick-at-a-time run of Algorithm S.1 that
  breaks ties by the same random priorities.
* TensorHypE selection (Algorithms S.10, S.11): with k = 1 the estimate of
  each point is its exclusive hypervolume, exact on a regular sample lattice;
  with one front and N = 1 the estimates sum to sum_i (n1 - c_i)/(n1 - 1)
  (c_i counted by brute force); P is kept, nothing beyond front l.
* One-shot niching (Algorithm S.4 + Update-Rank, Algorithm S.6): when the
  number of empty niches with candidates equals K, it selects exactly what
  the level form selects at its only level (a separate code path); adding
  or dropping points follows a plain sort of the Philox keys.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_2503_20286_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------- Philox
def test_philox_matches_triton_library():
    # the interpreter flag must be set before triton is first imported
    os.environ["TRITON_INTERPRET"] = "1"
    pytest.importorskip("triton")
    from tests import _triton_philox

    n = 64
    rng = np.random.default_rng(7)
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    key[0] = 0
    ctr[1] = 0xFFFFFFFF
    key[1] = 0xFFFFFFFF
    ref = _triton_philox.philox(ctr, key)
    mine = np.stack([oracle.philox4x32_10(ctr[i], key[i]) for i in range(n)])
    assert np.array_equal(mine, ref)


# ------------------------------------------------------------------ dominance
def grid(q, m):
    return np.array(list(itertools.product(range(q), repeat=m)), dtype=np.float32)


@pytest.mark.parametrize("q,m", [(3, 2), (3, 3), (4, 2), (2, 4)])
def test_dominance_grid_closed_forms(q, m):
    F = grid(q, m)
    n = F.shape[0]
    D = oracle.dominance_bits(F)
    bits = np.unpackbits(D.view(np.uint8), bitorder="little").reshape(n, -1)[:, :n]
    # total number of dominance pairs: coordinatewise <= pairs minus equal pairs
    assert bits.sum() == (q * (q + 1) // 2) ** m - q ** m
    # minimisation: point a dominates exactly prod(q - a_k) - 1 grid points
    for i in range(n):
        assert bits[i].sum() == int(np.prod(q - F[i])) - 1
    # never reflexive, never both ways
    assert not np.any(np.diag(bits))
    assert not np.any(bits & bits.T)
    # column sums are the dominator counts: prod(a_k + 1) - 1
    c = oracle.domination_counts(F)
    assert np.array_equal(c, (np.prod(F + 1, axis=1) - 1).astype(np.int32))
    assert np.array_equal(c, bits.sum(axis=0))


def test_dominance_direction_and_duplicates():
    assert oracle.dominates([0.0, 0.0], [1.0, 1.0])
    assert not oracle.dominates([1.0, 1.0], [0.0, 0.0])
    assert oracle.dominates([0.0, 1.0], [0.0, 2.0])
    assert not oracle.dominates([1.0, 1.0], [1.0, 1.0])       # identical points
    assert not oracle.dominates([0.0, 2.0], [1.0, 1.0])       # incomparable
    assert not oracle.dominates([-0.0, 1.0], [0.0, 1.0])      # -0 == +0


# ------------------------------------------------------------------- ranks
def longest_chain_ranks(F):
    """Rank = length of the longest dominance chain ending at the point."""
    F = F.astype(np.float64)
    le = np.all(F[:, None, :] <= F[None, :, :], axis=2)
    lt = np.any(F[:, None, :] < F[None, :, :], axis=2)
    dom = le & lt
    n = F.shape[0]
    rank = np.zeros(n, dtype=np.int64)
    for _ in range(n):
        cand = np.where(dom, rank[:, None] + 1, 0).max(axis=0)
        new = np.maximum(rank, cand)
        if np.array_equal(new, rank):
            break
        rank = new
    return rank.astype(np.int32)


@pytest.mark.parametrize("q,m", [(3, 2), (4, 3), (3, 4)])
def test_grid_ranks_are_coordinate_sums(q, m):
    F = grid(q, m)
    expect = F.sum(axis=1).astype(np.int32)
    assert np.array_equal(oracle.nd_sort_deb(F), expect)
    assert np.array_equal(oracle.nd_sort_peel(F), expect)


@pytest.mark.parametrize("seed", range(6))
def test_sorts_agree_with_longest_chain(seed):
    rng = np.random.default_rng(seed)
    m = int(rng.integers(2, 6))
    n = int(rng.integers(2, 90))
    F = rng.integers(0, 4, size=(n, m)).astype(np.float32)   # many ties/duplicates
    ref = longest_chain_ranks(F)
    assert np.array_equal(oracle.nd_sort_deb(F), ref)
    assert np.array_equal(oracle.nd_sort_peel(F), ref)


def test_exhaustive_tiny_populations():
    # every population of 4 points in {0,1,2}^2 (6561 populations)
    pts = grid(3, 2)
    for combo in itertools.product(range(9), repeat=4):
        F = pts[list(combo)]
        ref = longest_chain_ranks(F)
        assert np.array_equal(oracle.nd_sort_deb(F), ref), combo


@pytest.mark.parametrize("shape,m", [("linear", 3), ("sphere", 3), ("sphere", 5), ("linear", 8)])
def test_front_points_form_one_front(shape, m):
    F = wl.front_points(300, m, shape, seed=11)
    if shape == "linear":
        assert np.allclose(F.astype(np.float64).sum(1), 0.5, atol=1e-6)
    else:
        assert np.allclose(np.linalg.norm(F.astype(np.float64), axis=1), 1.0, atol=1e-6)
    r = oracle.nd_sort_deb(F)
    # float32 rounding can put two nearly identical points in a dominance
    # relation; check against the brute-force chain and that front 0 holds
    # almost everything
    assert np.array_equal(r, longest_chain_ranks(F))
    assert (r == 0).mean() > 0.97


# ---------------------------------------------------------------- selection
def test_das_dennis_counts():
    # closed form C(H+M-1, M-1); values of the five workloads
    assert wl.das_dennis(12, 3).shape[0] == 91
    assert wl.das_dennis(140, 3).shape[0] == 10011
    assert wl.das_dennis_two_layer(3, 2, 8).shape[0] == 156
    assert wl.das_dennis_count(631, 3) == 200028
    for h, m in [(4, 3), (5, 4), (3, 6)]:
        R = wl.das_dennis(h, m)
        assert R.shape[0] == math.comb(h + m - 1, m - 1)
        assert np.allclose(R.astype(np.float64).sum(1), 1.0, atol=1e-6)
        assert len({tuple(r) for r in R.tolist()}) == R.shape[0]


def check_selection_invariants(F, R, n_keep, surv, t):
    n2 = F.shape[0]
    rank = t["rank"]
    l = t["last_rank"]
    assert len(surv) == n_keep
    assert np.all(np.diff(surv) > 0)
    P = np.flatnonzero(rank < l)
    L = np.flatnonzero(rank == l)
    assert len(P) == t["n_before"] and len(L) == t["n_last"]
    assert len(P) < n_keep <= len(P) + len(L)
    assert np.sort(rank)[n_keep - 1] == l
    assert set(P.tolist()) <= set(surv.tolist())
    extra = sorted(set(surv.tolist()) - set(P.tolist()))
    assert set(extra) <= set(L.tolist())
    assert np.array_equal(np.flatnonzero(t["picked"]), np.array(extra, dtype=np.int64))
    S = rank <= l
    # ideal point = column minima of S = column minima of front 0
    assert np.array_equal(t["z"], F[S].astype(np.float64).min(0))
    assert np.array_equal(t["z"], F[rank == 0].astype(np.float64).min(0))
    # association outside S is undefined, inside it is a valid index
    assert np.all(t["pi"][~S] == -1) and np.all((t["pi"][S] >= 0) & (t["pi"][S] < R.shape[0]))
    # rho counts P members per reference
    assert np.array_equal(t["rho"], np.bincount(t["pi"][P], minlength=R.shape[0]).astype(np.int32))


@pytest.mark.parametrize("cfg_seed", range(4))
def test_selection_invariants_small(cfg_seed):
    F = wl.population(184, 3, 7, "linear", seed=100 + cfg_seed)
    R = wl.das_dennis(12, 3)
    surv, t = oracle.nsga3_select(F, R, 92, seed=5, generation=cfg_seed)
    check_selection_invariants(F, R, 92, surv, t)
    assert np.array_equal(t["rank"], longest_chain_ranks(F))


def test_intercepts_corner_points():
    rng = np.random.default_rng(3)
    alpha = np.array([0.5, 2.0, 4.0], dtype=np.float64)
    z = np.array([0.25, 1.0, -0.5])
    corners = z + np.diag(alpha)
    interior = z + rng.uniform(0.05, 0.45, size=(40, 3)) * alpha
    F = np.vstack([interior[:20], corners, interior[20:]]).astype(np.float32)
    R = wl.das_dennis(4, 3)
    surv, t = oracle.nsga3_select(F, R, 30, seed=1)
    assert np.array_equal(t["z"], z)
    assert list(t["extreme"]) == [20, 21, 22]
    assert t["fallback"] == 0
    np.testing.assert_allclose(t["a"], alpha, rtol=1e-14)
    # normalised corners sit on the axes at 1
    S = t["rank"] <= t["last_rank"]
    assert np.all(S[20:23])
    np.testing.assert_allclose(t["fnorm"][20:23], np.eye(3), atol=1e-15)


def test_intercepts_linear_front():
    F = wl.front_points(200, 3, "linear", seed=4).astype(np.float64)
    F = np.vstack([np.eye(3) * 0.5, F]).astype(np.float32)
    surv, t = oracle.nsga3_select(F, wl.das_dennis(6, 3), 100, seed=2)
    assert t["fallback"] == 0
    assert np.array_equal(t["z"], np.zeros(3))
    np.testing.assert_allclose(t["a"], [0.5, 0.5, 0.5], rtol=1e-12)


def test_intercepts_degenerate_fallback_to_nadir():
    F = wl.population(400, 4, 13, "sphere", seed=21)
    G = wl.ideal_corner_case(F)
    surv, t = oracle.nsga3_select(G, wl.das_dennis(4, 4), 200, seed=3)
    assert t["extreme"][0] == t["extreme"][1] == 0
    assert t["fallback"] == 1
    S = t["rank"] <= t["last_rank"]
    nadir = (G[S].astype(np.float64) - t["z"]).max(0)
    assert np.array_equal(t["a"], nadir)


def test_association_closed_forms():
    # points on reference lines and at known offsets from them
    R = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]], dtype=np.float32)
    corners = np.eye(3, dtype=np.float32)
    on_line = np.array([[0.25, 0.25, 0.25], [0.5, 0.5, 0.5]], dtype=np.float32)
    u = np.array([1.0, -1.0, 0.0])           # orthogonal to (1,1,1)
    delta = 0.0625
    off = (np.array([0.375, 0.375, 0.375]) + delta * u).astype(np.float32)
    F = np.vstack([corners, on_line, off[None]]).astype(np.float32)
    surv, t = oracle.nsga3_select(F, R, F.shape[0], seed=0)
    # z = 0, corners give a = 1, so f' = F
    assert np.array_equal(t["a"], [1.0, 1.0, 1.0])
    assert list(t["pi"][:3]) == [0, 1, 2]
    assert list(t["pi"][3:]) == [3, 3, 3]
    assert np.all(t["dist"][:5] == 0.0)
    np.testing.assert_allclose(t["dist"][5], delta * np.linalg.norm(u), rtol=1e-15)


def test_keep_whole_last_front_selects_it_all():
    F = wl.population(120, 3, 8, "sphere", seed=9)
    r = oracle.nd_sort_deb(F)
    sizes = np.bincount(r)
    n_keep = int(sizes[:3].sum())                   # exactly fills fronts 0..2
    surv, t = oracle.nsga3_select(F, wl.das_dennis(5, 3), n_keep, seed=4)
    assert t["last_rank"] == 2
    assert np.array_equal(surv, np.flatnonzero(r <= 2))


def niche_random(seed, gen, j, c, tag):
    ctr = [j & 0xFFFFFFFF, (2 * c + tag) & 0xFFFFFFFF, gen & 0xFFFFFFFF, gen >> 32]
    key = [seed & 0xFFFFFFFF, seed >> 32]
    return int(oracle.philox4x32_10(ctr, key)[0])


def sequential_s1(t, n_r, n_keep, seed, gen):
    """Algorithm S.1, one pick per iteration: least-crowded live reference
    (ties by the random priority of the current crowding), nearest member
    when it has no member yet, otherwise a random member."""
    rank, pi, dist = t["rank"], t["pi"], t["dist"]
    l = t["last_rank"]
    rho = np.bincount(pi[rank < l], minlength=n_r).astype(np.int64)
    C = {j: [] for j in range(n_r)}
    for i in np.flatnonzero(rank == l):
        C[int(pi[i])].append(int(i))
    live = {j for j in range(n_r) if C[j]}
    need = n_keep - int((rank < l).sum())
    picked = []
    while need > 0:
        cmin = min(rho[j] for j in live)
        ties = [j for j in live if rho[j] == cmin]
        j = min(ties, key=lambda q: (niche_random(seed, gen, q, cmin, 0), q))
        if rho[j] == 0:
            a = min(C[j], key=lambda i: (dist[i], i))
        else:
            u = niche_random(seed, gen, j, int(rho[j]), 1)
            a = C[j][(u * len(C[j])) >> 32]
        C[j].remove(a)
        picked.append(a)
        rho[j] += 1
        need -= 1
        if not C[j]:
            live.discard(j)
    return sorted(picked)


@pytest.mark.parametrize("case", range(8))
def test_niching_equals_sequential_algorithm_s1(case):
    rng = np.random.default_rng(50 + case)
    m = int(rng.integers(2, 5))
    n2 = int(rng.integers(40, 260))
    shape = "linear" if case % 2 else "sphere"
    F = wl.population(n2, m, m + 4, shape, seed=77 + case)
    if case >= 6:
        F = (np.round(F * 8) / 8).astype(np.float32)   # ties and duplicates
    H = int(rng.integers(2, 7))
    R = wl.das_dennis(H, m)
    n_keep = int(rng.integers(1, n2 + 1))
    seed, gen = int(rng.integers(0, 2 ** 63)), int(rng.integers(0, 2 ** 40))
    surv, t = oracle.nsga3_select(F, R, n_keep, seed=seed, generation=gen)
    check_selection_invariants(F, R, n_keep, surv, t)
    assert np.flatnonzero(t["picked"]).tolist() == sequential_s1(t, R.shape[0], n_keep, seed, gen)


def test_golden_config0():
    """Regression fixture written by tests/golden/make_golden.py (oracle only)."""
    path = os.path.join(GOLDEN, "config0_oracle.txt")
    gold = {}
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split(":", 1)
            gold[k.strip()] = v.strip()
    p = wl.config(0)
    surv, t = oracle.nsga3_select(p.F, p.R, p.n_keep, p.seed, p.generation)
    assert " ".join(map(str, surv.tolist())) == gold["survivors"]
    assert " ".join(map(str, t["rank"].tolist())) == gold["rank"]
    assert int(gold["last_rank"]) == t["last_rank"]


def _oneshot_key(seed, gen, i, tag):
    ctr = [i & 0xFFFFFFFF, 0xFFFFFFF0 + tag, gen & 0xFFFFFFFF, gen >> 32]
    key = [seed & 0xFFFFFFFF, seed >> 32]
    return (int(oracle.philox4x32_10(ctr, key)[0]) << 32) | i


def _empty_niche_case(idx):
    """A population and the n_keep at which K equals the number of empty
    niches holding last-front candidates (E0), with the level-form trace."""
    rng = np.random.default_rng(700 + idx)
    m = int(rng.integers(2, 5))
    n2 = int(rng.integers(120, 400))
    F = wl.population(n2, m, m + 4, "sphere" if idx % 2 else "linear", seed=900 + idx)
    if idx >= 4:
        F = (np.round(F * 16) / 16).astype(np.float32)   # ties and duplicates
    R = wl.das_dennis(wl.h_for_count(n2 // 2, m), m)   # about n2 / 2 references: many empty niches
    seed, gen = int(rng.integers(0, 2 ** 63)), int(rng.integers(0, 2 ** 40))
    n_keep = int(rng.integers(n2 // 4, 3 * n2 // 4))
    _, t = oracle.nsga3_select(F, R, n_keep, seed, gen)
    l, nP = t["last_rank"], t["n_before"]
    L = np.flatnonzero(t["rank"] == l)
    E0 = np.unique(t["pi"][L][t["rho"][t["pi"][L]] == 0])
    return F, R, seed, gen, nP, len(L), len(E0)


@pytest.mark.parametrize("idx", range(6))
def test_oneshot_equals_level_form_when_empty_niches_fill_k(idx):
    F, R, seed, gen, nP, nL, nE0 = _empty_niche_case(idx)
    if nE0 == 0:
        pytest.skip("no empty niche with candidates")
    n_keep = nP + nE0   # K = |E0|: one level of nearest picks, no add, no drop
    s0, t0 = oracle.nsga3_select(F, R, n_keep, seed, gen, mode=oracle.NICHE_EXACT)
    s1, t1 = oracle.nsga3_select(F, R, n_keep, seed, gen, mode=oracle.NICHE_ONESHOT)
    assert t0["n_levels"] == 1 and t0["n_before"] == nP
    assert np.array_equal(s0, s1)


@pytest.mark.parametrize("idx", range(6))
def test_oneshot_add_and_drop_follow_philox_order(idx):
    F, R, seed, gen, nP, nL, nE0 = _empty_niche_case(idx)
    if nE0 < 4 or nL - nE0 < 4:
        pytest.skip("too few empty niches or remaining candidates")
    base, t = oracle.nsga3_select(F, R, nP + nE0, seed, gen, mode=oracle.NICHE_EXACT)
    Q = np.setdiff1d(base, np.flatnonzero(t["rank"] < t["last_rank"]))
    P = np.flatnonzero(t["rank"] < t["last_rank"])
    L = np.flatnonzero(t["rank"] == t["last_rank"])
    # add 3: the three remaining last-front points with the smallest add keys
    rest = sorted(np.setdiff1d(L, Q).tolist(), key=lambda i: _oneshot_key(seed, gen, i, 1))
    s_add, _ = oracle.nsga3_select(F, R, nP + nE0 + 3, seed, gen, mode=oracle.NICHE_ONESHOT)
    assert np.array_equal(s_add, np.sort(np.concatenate([P, Q, rest[:3]])))
    # drop 3: the three taken points with the smallest drop keys
    taken = sorted(Q.tolist(), key=lambda i: _oneshot_key(seed, gen, i, 2))
    s_drop, _ = oracle.nsga3_select(F, R, nP + nE0 - 3, seed, gen, mode=oracle.NICHE_ONESHOT)
    assert np.array_equal(s_drop, np.sort(np.concatenate([P, taken[3:]])))
    # exactly N survivors, P kept, picks from the last front only
    for n_keep, sv in ((nP + nE0 + 3, s_add), (nP + nE0 - 3, s_drop)):
        assert len(sv) == n_keep and np.all(np.isin(P, sv)) and np.all(np.isin(np.setdiff1d(sv, P), L))


def _lattice(g, m=2):
    u = (np.arange(g, dtype=np.float64) + 0.5) / g
    grid = np.stack(np.meshgrid(*([u] * m), indexing="ij"), axis=-1).reshape(-1, m)
    return grid.astype(np.float32)


def test_hype_exclusive_volume_on_a_lattice():
    # three points of one front and one dominated point; f_l = (1, 1), v_ref = (4, 4)
    F = np.array([[1, 3], [2, 2], [3, 1], [2, 3]], np.float32)
    U = _lattice(30)                                   # samples 1.05, 1.15, ..., 3.95 per axis
    surv, vhv, l = oracle.hype_select(F, np.array([4, 4], np.float32), U, 2)   # k = 1
    assert l == 0
    # each front point alone dominates a 1 x 1 square: 100 lattice samples of 900, volume 9
    assert vhv[:3].tolist() == [1.0, 1.0, 1.0]
    assert vhv[3] == 0.0                              # every sample it dominates has c >= 3
    assert surv.tolist() == [0, 1]                    # equal estimates: lower indices kept


def test_hype_drops_the_smallest_exclusive_volume():
    # exclusive areas 0.5, 0.75 and 1.5; lattice samples 1.0375 + 0.075 i per
    # axis: 7 x 13, 20 x 7 and 13 x 20 of them fall in those regions
    F = np.array([[1, 3], [1.5, 2.5], [3, 1]], np.float32)
    U = _lattice(40)
    surv, vhv, _ = oracle.hype_select(F, np.array([4, 4], np.float32), U, 2)
    assert vhv.tolist() == [91 * 9 / 1600, 140 * 9 / 1600, 260 * 9 / 1600]
    assert surv.tolist() == [1, 2]


@pytest.mark.parametrize("m", [2, 3, 4])
def test_hype_weights_sum_identity(m):
    rng = np.random.default_rng(31 + m)
    F = wl.front_points(40, m, "linear", seed=60 + m)         # one front
    v_ref = np.full(m, 0.7, np.float32)
    U = rng.random((500, m)).astype(np.float32)
    _, vhv, l = oracle.hype_select(F, v_ref, U, 1)            # k = n1 - 1
    assert l == 0
    n1 = F.shape[0]
    fl = F.min(axis=0)
    S = (fl + U * (v_ref - fl).astype(np.float32)).astype(np.float32)
    c = (F[None, :, :] <= S[:, None, :]).all(axis=2).sum(axis=1)
    vol = np.prod(v_ref.astype(np.float64) - fl.astype(np.float64))
    expect = np.sum((n1 - c[c > 0]) / (n1 - 1)) * vol / U.shape[0]
    assert abs(vhv.sum() - expect) <= 1e-12 * max(1.0, expect)


@pytest.mark.parametrize("case", range(4))
def test_hype_selection_invariants(case):
    rng = np.random.default_rng(80 + case)
    m = int(rng.integers(2, 5))
    n2 = int(rng.integers(30, 200))
    F = wl.population(n2, m, m + 4, "sphere", seed=90 + case)
    U = rng.random((300, m)).astype(np.float32)
    n_keep = int(rng.integers(1, n2 + 1))
    surv, vhv, l = oracle.hype_select(F, (F.max(axis=0) + 0.1).astype(np.float32), U, n_keep)
    r = oracle.nd_sort_deb(F)
    assert l == np.sort(r)[n_keep - 1]
    assert len(surv) == n_keep and np.all(np.diff(surv) > 0)
    assert np.all(np.isin(np.flatnonzero(r < l), surv)) and np.all(r[surv] <= l)
    last = np.setdiff1d(np.flatnonzero(r == l), surv)
    kept = np.setdiff1d(surv, np.flatnonzero(r < l))
    if len(last) and len(kept):   # every kept last-front point scores at least every dropped one
        assert vhv[kept].min() >= vhv[last].max()


def _layering_2d(F):
    """Textbook two-objective non-dominated sorting: visit the points in
    lexicographic order (f1, then f2); a point joins the first front whose
    most recent member does not dominate it. The most recent member of a
    front has that front's smallest f2 among points with f1 <= the visited
    point's f1, so it is the only member that can dominate the point, and
    the fronts' most recent f2 values grow with the front index (binary
    search)."""
    order = sorted(range(len(F)), key=lambda i: (float(F[i][0]), float(F[i][1]), i))
    last = []                        # most recent member of each front
    rank = np.zeros(len(F), np.int32)

    def dominates(a, b):
        return a[0] <= b[0] and a[1] <= b[1] and (a[0] < b[0] or a[1] < b[1])

    for i in order:
        lo, hi = 0, len(last)
        while lo < hi:
            mid = (lo + hi) // 2
            if dominates(F[last[mid]], F[i]):
                lo = mid + 1
            else:
                hi = mid
        if lo == len(last):
            last.append(i)
        else:
            last[lo] = i
        rank[i] = lo
    return rank


@pytest.mark.parametrize("seed,q", [(1, 4), (2, 16), (3, 0)])
def test_two_objective_ranks_equal_textbook_layering(seed, q):
    rng = np.random.default_rng(seed)
    F = rng.random((600, 2)).astype(np.float32)
    if q:
        F = (np.round(F * q) / q).astype(np.float32)     # ties and duplicates
    ref = _layering_2d(F)
    assert np.array_equal(oracle.nd_sort_deb(F), ref)
    assert np.array_equal(oracle.nd_sort_peel(F), ref)
