"""Pins of the oracle's generation operators, the TensorMOEA/D selection and
IGD against closed forms, special cases and an independent formulation.

SBX and PM follow Appendix S.I; the MOEA/D selection is Algorithm S.8 with
the PBI aggregation of Section IV-B; IGD is the experiments' quality
measure. The expected values here come from the mathematics, not from the
oracle's own formulas.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2503_20286_gb300 import workloads as wl


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


# ------------------------------------------------------------------ SBX

def test_sbx_mu_half_returns_the_parents():
    """mu = 0.5 gives beta = 1 for every eta_c: c1 = x1 and c2 = x2."""
    for eta in (0.0, 1.0, 20.0):
        assert oracle.sbx_pair(0.2, 0.6, 0.5, eta) == (0.2, 0.6)


@pytest.mark.parametrize("mu,eta,beta", [(0.25, 0.0, 0.5), (0.75, 0.0, 2.0), (0.125, 1.0, 0.5),
                                         (0.875, 1.0, 2.0), (0.0, 20.0, 0.0)])
def test_sbx_closed_form_spread(mu, eta, beta):
    """eta_c = 0: beta = 2 mu below 0.5 and 1 / (2 - 2 mu) above; eta_c = 1:
    the square roots of those; mu = 0 collapses both children to the mean."""
    x1, x2 = 0.2, 0.6
    c1, c2 = oracle.sbx_pair(x1, x2, mu, eta)
    assert c1 == pytest.approx(0.5 * ((1 + beta) * x1 + (1 - beta) * x2), abs=1e-15)
    assert c2 == pytest.approx(0.5 * ((1 - beta) * x1 + (1 + beta) * x2), abs=1e-15)


def test_sbx_conserves_the_mean_and_mirrors_the_spread():
    """c1 + c2 = x1 + x2 for every mu; the spread |c1 - c2| / |x1 - x2| at mu
    and at 1 - mu multiply to 1 (the two branches are reciprocal)."""
    rng = np.random.default_rng(5)
    for _ in range(200):
        x1, x2 = rng.random(2)
        mu = rng.uniform(0.01, 0.49)
        eta = rng.uniform(0.0, 30.0)
        a1, a2 = oracle.sbx_pair(x1, x2, mu, eta)
        b1, b2 = oracle.sbx_pair(x1, x2, 1.0 - mu, eta)
        assert a1 + a2 == pytest.approx(x1 + x2, abs=1e-14)
        assert b1 + b2 == pytest.approx(x1 + x2, abs=1e-14)
        sa = abs(a1 - a2) / abs(x1 - x2)
        sb = abs(b1 - b2) / abs(x1 - x2)
        assert sa * sb == pytest.approx(1.0, rel=1e-12)
        assert sa <= 1.0 <= sb


# ------------------------------------------------------------------ PM

def test_pm_mu_half_is_the_identity():
    for x in (0.0, 0.3, 0.999, 1.0):
        assert oracle.pm_value(x, 0.0, 1.0, 0.5, 20.0) == x


def test_pm_extremes_reach_the_bounds():
    """mu = 0 moves x to the lower bound and mu = 1 to the upper bound, for
    any eta_m (the step is -delta_1 and +delta_2 of the width)."""
    for eta in (0.0, 5.0, 20.0):
        for x in (0.1, 0.5, 0.9):
            assert oracle.pm_value(x, -2.0, 3.0, 0.0, eta) == pytest.approx(-2.0, abs=1e-12)
            assert oracle.pm_value(x, -2.0, 3.0, 1.0, eta) == pytest.approx(3.0, abs=1e-12)


def test_pm_linear_case():
    """eta_m = 0 (eta = 1): the step is 2 mu + (1 - 2 mu)(1 - delta_1) - 1
    below 0.5 and 1 - (2 - 2 mu + (2 mu - 1)(1 - delta_2)) above."""
    assert oracle.pm_value(0.3, 0.0, 1.0, 0.25, 0.0) == pytest.approx(0.15, abs=1e-15)
    assert oracle.pm_value(0.3, 0.0, 1.0, 0.75, 0.0) == pytest.approx(0.65, abs=1e-15)


def test_pm_is_monotone_in_mu_and_stays_in_bounds():
    mus = np.linspace(0.0, 1.0, 401)
    for x in (0.05, 0.5, 0.95):
        y = np.array([oracle.pm_value(x, 0.0, 1.0, mu, 20.0) for mu in mus])
        assert np.all(np.diff(y) >= -1e-15)
        assert y.min() >= -1e-12 and y.max() <= 1.0 + 1e-12


# ------------------------------------------------------------------ generation operators

def test_variation_without_crossover_or_mutation_copies_the_parents():
    X = wl.decision_vectors(50, 7, seed=3)
    off, par = oracle.variation(X, 0.0, 1.0, 50, seed=9, generation=2, p_c=0.0, p_m=0.0)
    assert np.array_equal(off[:25], X[par[:, 0]])
    assert np.array_equal(off[25:], X[par[:, 1]])


def test_variation_crossover_only_conserves_pair_sums():
    """With p_m = 0 each pair's two children sum to the parents' sum wherever
    neither child was clipped to the bounds."""
    X = wl.decision_vectors(400, 12, seed=4)
    off, par = oracle.variation(X, 0.0, 1.0, 400, seed=5, generation=1, p_c=1.0, p_m=0.0)
    c1, c2 = off[:200].astype(np.float64), off[200:].astype(np.float64)
    xs = X[par[:, 0]].astype(np.float64) + X[par[:, 1]].astype(np.float64)
    inside = (c1 > 0) & (c1 < 1) & (c2 > 0) & (c2 < 1)
    assert inside.mean() > 0.9
    assert np.max(np.abs((c1 + c2 - xs)[inside])) < 4e-7       # two FP32 roundings of values <= 1
    assert not np.array_equal(off[:200], X[par[:, 0]])         # crossover did act


def test_variation_mutation_rate_and_bounds():
    """p_m = 1/D mutates about one variable per row; all values stay in [L, U]."""
    n, d = 4000, 10
    X = wl.decision_vectors(n, d, seed=6)
    base, par = oracle.variation(X, 0.0, 1.0, n, seed=7, generation=3, p_c=0.0, p_m=0.0)
    mut, par2 = oracle.variation(X, 0.0, 1.0, n, seed=7, generation=3, p_c=0.0)
    assert np.array_equal(par, par2)
    frac = np.mean(mut != base)
    sigma = math.sqrt(0.1 * 0.9 / (n * d))
    assert abs(frac - 0.1) < 5 * sigma
    assert mut.min() >= 0.0 and mut.max() <= 1.0


def test_variation_parents_are_uniform_and_streams_differ():
    n = 16
    X = wl.decision_vectors(n, 3, seed=1)
    _, par = oracle.variation(X, 0.0, 1.0, 40000, seed=11, generation=0)
    counts = np.bincount(par.reshape(-1), minlength=n)
    expected = par.size / n
    chi2 = float(np.sum((counts - expected) ** 2 / expected))
    assert chi2 < 50.0                                          # 15 d.o.f.: p ~ 1e-5
    _, par_b = oracle.variation(X, 0.0, 1.0, 40000, seed=11, generation=1)
    _, par_c = oracle.variation(X, 0.0, 1.0, 40000, seed=11, generation=0)
    assert np.array_equal(par, par_c) and not np.array_equal(par, par_b)


def test_variation_odd_offspring_count():
    X = wl.decision_vectors(9, 4, seed=2)
    off, par = oracle.variation(X, 0.0, 1.0, 9, seed=3, generation=0, p_c=0.0, p_m=0.0)
    assert par.shape == (5, 2)
    assert np.array_equal(off[:5], X[par[:, 0]]) and np.array_equal(off[5:], X[par[:4, 1]])


# ------------------------------------------------------------------ PBI

def test_pbi_on_the_direction_and_perpendicular_to_it():
    z = np.zeros(2, np.float32)
    assert oracle.pbi([2.0, 0.0], [1.0, 0.0], z, 5.0) == 2.0
    assert oracle.pbi([3.0, 4.0], [3.0, 4.0], z, 5.0) == pytest.approx(5.0, abs=1e-12)
    assert oracle.pbi([1.0, -1.0], [1.0, 1.0], z, 5.0) == pytest.approx(5.0 * math.sqrt(2.0), abs=1e-12)
    assert oracle.pbi([5.0, 4.0], [1.0, 0.0], [2.0, 1.0], 0.5) == pytest.approx(3.0 + 0.5 * 3.0, abs=1e-15)


def test_pbi_geometric_decomposition_and_scale_invariance():
    """f - z = a w_hat + b u with a >= 0 and u a unit vector orthogonal to w
    gives g = a + theta |b|; g does not change when w is scaled. (a >= 0 is
    the method's domain: f >= z_min and w >= 0.)"""
    rng = np.random.default_rng(8)
    for m in (2, 3, 5, 8):
        for _ in range(50):
            w = rng.random(m) + 0.05
            wh = w / np.linalg.norm(w)
            u = rng.standard_normal(m)
            u -= (u @ wh) * wh
            u /= np.linalg.norm(u)
            a, b, theta = rng.uniform(0.01, 2), rng.uniform(0, 2), rng.uniform(0, 10)
            z = rng.random(m)
            f = z + a * wh + b * u
            # build exactly representable FP32 inputs, then recompute a, b from them
            f32, w32, z32 = f.astype(np.float32), w.astype(np.float32), z.astype(np.float32)
            e = f32.astype(np.float64) - z32.astype(np.float64)
            wh32 = w32.astype(np.float64) / np.linalg.norm(w32.astype(np.float64))
            a32 = e @ wh32
            b32 = np.linalg.norm(e - a32 * wh32)
            g = oracle.pbi(f32, w32, z32, theta)
            assert a32 > 0
            assert g == pytest.approx(a32 + theta * b32, rel=1e-9, abs=1e-9)
            assert oracle.pbi(f32, (4.0 * w32).astype(np.float32), z32, theta) == pytest.approx(g, rel=1e-12)


# ------------------------------------------------------------------ TensorMOEA/D selection

def _g(f, w, z, theta=5.0):
    return oracle.pbi(f, w, z, theta)


def test_moead_worked_example():
    """n = 3, m = 2, z = 0, theta = 5, W = (1,0), (0,1), (1,1), T = 2.
    PBI: w = (1,0) gives f1 + 5 f2; w = (0,1) gives f2 + 5 f1; w = (1,1)
    gives (f1 + f2 + 5 |f1 - f2|) / sqrt 2.
    Current F1 = (1,3), (3,1), (2,2): own values 16, 16, 2.83.
    Offspring F2 = (0.5,4), (4,2), (1,1) with neighbours {0,2}, {1,2}, {2,0}:
    offspring 0 gives 20.5 at 0 and 15.6 at 2, offspring 1 gives 22 at 1 and
    11.3 at 2 (no replacement); offspring 2 gives 1.41 at 2 and 6 at 0 (both
    replace). So subproblems 0 and 2 take offspring 2 and 1 keeps its own;
    z stays 0 (every offspring objective is positive)."""
    X = np.arange(6, dtype=np.float32).reshape(3, 2)
    O = 10 + np.arange(6, dtype=np.float32).reshape(3, 2)
    F1 = np.array([[1, 3], [3, 1], [2, 2]], np.float32)
    F2 = np.array([[0.5, 4], [4, 2], [1, 1]], np.float32)
    W = np.array([[1, 0], [0, 1], [1, 1]], np.float32)
    I_nb = np.array([[0, 2], [1, 2], [2, 0]], np.int32)
    Xn, Fn, z, win = oracle.moead_select(X, F1, O, F2, np.zeros(2, np.float32), W, I_nb, 5.0)
    assert win.tolist() == [2, -1, 2]
    assert Fn.tolist() == [[1, 1], [3, 1], [1, 1]]
    assert np.array_equal(Xn, np.stack([O[2], X[1], O[2]]))
    assert z.tolist() == [0.0, 0.0]


def _moead_case(n, m, d, t, seed, h=None):
    rng = np.random.default_rng(seed)
    W = wl.das_dennis(h, m) if h else (rng.random((n, m)) + 0.05).astype(np.float32)
    n = W.shape[0]
    X = rng.random((n, d), dtype=np.float32)
    O = rng.random((n, d), dtype=np.float32)
    F1 = (rng.random((n, m)) + 0.1).astype(np.float32)
    F2 = (rng.random((n, m)) + 0.1).astype(np.float32)
    z = np.full(m, 0.2, np.float32)
    I_nb = wl.moead_neighbours(W, t)
    return X, F1, O, F2, z, W, I_nb


def test_moead_single_neighbour_is_the_better_of_two():
    """T = 1 (each offspring only competes for its own subproblem): the new
    solution of j is offspring j exactly when it has the lower PBI value."""
    X, F1, O, F2, z, W, _ = _moead_case(200, 3, 5, 1, seed=21)
    I_nb = np.arange(200, dtype=np.int32).reshape(-1, 1)
    Xn, Fn, zn, win = oracle.moead_select(X, F1, O, F2, z, W, I_nb, 5.0)
    zmin = np.minimum(z, F2.min(axis=0))
    assert np.array_equal(zn, zmin)
    for j in range(200):
        better = _g(F2[j], W[j], zmin) < _g(F1[j], W[j], zmin)
        assert win[j] == (j if better else -1)
        assert np.array_equal(Xn[j], O[j] if better else X[j])


def test_moead_disjoint_neighbourhoods_equal_the_sequential_original():
    """When every subproblem is in exactly one neighbourhood, Algorithm S.8
    matches Algorithm S.7 run one offspring at a time (with the ideal point
    already updated by all offspring): no subproblem sees two offspring."""
    n, m, d, t = 120, 3, 4, 4
    X, F1, O, F2, z, W, _ = _moead_case(n, m, d, t, seed=22)
    perm = np.random.default_rng(3).permutation(n).astype(np.int32)
    groups = perm.reshape(-1, t)                        # 30 disjoint neighbourhoods
    owner = np.repeat(np.arange(groups.shape[0]), t)
    I_nb = np.zeros((n, t), np.int32)
    I_nb[: groups.shape[0]] = groups                    # offspring 0..29 own the groups
    rest = np.arange(groups.shape[0], n)
    far = np.full((len(rest), m), 1e30, np.float32)     # the other offspring never win
    F2 = F2.copy()
    F2[rest] = far
    I_nb[rest] = groups[owner[: len(rest)] % groups.shape[0]]
    zmin = np.minimum(z, F2.min(axis=0))
    # Algorithm S.7, sequentially over the offspring, replacement on <=
    Xs, Fs = X.copy(), F1.copy()
    for i in range(n):
        for j in I_nb[i]:
            if _g(F2[i], W[j], zmin) <= _g(Fs[j], W[j], zmin):
                Xs[j], Fs[j] = O[i], F2[i]
    Xn, Fn, _, _ = oracle.moead_select(X, F1, O, F2, z, W, I_nb, 5.0)
    assert np.array_equal(Xn, Xs) and np.array_equal(Fn, Fs)


def test_moead_overlapping_neighbourhoods_take_the_best_candidate():
    """Each subproblem ends with the lowest PBI value among its current
    solution and every offspring that has it as a neighbour; a winning
    offspring always lists the subproblem in its neighbourhood."""
    X, F1, O, F2, z, W, I_nb = _moead_case(0, 3, 6, 10, seed=23, h=12)
    n = W.shape[0]
    Xn, Fn, zn, win = oracle.moead_select(X, F1, O, F2, z, W, I_nb, 5.0)
    members = [[] for _ in range(n)]
    for i in range(n):
        for j in set(I_nb[i].tolist()):
            members[j].append(i)
    replaced = 0
    for j in range(n):
        best = min([_g(F1[j], W[j], zn)] + [_g(F2[i], W[j], zn) for i in members[j]])
        assert _g(Fn[j], W[j], zn) == best
        if win[j] >= 0:
            replaced += 1
            assert win[j] in members[j]
            assert np.array_equal(Fn[j], F2[win[j]]) and np.array_equal(Xn[j], O[win[j]])
        else:
            assert np.array_equal(Fn[j], F1[j]) and np.array_equal(Xn[j], X[j])
    assert 0 < replaced < n


def test_moead_ties_follow_the_first_argmin():
    """An offspring equal to the current solution of its only neighbour j
    replaces it (H(0) = 1), but the column's argmin then meets the same
    value first at a position that kept F1[j] unless that offspring is
    position 0: the current solution stays for j > 0."""
    X, F1, O, F2, z, W, _ = _moead_case(6, 2, 3, 1, seed=24)
    I_nb = np.arange(6, dtype=np.int32).reshape(-1, 1)
    F2 = F1.copy()
    _, _, _, win = oracle.moead_select(X, F1, O, F2, np.zeros(2, np.float32), W, I_nb, 5.0)
    assert win.tolist() == [0, -1, -1, -1, -1, -1]


def test_moead_hopeless_offspring_change_nothing():
    X, F1, O, F2, z, W, I_nb = _moead_case(0, 3, 4, 8, seed=25, h=9)
    F2 = np.full_like(F2, 1e30)
    Xn, Fn, zn, win = oracle.moead_select(X, F1, O, F2, z, W, I_nb, 5.0)
    assert np.all(win == -1) and np.array_equal(Xn, X) and np.array_equal(Fn, F1)
    assert np.array_equal(zn, z)


def test_moead_rejects_bad_input():
    X, F1, O, F2, z, W, I_nb = _moead_case(20, 2, 3, 4, seed=26)
    bad = I_nb.copy()
    bad[3, 1] = 20
    with pytest.raises(oracle.OracleError):
        oracle.moead_select(X, F1, O, F2, z, W, bad)
    W0 = W.copy()
    W0[4] = 0.0
    with pytest.raises(oracle.OracleError):
        oracle.moead_select(X, F1, O, F2, z, W0, I_nb)


def test_moead_offspring_parents_come_from_the_neighbourhood():
    W = wl.das_dennis(12, 3)
    I_nb = wl.moead_neighbours(W, 6)
    X = wl.decision_vectors(W.shape[0], 8, seed=4)
    O, par = oracle.moead_offspring(X, 0.0, 1.0, I_nb, seed=5, generation=1)
    for i in range(W.shape[0]):
        assert par[i, 0] in I_nb[i] and par[i, 1] in I_nb[i]
    assert O.min() >= 0.0 and O.max() <= 1.0
    O0, par0 = oracle.moead_offspring(X, 0.0, 1.0, I_nb, seed=5, generation=1, p_m=0.0)
    same = par0[:, 0] == par0[:, 1]                              # SBX of a point with itself is the point
    assert same.any() and np.array_equal(O0[same], X[par0[same, 0]])


def test_neighbours_are_nearest_weights():
    W = wl.das_dennis(6, 3)
    I_nb = wl.moead_neighbours(W, 4)
    assert np.array_equal(I_nb[:, 0], np.arange(W.shape[0]))
    d = np.linalg.norm(W[:, None, :].astype(np.float64) - W[None, :, :].astype(np.float64), axis=2)
    for i in range(W.shape[0]):
        inside = d[i, I_nb[i]].max()
        outside = np.delete(d[i], I_nb[i]).min()
        assert inside <= outside


def test_fast_neighbours_equal_the_exhaustive_definition():
    for h, m, t in ((12, 3, 10), (30, 3, 20), (8, 5, 15), (4, 8, 30)):
        W = wl.das_dennis(h, m)
        assert np.array_equal(wl.moead_neighbours_fast(W, t), wl.moead_neighbours(W, t))


# ------------------------------------------------------------------ IGD

def test_igd_closed_forms():
    R = wl.reference_front(12, 3, "sphere")
    assert oracle.igd(R, R) == 0.0
    assert oracle.igd([[0.0, 1.0]], [[0.0, 0.0], [1.0, 0.0]]) == pytest.approx((1 + math.sqrt(2)) / 2, abs=1e-15)
    # every reference point's nearest population point is its own radial copy
    g = 0.01
    assert oracle.igd((1 + g) * R.astype(np.float64), R) == pytest.approx(g, rel=1e-6)
    np.testing.assert_allclose(np.linalg.norm(R.astype(np.float64), axis=1), 1.0, rtol=1e-7)
    L = wl.reference_front(10, 4, "linear")
    np.testing.assert_allclose(L.astype(np.float64).sum(axis=1), 0.5, rtol=1e-6)


def test_igd_never_grows_when_points_are_added():
    rng = np.random.default_rng(9)
    R = wl.reference_front(8, 3, "sphere")
    F = rng.random((30, 3), dtype=np.float32)
    G = np.concatenate([F, rng.random((10, 3), dtype=np.float32)])
    assert oracle.igd(G, R) <= oracle.igd(F, R)
