"""Whole generations on the oracle: variation (Appendix S.I), stand-in
evaluation, and environmental selection (Algorithm S.1 / S.4 + S.6 for
NSGA-III, Algorithm S.8 for TensorMOEA/D). The loops must keep their
invariants and move the population towards the front (IGD falls)."""
import numpy as np
import pytest

import oracle
from paper_2503_20286_gb300 import workloads as wl


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _nsga3_run(mode, gens=12, n=92, m=3, d=7, shape="linear", seed=0x250320286):
    R = wl.das_dennis(12, m)
    front = wl.reference_front(30, m, shape)
    X = wl.decision_vectors(n, d, seed)
    F = wl.objectives_from_decisions(X, m, shape)
    igd = [oracle.igd(F, front)]
    for g in range(gens):
        O, _ = oracle.variation(X, 0.0, 1.0, n, seed, g)
        FO = wl.objectives_from_decisions(O, m, shape)
        XX = np.concatenate([X, O])
        FF = np.concatenate([F, FO])
        surv, info = oracle.nsga3_select(FF, R, n, seed, g, trace=False, mode=mode)
        assert surv.shape == (n,) and np.all(np.diff(surv) > 0)
        X, F = XX[surv], FF[surv]
        igd.append(oracle.igd(F, front))
    return igd


@pytest.mark.parametrize("mode", [oracle.NICHE_EXACT, oracle.NICHE_ONESHOT])
def test_nsga3_generations_approach_the_front(mode):
    igd = _nsga3_run(mode, gens=30)
    assert igd[-1] < 0.3 * igd[0]


def test_nsga3_sphere_generations_approach_the_front():
    igd = _nsga3_run(oracle.NICHE_EXACT, gens=8, n=100, d=12, shape="sphere")
    assert igd[-1] < igd[0]


def test_moead_generations_approach_the_front():
    m, d, shape, seed = 3, 7, "linear", 7
    W = wl.das_dennis(12, m)
    n = W.shape[0]
    I_nb = wl.moead_neighbours(W, 10)
    front = wl.reference_front(30, m, shape)
    X = wl.decision_vectors(n, d, seed)
    F = wl.objectives_from_decisions(X, m, shape)
    z = F.min(axis=0)
    igd0 = oracle.igd(F, front)
    for g in range(15):
        O, _ = oracle.moead_offspring(X, 0.0, 1.0, I_nb, seed, g)
        FO = wl.objectives_from_decisions(O, m, shape)
        z_before = z.copy()
        X, F, z, win = oracle.moead_select(X, F, O, FO, z, W, I_nb, 5.0)
        assert np.all(z <= z_before) and np.array_equal(z, np.minimum(z_before, FO.min(axis=0)))
        assert np.all(F >= z)                           # the PBI projection stays non-negative
    assert oracle.igd(F, front) < 0.5 * igd0
