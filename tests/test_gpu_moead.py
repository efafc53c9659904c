"""TensorMOEA/D selection (Algorithm S.8) on the GPU against the FP64 oracle:
winners, X_next, F_next and z_min bit-exact (every PBI decision is taken in
FP64 with the same operations on both sides)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2503_20286_gb300 import _binding as emo
from paper_2503_20286_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _gpu(X, F1, O, F2, z, W, I_nb, theta=5.0, inplace=False):
    dev = torch.device("cuda")
    t = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in
         dict(X=X, F1=F1, O=O, F2=F2, z=z, W=W, I=I_nb).items()}
    kw = dict(X_next=t["X"], F_next=t["F1"]) if inplace else {}
    Xn, Fn, win, st = emo.emo_moead_select(t["X"], t["F1"], t["O"], t["F2"], t["z"], t["W"], t["I"], theta, **kw)
    torch.cuda.synchronize()
    return Xn.cpu().numpy(), Fn.cpu().numpy(), t["z"].cpu().numpy(), win.cpu().numpy(), int(st.item())


def _compare(X, F1, O, F2, z, W, I_nb, theta=5.0, inplace=False):
    ref = oracle.moead_select(X, F1, O, F2, z, W, I_nb, theta)
    got = _gpu(X, F1, O, F2, z, W, I_nb, theta, inplace)
    assert got[4] == 0
    assert np.array_equal(got[3], ref[3]), np.flatnonzero(got[3] != ref[3])[:10]
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    assert np.array_equal(got[2], ref[2])
    return ref


def _case(h, m, d, t, seed, shape="sphere"):
    W = wl.das_dennis(h, m)
    n = W.shape[0]
    X = wl.decision_vectors(n, d, seed, stream=1)
    O = wl.decision_vectors(n, d, seed, stream=2)
    F1 = wl.objectives_from_decisions(X, m, shape)
    F2 = wl.objectives_from_decisions(O, m, shape)
    return X, F1, O, F2, F1.min(axis=0), W, wl.moead_neighbours(W, t)


def test_worked_example():
    X = np.arange(6, dtype=np.float32).reshape(3, 2)
    O = 10 + np.arange(6, dtype=np.float32).reshape(3, 2)
    F1 = np.array([[1, 3], [3, 1], [2, 2]], np.float32)
    F2 = np.array([[0.5, 4], [4, 2], [1, 1]], np.float32)
    W = np.array([[1, 0], [0, 1], [1, 1]], np.float32)
    I_nb = np.array([[0, 2], [1, 2], [2, 0]], np.int32)
    ref = _compare(X, F1, O, F2, np.zeros(2, np.float32), W, I_nb)
    assert ref[3].tolist() == [2, -1, 2]


@pytest.mark.parametrize("h,m,d,t", [(12, 3, 6, 10), (40, 3, 30, 20), (8, 5, 33, 15), (3, 8, 7, 12)])
def test_matches_oracle(h, m, d, t):
    _compare(*_case(h, m, d, t, seed=100 + h))


def test_linear_front_and_small_theta():
    _compare(*_case(20, 3, 9, 8, seed=5, shape="linear"), theta=0.5)


def test_single_neighbour_and_exact_ties():
    X, F1, O, F2, z, W, _ = _case(12, 3, 5, 1, seed=6)
    I_nb = np.arange(W.shape[0], dtype=np.int32).reshape(-1, 1)
    _compare(X, F1, O, F2, z, W, I_nb)
    ref = _compare(X, F1, O, F1.copy(), np.zeros(3, np.float32), W, I_nb)   # every offspring ties
    assert ref[3][0] == 0 and np.all(ref[3][1:] == -1)


def test_repeated_neighbours_count_once():
    X, F1, O, F2, z, W, I_nb = _case(12, 3, 5, 6, seed=7)
    I_nb = I_nb.copy()
    I_nb[:, 3] = I_nb[:, 1]
    _compare(X, F1, O, F2, z, W, I_nb)


def test_in_place_update():
    args = _case(30, 3, 12, 20, seed=8)
    ref = oracle.moead_select(*args)
    got = _gpu(*args, inplace=True)
    assert got[4] == 0 and np.array_equal(got[3], ref[3])
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_generations_stay_identical():
    """Five generations fed with the oracle's offspring: the device and the
    oracle keep identical populations and ideal points."""
    m, d, seed = 3, 7, 9
    W = wl.das_dennis(20, m)
    I_nb = wl.moead_neighbours(W, 12)
    X = wl.decision_vectors(W.shape[0], d, seed)
    F = wl.objectives_from_decisions(X, m, "linear")
    z = F.min(axis=0)
    for g in range(5):
        O, _ = oracle.moead_offspring(X, 0.0, 1.0, I_nb, seed, g)
        FO = wl.objectives_from_decisions(O, m, "linear")
        Xr, Fr, zr, wr = oracle.moead_select(X, F, O, FO, z, W, I_nb, 5.0)
        Xg, Fg, zg, wg, st = _gpu(X, F, O, FO, z, W, I_nb)
        assert st == 0 and np.array_equal(wg, wr) and np.array_equal(Xg, Xr) and np.array_equal(zg, zr)
        X, F, z = Xr, Fr, zr


def test_device_status_for_bad_neighbours_and_non_finite_objectives():
    emo.emo_get_last_device_status()
    X, F1, O, F2, z, W, I_nb = _case(12, 3, 5, 4, seed=10)
    bad = I_nb.copy()
    bad[7, 2] = W.shape[0]                    # out of range: skipped before any use, reported
    assert _gpu(X, F1, O, F2, z, W, bad)[4] == 1
    assert emo.emo_get_last_device_status() == 1
    F2n = F2.copy()
    F2n[3, 1] = np.nan
    assert _gpu(X, F1, O, F2n, z, W, I_nb)[4] == 2
    assert emo.emo_get_last_device_status() == 2
    assert emo.emo_get_last_device_status() == 0


def test_bench_helper_runs_small():
    import bench
    dev = torch.device("cuda")
    flush = torch.empty(1 << 20, dtype=torch.uint8, device=dev)
    r = bench.moead_timing(emo, torch, dev, flush, torch.cuda.current_stream(), 2, h=30, m=3, d=12, t=20)
    assert r["subproblems"] == 496 and r["ms_per_step"] > 0 and 0 < r["replaced"] < 496
