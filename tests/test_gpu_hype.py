"""TensorHypE selection (Algorithms S.10, S.11) on the GPU against the
oracle: survivors and the contributions of front l bit for bit."""
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


def gpu_hype(F, v_ref, U, n_keep):
    dev = torch.device("cuda")
    Ft = torch.from_numpy(np.ascontiguousarray(F, np.float32)).to(dev)
    vt = torch.from_numpy(np.ascontiguousarray(v_ref, np.float32)).to(dev)
    Ut = torch.from_numpy(np.ascontiguousarray(U, np.float32)).to(dev)
    info = torch.full((8,), -7, dtype=torch.int32, device=dev)
    hv = torch.full((F.shape[0],), -1.0, dtype=torch.float64, device=dev)
    surv = emo.emo_hype_select(Ft, vt, Ut, n_keep, info=info, hv=hv)
    torch.cuda.synchronize()
    inf = dict(zip(("status", "last_rank", "n_before", "n_last"), info.cpu().tolist()[:4]))
    return surv.cpu().numpy(), hv.cpu().numpy(), inf


def compare(F, v_ref, U, n_keep):
    s_or, hv_or, l = oracle.hype_select(F, v_ref, U, n_keep)
    s_g, hv_g, info = gpu_hype(F, v_ref, U, n_keep)
    assert info["status"] == 0 and info["last_rank"] == l, info
    assert np.array_equal(hv_g, hv_or), np.flatnonzero(hv_g != hv_or)[:10]
    assert np.array_equal(s_g, s_or)


def test_hype_lattice_exclusive_volumes():
    F = np.array([[1, 3], [2, 2], [3, 1], [2, 3]], np.float32)
    u = (np.arange(30) + 0.5) / 30
    U = np.stack(np.meshgrid(u, u, indexing="ij"), -1).reshape(-1, 2).astype(np.float32)
    compare(F, np.array([4, 4], np.float32), U, 2)


@pytest.mark.parametrize("case", range(8))
def test_hype_random_cases(case):
    rng = np.random.default_rng(2000 + case)
    m = int(rng.choice([2, 3, 4, 6]))
    n2 = int(rng.choice([40, 700, 2049, 3000]))
    F = wl.population(n2, m, m + 5, "sphere" if case % 2 else "linear", seed=170 + case,
                      quantize=[None, 16.0][case % 2])
    s = int(rng.choice([1, 300, 2500]))
    U = rng.random((s, m)).astype(np.float32)
    v_ref = (F.max(axis=0) * 1.1 + 0.01).astype(np.float32)
    compare(F, v_ref, U, int(rng.integers(1, n2 + 1)))


def test_hype_exactly_filled_fronts_and_keep_one():
    F = wl.population(1500, 3, 9, "sphere", seed=5)
    U = np.random.default_rng(3).random((800, 3)).astype(np.float32)
    v_ref = np.full(3, 3.0, np.float32)
    r = oracle.nd_sort_deb(F)
    compare(F, v_ref, U, int((r <= 2).sum()))   # k = 0: front 2 is kept whole
    compare(F, v_ref, U, 1)


def test_hype_larger_population():
    F = wl.population(20000, 3, 12, "sphere", seed=44)
    U = np.random.default_rng(9).random((3000, 3)).astype(np.float32)
    compare(F, np.full(3, 2.5, np.float32), U, 10000)


@pytest.mark.parametrize("m,quant", [(5, 8.0), (8, None), (12, 4.0), (16, None)])
def test_hype_many_objectives_and_ties(m, quant):
    """Prefix sets with checkpoints every 2 to 16 columns (m >= 5), several
    column blocks and, on a coarse grid, samples that tie point values in
    single objectives (weak dominance: ties count)."""
    F = wl.population(2600, m, m + 4, "sphere", seed=300 + m, quantize=quant)
    rng = np.random.default_rng(m)
    U = rng.random((1500, m)).astype(np.float32)
    v_ref = (F.max(axis=0) * 1.05 + 0.02).astype(np.float32)
    if quant:  # samples on the same grid as the points
        lo = F.min(axis=0)
        S_grid = np.round((lo + U * (v_ref - lo)) * quant) / quant
        U = np.clip((S_grid - lo) / (v_ref - lo), 0.0, np.nextafter(np.float32(1), np.float32(0))).astype(np.float32)
    compare(F, v_ref, U, 1300)
