"""One-shot niche selection (Algorithm S.4 with Update-Rank, Algorithm S.6)
on the GPU against the oracle's mode 1: survivors and every intermediate bit
for bit, in the add, drop and exact-fit regimes, at full size and batched
together with the level-form mode."""
import numpy as np
import pytest
import torch

import oracle
from paper_2503_20286_gb300 import _binding as emo
from paper_2503_20286_gb300 import workloads as wl

from . import _gpu
from .test_oracle_pins import _empty_niche_case

pytestmark = pytest.mark.gpu

ONESHOT = emo.EMO_NICHE_ONESHOT


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


@pytest.mark.parametrize("idx", range(6))
@pytest.mark.parametrize("delta", [-3, 0, 3])
def test_oneshot_add_drop_exact_fit(idx, delta):
    F, R, seed, gen, nP, nL, nE0 = _empty_niche_case(idx)
    n_keep = nP + nE0 + delta
    if not (nP < n_keep <= nP + nL):
        pytest.skip("n_keep outside the last front")
    _gpu.compare_select(F, R, n_keep, seed, gen, mode=ONESHOT)


@pytest.mark.parametrize("case", range(8))
def test_oneshot_random_cases(case):
    rng = np.random.default_rng(1300 + case)
    m = int(rng.choice([2, 3, 4, 5, 8]))
    n2 = int(rng.choice([37, 500, 1100, 2049, 3333]))
    q = [None, 16.0][case % 2]
    F = wl.population(n2, m, m + 5, "linear" if case % 3 else "sphere", seed=61 + case, quantize=q)
    R = wl.das_dennis(wl.h_for_count(max(2, n2 // int(rng.choice([2, 8]))), m), m)
    n_keep = int(rng.integers(1, n2 + 1))
    _gpu.compare_select(F, R, n_keep, seed=int(rng.integers(0, 2 ** 63)), gen=int(rng.integers(0, 2 ** 40)),
                        mode=ONESHOT)


def test_oneshot_keep_whole_front_and_one():
    F = wl.population(1500, 3, 9, "sphere", seed=8)
    R = wl.das_dennis(20, 3)
    _gpu.compare_select(F, R, 1500, seed=1, mode=ONESHOT)
    _gpu.compare_select(F, R, 1, seed=1, mode=ONESHOT)


def test_oneshot_config1_full_size():
    p = wl.config(1)
    _gpu.compare_select(p.F, p.R, p.n_keep, p.seed, p.generation, mode=ONESHOT)


def test_oneshot_in_a_batch_with_the_level_form():
    dev = torch.device("cuda")
    items, ref = [], []
    for b in range(6):
        rng = np.random.default_rng(40 + b)
        m = int(rng.choice([2, 3, 5]))
        n2 = int(rng.integers(500, 3000)) // 2 * 2
        F = wl.population(n2, m, m + 9, "sphere" if b % 2 else "linear", seed=500 + b)
        R = wl.das_dennis(wl.h_for_count(n2 // 2, m), m)
        mode = b % 2
        s_or, _ = oracle.nsga3_select(F, R, n2 // 2, 11 + b, 3, mode=mode)
        ref.append(s_or)
        items.append({"F": torch.from_numpy(F).to(dev), "R": torch.from_numpy(R).to(dev), "n_keep": n2 // 2,
                      "seed": 11 + b, "generation": 3, "niche_mode": mode,
                      "survivors": torch.empty(n2 // 2, dtype=torch.int32, device=dev),
                      "info": torch.zeros(8, dtype=torch.int32, device=dev)})
    emo.emo_nsga3_select_batch(items)
    torch.cuda.synchronize()
    for it, s_or in zip(items, ref):
        assert int(it["info"][0]) == 0
        assert np.array_equal(it["survivors"].cpu().numpy(), s_or)
