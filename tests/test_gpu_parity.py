"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs, element by element. Sizes span several 32-row and
1024-column tiles and a ragged tail; edge cases cover one point, keeping
everything, duplicates, a total order, a single front, two objectives, one
reference, and the degenerate-intercept fallback."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_2503_20286_gb300 import _binding as emo  # noqa: E402
from paper_2503_20286_gb300 import build as _build  # noqa: E402
from paper_2503_20286_gb300 import workloads as wl  # noqa: E402
from tests import _gpu  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    emo.lib()


# ------------------------------------------------------------ dominance
@pytest.mark.parametrize("n2,m", [(1, 2), (31, 3), (33, 2), (1025, 3), (2100, 5), (3001, 8), (700, 16)])
def test_dominance_bits_and_counts(n2, m):
    F = wl.population(n2, m, m + 5, "sphere", seed=1000 + n2 + m)
    F = (np.round(F * 16) / 16).astype(np.float32)  # ties and duplicates
    D, c = _gpu.gpu_dominance(F)
    ref = oracle.dominance_bits(F)
    assert np.array_equal(D, ref)
    assert np.array_equal(c, oracle.domination_counts(F))


def test_dominance_padded_leading_dimension():
    F = wl.population(1500, 3, 8, "linear", seed=5)
    ld = (1500 + 31) // 32 + 45
    D, c = _gpu.gpu_dominance(F, ld=ld)
    assert np.array_equal(D, oracle.dominance_bits(F, ld=ld))


def test_dominance_negative_zero_equals_zero():
    F = np.array([[0.0, 1.0], [-0.0, 1.0], [0.0, 2.0], [-0.0, 0.5]], dtype=np.float32)
    D, _ = _gpu.gpu_dominance(F)
    assert np.array_equal(D, oracle.dominance_bits(F))


# ------------------------------------------------------------ ranking
@pytest.mark.parametrize("n2,m,shape,q", [(2, 2, "sphere", 0), (33, 3, "linear", 0), (1500, 2, "sphere", 0),
                                          (3001, 3, "sphere", 0), (4100, 5, "linear", 8), (2500, 8, "sphere", 16)])
def test_nd_rank_all_fronts(n2, m, shape, q):
    F = wl.population(n2, m, m + 6, shape, seed=2000 + n2, quantize=q or None)
    r, last = _gpu.gpu_rank(F)
    ref = oracle.nd_sort_deb(F)
    assert np.array_equal(r, ref)
    assert last == ref.max()


@pytest.mark.parametrize("frac", [0.01, 0.3, 0.5, 1.0])
def test_nd_rank_stops_at_last_needed_front(frac):
    F = wl.population(3000, 3, 9, "sphere", seed=77)
    n_keep = max(1, int(frac * 3000))
    r, last = _gpu.gpu_rank(F, n_keep)
    ref = oracle.nd_sort_deb(F)
    l = np.sort(ref)[n_keep - 1]
    assert last == l
    assert np.array_equal(r[ref <= l], ref[ref <= l])
    assert np.all(r[ref > l] == emo.EMO_NOT_RANKED)


def test_fronts_larger_than_member_chunk():
    # fronts of 2000 to 9000 points: the peel stages the members of a front
    # in chunks of 4096, and new members of one column block found in later
    # chunks are appended after those of the earlier ones
    F = np.concatenate([wl.front_points(9000, 3, "sphere", seed=50 + i) + np.float32(0.3 * i)
                        for i in range(3)]).astype(np.float32)
    ref = oracle.nd_sort_deb(F)
    assert np.bincount(ref)[0] > 2 * 4096
    r, last = _gpu.gpu_rank(F)
    assert np.array_equal(r, ref) and last == ref.max()
    _gpu.compare_select(F, wl.das_dennis(30, 3), 20000, seed=6)


def test_nd_rank_total_order_many_fronts():
    t = np.arange(1200, dtype=np.float32)[::-1].copy()
    F = np.stack([t, t * 2, t + 1], axis=1)          # one point per front
    r, last = _gpu.gpu_rank(F)
    assert np.array_equal(r, oracle.nd_sort_deb(F))
    assert last == 1199


# ------------------------------------------------------------ selection
def test_select_config0_matches_oracle():
    p = wl.config(0)
    _gpu.compare_select(p.F, p.R, p.n_keep, p.seed, p.generation)


@pytest.mark.parametrize("case", range(10))
def test_select_random_cases(case):
    rng = np.random.default_rng(900 + case)
    m = int(rng.choice([2, 3, 4, 5, 8]))
    n2 = int(rng.choice([37, 500, 1100, 2049, 3333]))
    shape = "linear" if case % 2 else "sphere"
    q = [None, None, 8.0, 32.0][case % 4]
    F = wl.population(n2, m, m + 5, shape, seed=31 + case, quantize=q)
    H = {2: 40, 3: 12, 4: 7, 5: 5, 8: 3}[m]
    R = wl.das_dennis(H, m)
    n_keep = int(rng.integers(1, n2 + 1))
    _gpu.compare_select(F, R, n_keep, seed=int(rng.integers(0, 2 ** 63)), gen=int(rng.integers(0, 2 ** 40)))


@pytest.mark.parametrize("m", [2, 3, 6, 16])
def test_select_objective_counts(m):
    F = wl.population(1800, m, m + 4, "sphere", seed=400 + m)
    R = wl.das_dennis({2: 99, 3: 13, 6: 4, 16: 2}[m], m)
    _gpu.compare_select(F, R, 900, seed=m, gen=3)


def test_select_keep_everything_and_keep_one():
    F = wl.population(1300, 3, 9, "linear", seed=8)
    R = wl.das_dennis(10, 3)
    _gpu.compare_select(F, R, 1300, seed=1)
    _gpu.compare_select(F, R, 1, seed=1)


def test_select_exactly_filled_fronts():
    F = wl.population(2000, 3, 9, "sphere", seed=12)
    r = oracle.nd_sort_deb(F)
    n_keep = int((r <= 4).sum())
    info, t = _gpu.compare_select(F, wl.das_dennis(12, 3), n_keep, seed=2)
    assert t["last_rank"] == 4 and t["n_before"] + t["n_last"] == n_keep


@pytest.mark.parametrize("n2,m,run", [(3000, 3, 3), (3000, 3, 40), (3000, 3, 700), (3000, 3, 3000),
                                       (10000, 3, 9000), (6000, 8, 1500), (6000, 8, 5000)])
def test_select_ties_in_the_first_objective(n2, m, run):
    # f_1 takes each value `run` times (runs of equal f_1 in the sorted
    # order): short runs are ordered in place, a run longer than 32 makes the
    # sort fall back to the full radix sort over every objective
    F = wl.population(n2, m, m + 6, "sphere", seed=31 + run)
    order = np.argsort(F[:, 0], kind="stable")
    F[order, 0] = (np.arange(n2) // run).astype(np.float32) / np.float32(1024)
    R = wl.das_dennis(30, 3) if m == 3 else wl.das_dennis(3, m)
    _gpu.compare_select(F, R, n2 * 7 // 15, seed=5)
    r, _ = _gpu.gpu_rank(F)
    assert np.array_equal(r, oracle.nd_sort_deb(F))


def test_select_all_duplicates():
    F = np.tile(np.array([[0.25, 0.5, 0.125]], dtype=np.float32), (700, 1))
    _gpu.compare_select(F, wl.das_dennis(6, 3), 300, seed=3)


def test_select_single_front():
    F = wl.front_points(2500, 3, "sphere", seed=21)
    _gpu.compare_select(F, wl.das_dennis(20, 3), 1200, seed=4, gen=9)


def test_select_total_order():
    t = np.linspace(1.0, 2.0, 900).astype(np.float32)
    F = np.stack([t, t * t, t + 0.5], axis=1)
    _gpu.compare_select(F, wl.das_dennis(5, 3), 450, seed=5)


def test_select_one_reference():
    F = wl.population(1000, 3, 9, "sphere", seed=22)
    _gpu.compare_select(F, np.array([[1.0, 1.0, 1.0]], np.float32), 500, seed=6)


def test_select_degenerate_intercepts_use_nadir():
    F = wl.ideal_corner_case(wl.population(3000, 5, 14, "sphere", seed=23))
    info, t = _gpu.compare_select(F, wl.das_dennis(5, 5), 1500, seed=7)
    assert t["fallback"] == 1 and info["fallback_used"] == 1


def test_select_same_seed_same_survivors_other_generation_differs():
    F = wl.population(4000, 3, 9, "sphere", seed=24)
    R = wl.das_dennis(30, 3)
    a, _, _ = _gpu.gpu_select(F, R, 2000, seed=11, gen=1, debug=False)
    b, _, _ = _gpu.gpu_select(F, R, 2000, seed=11, gen=1, debug=False)
    assert np.array_equal(a, b)
    # the random niching choices are keyed by the generation
    c, _, _ = _gpu.gpu_select(F, R, 2000, seed=11, gen=2, debug=False)
    assert np.array_equal(c, oracle.nsga3_select(F, R, 2000, 11, 2)[0])
    assert not np.array_equal(a, c)


def test_select_config1_full_size():
    p = wl.config(1)
    _gpu.compare_select(p.F, p.R, p.n_keep, p.seed, p.generation)


# ------------------------------------------------------------ failure detection
def test_nonfinite_objective_reported_on_device():
    F = wl.population(600, 3, 9, "sphere", seed=30)
    F[123, 1] = np.nan
    s, info, _ = _gpu.gpu_select(F, wl.das_dennis(8, 3), 300, seed=1, debug=False)
    assert info["status"] == 2


def test_zero_reference_rejected_on_device():
    F = wl.population(600, 3, 9, "sphere", seed=31)
    R = wl.das_dennis(8, 3)
    R[4] = 0.0
    s, info, _ = _gpu.gpu_select(F, R, 300, seed=1, debug=False)
    assert info["status"] == 2


def test_negative_reference_rejected_on_device():
    F = wl.population(600, 3, 9, "sphere", seed=33)
    R = wl.das_dennis(8, 3)
    R[5, 1] = -0.25
    s, info, _ = _gpu.gpu_select(F, R, 300, seed=1, debug=False)
    assert info["status"] == 1


@pytest.mark.parametrize("H", [300, 631])
def test_select_many_references_angular_index(H):
    """Large direction sets exercise the pruned angular scan of the
    association (and the exhaustive FP64 scan of near ties)."""
    F = wl.population(6000, 3, 12, "sphere", seed=40 + H)
    R = wl.das_dennis(H, 3)
    info, t = _gpu.compare_select(F, R, 3000, seed=H)


def test_bounded_wait_times_out_and_context_survives():
    """A one-cycle budget makes every cross-CTA barrier give up: the call
    reports EMO_ERR_TIMEOUT through its status word instead of hanging, and
    the next call with the normal budget is correct."""
    F = wl.population(5000, 3, 9, "sphere", seed=32)
    R = wl.das_dennis(12, 3)
    emo.emo_set_spin_budget(1)
    try:
        dev = torch.device("cuda")
        Ft, Rt = torch.from_numpy(F).to(dev), torch.from_numpy(R).to(dev)
        ws = torch.empty(emo.emo_workspace_size(2, 5000, 3, R.shape[0]), dtype=torch.uint8, device=dev)
        emo.emo_nsga3_select(Ft, Rt, 2500, 1, 0, ws=ws)
        assert emo.emo_workspace_status(ws) == 5
    finally:
        emo.emo_set_spin_budget(0)
    _gpu.compare_select(F, R, 2500, seed=1)


@pytest.mark.parametrize("n2,m,h,keep_frac,q", [(6000, 3, 3, 0.5, None), (12000, 5, 2, 0.6, 8.0),
                                                (4000, 8, 1, 0.45, 16.0), (20000, 3, 6, 0.9, None)])
def test_many_niching_levels(n2, m, h, keep_frac, q):
    """Few reference directions and a large last front: hundreds of niching
    levels, served one at a time and then in bulk (the same picks and level
    count as the oracle's loop of Algorithm S.1)."""
    F = wl.population(n2, m, m + 5, "sphere", seed=800 + n2 + m, quantize=q)
    R = wl.das_dennis(h, m)
    info, t = _gpu.compare_select(F, R, int(keep_frac * n2), seed=3, gen=5)
    assert t["n_levels"] > 20


@pytest.mark.parametrize("n_last,keep_last", [(10000, 6000), (9000, 8900)])
def test_niching_levels_beyond_one_window(n_last, keep_last):
    """Niche counts spread over more than 4096 levels with one reference
    serving a pick per level: front 0 spread over the line f1 + f2 = 0.8,
    front 1 (the last) a narrow band around the diagonal of f1 + f2 = 1, all
    nearest the diagonal direction (21 directions). The bulk niching serves
    a whole window of 4096 levels and goes on from the next level; picks and
    the level count equal the oracle's."""
    rng = np.random.default_rng(n_last)
    x = np.sort(rng.uniform(0.0, 0.8, 2000)).astype(np.float32)
    P = np.stack([x, np.float32(0.8) - x], axis=1)
    a = np.float32(0.49) + np.arange(n_last, dtype=np.float32) * np.float32(0.02 / n_last)
    Lf = np.stack([a, np.float32(1.0) - a], axis=1)
    F = np.ascontiguousarray(np.concatenate([P, Lf])[rng.permutation(2000 + n_last)])
    R = wl.das_dennis(20, 2)
    info, t = _gpu.compare_select(F, R, 2000 + keep_last, seed=7, gen=2)
    assert t["last_rank"] == 1 and t["n_last"] == n_last
    assert t["n_levels"] > 4096
