"""The two schedules of the front peeling (Algorithm S.3) give the same ranks
and survivors: one grid barrier per front, and the wavefront, where a column
block's task for front k starts once every lower block has finished front
k - 1. Each schedule runs with every CTA of the cooperative launch, a few
CTAs, and a single CTA; ranks and survivors are compared with the oracle
element by element (Deb's sort, Algorithm S.2, and the selection of
Algorithm S.1)."""
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

SCHEDULES = [(1, 0), (1, 5), (1, 1), (0, 1), (0, 0)]  # (wavefront, peel CTAs; 0 = every CTA)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    emo.lib()


@pytest.fixture(params=SCHEDULES, ids=[f"wave{w}-ctas{c}" for w, c in SCHEDULES])
def schedule(request, tmp_path):
    """Every (m, size) runs with the given peeling schedule (the other
    shapes at their defaults)."""
    wave, ctas = request.param
    major, minor = torch.cuda.get_device_capability()
    arch = 10 * major + minor
    lines = [f"{arch} {m} {b} 8 256 {ctas} 0 {wave}" for m in range(2, 17) for b in range(0, 22)]
    path = tmp_path / "schedule.txt"
    path.write_text("\n".join(lines) + "\n")
    emo.emo_autotune_reset()
    emo.emo_autotune(3, 1000, str(path))  # loads the file (the entry exists, nothing is timed)
    sh = emo.emo_launch_shape(3, 20000)
    assert sh["peel_wavefront"] == wave
    if ctas:
        assert sh["peel_ctas"] == ctas
    yield request.param
    emo.emo_autotune_reset()


@pytest.mark.parametrize("n2,m,shape,q", [(2, 2, "sphere", 0), (1500, 2, "sphere", 0), (3001, 3, "sphere", 0),
                                          (4100, 5, "linear", 8), (2500, 8, "sphere", 16)])
def test_all_fronts(schedule, n2, m, shape, q):
    F = wl.population(n2, m, m + 6, shape, seed=2000 + n2, quantize=q or None)
    r, last = _gpu.gpu_rank(F)
    ref = oracle.nd_sort_deb(F)
    assert np.array_equal(r, ref)
    assert last == ref.max()


@pytest.mark.parametrize("frac", [0.01, 0.5, 1.0])
def test_stops_at_last_needed_front(schedule, frac):
    F = wl.population(5000, 3, 9, "sphere", seed=78)
    n_keep = max(1, int(frac * 5000))
    r, last = _gpu.gpu_rank(F, n_keep)
    ref = oracle.nd_sort_deb(F)
    l = np.sort(ref)[n_keep - 1]
    assert last == l
    assert np.array_equal(r[ref <= l], ref[ref <= l])
    assert np.all(r[ref > l] == emo.EMO_NOT_RANKED)


def test_total_order_one_point_per_front(schedule):
    t = np.arange(2100, dtype=np.float32)[::-1].copy()
    F = np.stack([t, t * 2, t + 1], axis=1)
    r, last = _gpu.gpu_rank(F)
    assert np.array_equal(r, oracle.nd_sort_deb(F))
    assert last == 2099


def test_fronts_larger_than_member_chunk(schedule):
    F = np.concatenate([wl.front_points(9000, 3, "sphere", seed=50 + i) + np.float32(0.3 * i)
                        for i in range(3)]).astype(np.float32)
    ref = oracle.nd_sort_deb(F)
    assert np.bincount(ref)[0] > 8192
    r, last = _gpu.gpu_rank(F)
    assert np.array_equal(r, ref) and last == ref.max()


@pytest.mark.parametrize("case", range(4))
def test_selection(schedule, case):
    rng = np.random.default_rng(700 + case)
    m = [2, 3, 5, 3][case]
    n2 = [3333, 20000, 2049, 4097][case]
    F = wl.population(n2, m, m + 5, "linear" if case % 2 else "sphere", seed=31 + case,
                      quantize=[None, None, 8.0, 32.0][case])
    R = wl.das_dennis({2: 40, 3: 12, 5: 5}[m], m)
    _gpu.compare_select(F, R, int(rng.integers(1, n2 + 1)), seed=5 + case, gen=case)
