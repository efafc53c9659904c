"""The kernels of the split of one population over GPUs, and the split
exchange itself with its ranks driven in one process on this GPU
(paper_2503_20286_gb300.split.run_virtual): the column share of the
dominance matrix, one peeling step and the selection from given ranks are
checked against the oracle, then whole split selections for 1, 2 and 3
ranks give the oracle's ranks and survivors."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_2503_20286_gb300 import _binding as emo  # noqa: E402
from paper_2503_20286_gb300 import build as _build  # noqa: E402
from paper_2503_20286_gb300 import split  # noqa: E402
from paper_2503_20286_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    emo.lib()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _bits(D, ncols):
    return np.unpackbits(np.ascontiguousarray(D).view(np.uint8), bitorder="little", axis=1)[:, :ncols]


@pytest.mark.parametrize("lo,hi", [(0, 2500), (0, 1024), (1024, 2500), (2048, 2049)])
def test_dominance_columns_match_the_oracle(lo, hi):
    F = wl.population(2500, 4, 10, "sphere", seed=81, quantize=16.0)
    D, c = emo.emo_dominance_cols(_dev(F), lo, hi)
    torch.cuda.synchronize()
    ref = _bits(oracle.dominance_bits(F), 2500)[:, lo:hi]
    assert np.array_equal(_bits(D.cpu().numpy(), hi - lo), ref)
    assert np.array_equal(c.cpu().numpy(), ref.sum(axis=0))
    words = D.cpu().numpy().view(np.uint32)
    assert np.all(_bits(words, words.shape[1] * 32)[:, hi - lo:] == 0)  # padding bits are zero


def test_one_peeling_step():
    F = wl.population(3000, 3, 9, "linear", seed=82)
    lo, hi = 1024, 3000
    D, c = emo.emo_dominance_cols(_dev(F), lo, hi)
    ranks = oracle.nd_sort_deb(F)
    front0 = np.flatnonzero(ranks == 0).astype(np.int32)
    flags = emo.emo_front_counts(D, hi - lo, _dev(front0), c)
    torch.cuda.synchronize()
    bits = _bits(oracle.dominance_bits(F), 3000)[:, lo:hi].astype(np.int64)
    counts = bits.sum(axis=0) - bits[front0].sum(axis=0)
    assert np.array_equal(c.cpu().numpy(), counts)
    expect = (ranks[lo:hi] == 1)
    assert np.array_equal(flags.cpu().numpy().astype(bool), expect)


@pytest.mark.parametrize("keep_all_fronts", [True, False])
def test_selection_from_given_ranks(keep_all_fronts):
    p = wl.config(1)
    ranks = oracle.nd_sort_deb(p.F).astype(np.int32)
    surv_ref, t = oracle.nsga3_select(p.F, p.R, p.n_keep, p.seed, 2)
    if not keep_all_fronts:
        ranks[ranks > t["last_rank"]] = emo.EMO_NOT_RANKED
    info = torch.zeros(8, dtype=torch.int32, device="cuda")
    s = emo.emo_nsga3_select_ranked(_dev(p.F), _dev(p.R), p.n_keep, p.seed, 2, _dev(ranks), info=info)
    torch.cuda.synchronize()
    inf = info.cpu().numpy()
    assert inf[0] == 0 and inf[1] == t["last_rank"] and inf[2] == t["n_before"] and inf[3] == t["n_last"]
    assert np.array_equal(s.cpu().numpy(), surv_ref)


def test_ranked_workspace_has_no_dominance_matrix():
    full = emo.emo_workspace_size(emo.EMO_OP_NSGA3_SELECT, 100000, 3, 100)
    ranked = emo.emo_workspace_size(emo.EMO_OP_SELECT_RANKED, 100000, 3, 100)
    assert 0 < ranked < full // 10


def test_selection_from_too_few_ranks_is_reported():
    p = wl.config(0)
    ranks = np.full(p.n2, emo.EMO_NOT_RANKED, np.int32)
    ranks[:10] = 0
    info = torch.zeros(8, dtype=torch.int32, device="cuda")
    emo.emo_nsga3_select_ranked(_dev(p.F), _dev(p.R), p.n_keep, 1, 0, _dev(ranks), info=info)
    torch.cuda.synchronize()
    assert int(info[0].item()) == 1
    emo.emo_get_last_device_status()  # clear the sticky word for later tests


@pytest.mark.parametrize("world", [1, 2, 3])
@pytest.mark.parametrize("ci", range(3))
def test_split_selection_equals_the_oracle(world, ci):
    cases = [(wl.config(1).F, wl.config(1).R, 10000, 5, 0),
             (wl.population(2500, 5, 14, "linear", seed=61, quantize=8.0), wl.das_dennis(5, 5), 1200, 7, 3),
             (wl.population(1500, 3, 9, "sphere", seed=62), wl.das_dennis(12, 3), 750, 9, 1)]
    F, R, n_keep, seed, gen = cases[ci]
    res = split.run_virtual(_dev(F), _dev(R), n_keep, seed, gen, split.GpuOps(), world)
    ref, t = oracle.nsga3_select(F, R, n_keep, seed, gen)
    l = t["last_rank"]
    for surv, info, ranks in res:
        torch.cuda.synchronize()
        r = ranks.cpu().numpy()
        assert np.array_equal(r[t["rank"] <= l], t["rank"][t["rank"] <= l])
        assert np.all(r[t["rank"] > l] == emo.EMO_NOT_RANKED)
        assert int(info[0].item()) == 0
        assert np.array_equal(surv.cpu().numpy(), ref)
