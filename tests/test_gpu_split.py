"""The kernels of the split of one population over GPUs, and the split
exchange itself with its ranks driven in one process on this GPU
(paper_2503_20286_gb300.split.run_virtual): the column share of the
dominance matrix, one peeling step, the selection from given ranks, the
association of a column range (references, FP64 distances and niche counts
of P, Section IV-A) and the niching from a gathered association are checked
against the oracle element by element, inconsistent gathered data is
reported, then whole split selections for 1, 2 and 3 ranks give the
oracle's ranks and survivors."""
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


def _assoc_case(ci):
    if ci == 0:
        p = wl.config(1)
        return p.F, p.R, p.n_keep
    if ci == 1:  # ties on a 1/8 grid, five objectives
        return wl.population(2500, 5, 14, "linear", seed=61, quantize=8.0), wl.das_dennis(5, 5), 1200
    F = wl.population(3000, 3, 9, "sphere", seed=63)  # one point ideal on two axes: nadir fallback
    return wl.ideal_corner_case(F), wl.das_dennis(12, 3), 1500


@pytest.mark.parametrize("ci", range(3))
def test_association_of_column_ranges_equals_the_oracle(ci):
    F, R, n_keep = _assoc_case(ci)
    n2 = F.shape[0]
    ranks = oracle.nd_sort_deb(F).astype(np.int32)
    _, t = oracle.nsga3_select(F, R, n_keep, 0, 0)
    l = t["last_rank"]
    ranks[ranks > l] = emo.EMO_NOT_RANKED
    cuts = sorted({0, n2, 1024, min(n2, 2048), n2 // 3, n2 // 3 + 1})
    rho_sum = np.zeros(R.shape[0], np.int64)
    for lo, hi in zip(cuts, cuts[1:]):
        info = torch.zeros(8, dtype=torch.int32, device="cuda")
        pi, dist, rho = emo.emo_nsga3_associate_range(_dev(F), _dev(R), n_keep, _dev(ranks), lo, hi, info=info)
        torch.cuda.synchronize()
        inf = info.cpu().numpy()
        assert inf[0] == 0 and inf[1] == l and inf[2] == t["n_before"] and inf[3] == t["n_last"]
        assert inf[4] == t["fallback"]
        assert np.array_equal(pi.cpu().numpy(), t["pi"][lo:hi])
        assert np.array_equal(dist.cpu().numpy(), t["dist"][lo:hi], equal_nan=True)
        P = np.flatnonzero(t["rank"][lo:hi] < l)
        assert np.array_equal(rho.cpu().numpy(), np.bincount(t["pi"][lo:hi][P], minlength=R.shape[0]))
        rho_sum += rho.cpu().numpy()
    assert np.array_equal(rho_sum, t["rho"])


def test_association_of_an_empty_range():
    F, R, n_keep = _assoc_case(1)
    ranks = oracle.nd_sort_deb(F).astype(np.int32)
    pi, dist, rho = emo.emo_nsga3_associate_range(_dev(F), _dev(R), n_keep, _dev(ranks), 1024, 1024)
    torch.cuda.synchronize()
    assert pi.numel() == 0 and dist.numel() == 0 and int(rho.sum().item()) == 0


def _given(F, R, n_keep, seed, gen, mode):
    surv, t = oracle.nsga3_select(F, R, n_keep, seed, gen, mode=mode)
    l = t["last_rank"]
    ranks = t["rank"].astype(np.int32)
    ranks[ranks > l] = emo.EMO_NOT_RANKED
    L = np.flatnonzero(t["rank"] == l).astype(np.int32)
    return surv, t, ranks, L


@pytest.mark.parametrize("mode", [oracle.NICHE_EXACT, oracle.NICHE_ONESHOT])
@pytest.mark.parametrize("ci", range(3))
def test_niching_from_a_given_association_equals_the_oracle(ci, mode):
    F, R, n_keep = _assoc_case(ci)
    surv, t, ranks, L = _given(F, R, n_keep, 11 + ci, 4, mode)
    info = torch.zeros(8, dtype=torch.int32, device="cuda")
    s = emo.emo_nsga3_niche_given(F.shape[0], R.shape[0], n_keep, 11 + ci, 4, _dev(ranks), _dev(t["rho"]), _dev(L),
                                  _dev(t["pi"][L]), _dev(t["dist"][L]), niche_mode=mode, info=info)
    torch.cuda.synchronize()
    inf = info.cpu().numpy()
    assert inf[0] == 0 and inf[1] == t["last_rank"] and inf[3] == L.size
    assert np.array_equal(s.cpu().numpy(), surv)
    if mode == oracle.NICHE_EXACT and n_keep - t["n_before"] < t["n_last"]:  # niching chose
        assert inf[7] == t["n_levels"]


@pytest.mark.parametrize("fault", ["drop_member", "unordered", "rho_sum", "pi_range", "negative_dist", "not_last"])
def test_inconsistent_gathered_association_is_reported(fault):
    F, R, n_keep = _assoc_case(0)
    _, t, ranks, L = _given(F, R, n_keep, 3, 0, oracle.NICHE_EXACT)
    rho = t["rho"].astype(np.int32).copy()
    last, lpi, ld = L.copy(), t["pi"][L].astype(np.int32), t["dist"][L].copy()
    assert L.size >= 2
    if fault == "drop_member":
        last, lpi, ld = last[1:], lpi[1:], ld[1:]
    elif fault == "unordered":
        last[[0, 1]] = last[[1, 0]]
    elif fault == "rho_sum":
        rho[0] += 1
    elif fault == "pi_range":
        lpi[0] = R.shape[0]
    elif fault == "negative_dist":
        ld[0] = -1.0
    else:  # a point of P given as a member of front l
        last[0] = np.flatnonzero(t["rank"] < t["last_rank"])[0]
        last.sort()
    info = torch.zeros(8, dtype=torch.int32, device="cuda")
    emo.emo_nsga3_niche_given(F.shape[0], R.shape[0], n_keep, 3, 0, _dev(ranks), _dev(rho), _dev(last), _dev(lpi),
                              _dev(ld), info=info)
    torch.cuda.synchronize()
    assert int(info[0].item()) == 1
    emo.emo_get_last_device_status()  # clear the sticky word for later tests
