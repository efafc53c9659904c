"""GPU parity at the five workloads' full sizes.

* many-objective population with ties (2N=100,000, M=8, 1/64 grid, 156
  two-layer directions) and its degenerate-intercept variant: bit-exact
  against the oracle, intermediates included;
* 64 uneven populations in one batched call: identical to 64 plain calls
  and, for the populations the oracle finishes quickly, to the oracle;
* 2N=400,000 (the benchmark workload): properties that characterise the
  result at any size, checked on samples -- every sampled rank equals one
  plus the largest rank among its dominators, the ideal point equals the
  column minima, P is kept, extra survivors come from the last front, the
  association is the FP64 nearest reference line of the normalised point.
"""
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


def test_config2_many_objectives_with_ties():
    p = wl.config(2)
    F = p.F
    dup = 1.0 - len(np.unique(F, axis=0)) / F.shape[0]
    assert dup > 0.0  # the 1/64 grid creates duplicated points
    _gpu.compare_select(F, p.R, p.n_keep, p.seed, p.generation)


def test_config2_degenerate_extreme_point_fallback():
    p = wl.config(2)
    F = wl.ideal_corner_case(p.F)
    info, t = _gpu.compare_select(F, p.R, p.n_keep, p.seed, p.generation)
    assert t["fallback"] == 1 and info["fallback_used"] == 1


def _batch(probs):
    dev = torch.device("cuda")
    items = []
    for b, p in enumerate(probs):
        items.append({"F": torch.from_numpy(p.F).to(dev), "R": torch.from_numpy(p.R).to(dev),
                      "n_keep": p.n_keep, "seed": p.seed, "generation": p.generation,
                      "survivors": torch.empty(p.n_keep, dtype=torch.int32, device=dev),
                      "info": torch.zeros(8, dtype=torch.int32, device=dev)})
    return items


def test_config3_batch_equals_plain_and_oracle():
    probs = wl.config(3)
    items = _batch(probs)
    ws = emo.emo_nsga3_select_batch(items)
    torch.cuda.synchronize()
    assert emo.emo_workspace_status(ws) == 0
    checked = 0
    for p, it in zip(probs, items):
        info = it["info"].cpu().numpy()
        assert info[0] == 0, (p.name, info)
        got = it["survivors"].cpu().numpy()
        plain, pinfo, _ = _gpu.gpu_select(p.F, p.R, p.n_keep, p.seed, p.generation, debug=False)
        assert np.array_equal(got, plain), p.name
        if p.n2 <= 6000:
            ref, _ = oracle.nsga3_select(p.F, p.R, p.n_keep, p.seed, p.generation, trace=False)
            assert np.array_equal(got, ref), p.name
            checked += 1
    assert checked >= 5


def test_config3_batch_graph_replay_matches():
    """The batched call captured in a CUDA graph replays to the same survivors."""
    probs = wl.config(3)[:16]
    items = _batch(probs)
    ws = torch.empty(emo.emo_batch_workspace_size(items), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        emo.emo_nsga3_select_batch(items, ws=ws, stream=s)  # warm-up outside capture
    s.synchronize()
    ref = [it["survivors"].clone() for it in items]
    for it in items:
        it["survivors"].fill_(-1)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        emo.emo_nsga3_select_batch(items, ws=ws, stream=s)
    g.replay()
    torch.cuda.synchronize()
    for r, it in zip(ref, items):
        assert torch.equal(r, it["survivors"])


def test_config4_full_size_properties():
    p = wl.config(4)
    F, R = p.F, p.R
    n2 = F.shape[0]
    s, info, g = _gpu.gpu_select(F, R, p.n_keep, p.seed, p.generation, debug=True)
    assert info["status"] == 0
    l = info["last_rank"]
    rank = g["rank"]
    nP, nL = info["n_before"], info["n_last"]
    assert (rank < l).sum() == nP and (rank == l).sum() == nL
    assert nP < p.n_keep <= nP + nL
    assert len(s) == p.n_keep and np.all(np.diff(s) > 0)
    P = np.flatnonzero(rank < l)
    assert np.all(np.isin(P, s))
    extra = np.setdiff1d(s, P)
    assert np.all(rank[extra] == l) and len(extra) == p.n_keep - nP
    # ideal point: column minima of the population (attained in front 0)
    assert np.array_equal(g["z"], F.min(axis=0))
    # ranks: rank(i) = 1 + max rank of its dominators (0 without dominators)
    rng = np.random.default_rng(5)
    F64 = F.astype(np.float64)
    for i in rng.choice(n2, 150, replace=False):
        dom = np.all(F64 <= F64[i], axis=1) & np.any(F64 < F64[i], axis=1)
        rd = rank[dom]
        if rank[i] == emo.EMO_NOT_RANKED:
            assert dom.any() and (rd >= l).any()
        else:
            assert np.all(rd < rank[i])
            assert rank[i] == (rd.max() + 1 if dom.any() else 0)
    # association of sampled S points: nearest line in FP64 to the
    # normalised point (GPU normalisation, reference formula)
    S = np.flatnonzero(rank <= l)
    R64 = R.astype(np.float64)
    rr = (R64 * R64).sum(1)
    for i in rng.choice(S, 100, replace=False):
        fn = (F64[i] - g["z"].astype(np.float64)) / g["a"]
        t = (R64 @ fn) / rr
        d2 = ((fn[None, :] - t[:, None] * R64) ** 2).sum(1)
        j = int(np.argmin(d2))
        assert g["pi"][i] == j or np.isclose(d2[g["pi"][i]], d2[j], rtol=1e-12, atol=0), (i, g["pi"][i], j)
    np.testing.assert_allclose(g["fnorm"][S[:1000]], ((F64[S[:1000]] - g["z"]) / g["a"]), rtol=1e-5)


def _sha(a) -> str:
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def test_config4_bit_exact_against_oracle_fixture():
    """2N = 400,000 (the benchmark workload) against the oracle's fixture
    (tests/golden/make_config4_golden.py, written by the all-core oracle):
    survivors and ranks of S element by element, z, extreme points and FP64
    intercepts exactly, pi and the FP64 distances over S by SHA-256 (and per
    chunk, to locate a difference), the sampled pi / distances exactly, the
    normalised objectives within 1e-5 relative of FP64."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "config4_oracle.npz")
    gold = np.load(path)
    p = wl.config(4)
    assert _sha(p.F.astype("<f4")) == str(gold["F_sha256"]), "the generator produced a different population"
    assert _sha(p.R.astype("<f4")) == str(gold["R_sha256"])
    s, info, g = _gpu.gpu_select(p.F, p.R, p.n_keep, p.seed, p.generation, debug=True)
    assert info["status"] == 0
    n2 = p.n2
    assert info["last_rank"] == int(gold["last_rank"])
    assert info["n_before"] == int(gold["n_before"]) and info["n_last"] == int(gold["n_last"])
    assert info["fallback_used"] == int(gold["fallback"])
    mask = np.unpackbits(gold["survivor_mask"], count=n2, bitorder="little").astype(bool)
    ref_surv = np.flatnonzero(mask)
    assert np.array_equal(s, ref_surv), (np.setdiff1d(s, ref_surv)[:10], np.setdiff1d(ref_surv, s)[:10])
    rank_u8 = gold["rank_u8"]
    S = np.flatnonzero(rank_u8 != 255)
    assert np.array_equal(g["rank"][S], rank_u8[S].astype(np.int32))
    assert np.all(g["rank"][rank_u8 == 255] == emo.EMO_NOT_RANKED)
    assert np.array_equal(g["z"].astype(np.float64), gold["z"])
    assert np.array_equal(g["extreme"], gold["extreme"])
    assert np.array_equal(g["a"], gold["a"])
    si = gold["sample_index"]
    assert np.array_equal(g["pi"][si], gold["sample_pi"])
    assert np.array_equal(g["dist"][si], gold["sample_dist"])
    pi_S, dist_S = g["pi"][S].astype("<i4"), g["dist"][S].astype("<f8")
    if _sha(pi_S) != str(gold["pi_sha256"]) or _sha(dist_S) != str(gold["dist_sha256"]):
        bad = [c for c, (a, b, ga, gb) in enumerate(zip(np.array_split(pi_S, 64), np.array_split(dist_S, 64),
                                                        gold["pi_chunk_sha256"], gold["dist_chunk_sha256"]))
               if _sha(a) != str(ga) or _sha(b) != str(gb)]
        raise AssertionError(f"pi / FP64 distances differ from the oracle in chunks {bad} of S (64 chunks)")
    assert _sha(g["rho"].astype("<i4")) == str(gold["rho_sha256"])
    fn64 = (p.F[S].astype(np.float64) - gold["z"]) / gold["a"]
    np.testing.assert_allclose(g["fnorm"][S], fn64, rtol=1e-5, atol=0)
