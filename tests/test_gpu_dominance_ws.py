"""The caller-order dominance matrix through prefix sets (emo_dominance_ws)
against Listing 1 (the oracle's pairwise definition, all <= and some <) and
against the direct kernel of emo_dominance: bits and dominator counts equal,
with duplicated points, -0 and +0, padded and odd leading dimensions, ragged
tails and every objective count it serves (m <= 5; larger m runs the direct
kernel)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_2503_20286_gb300 import _binding as emo  # noqa: E402
from paper_2503_20286_gb300 import build as _build  # noqa: E402
from paper_2503_20286_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    emo.lib()


def _run(F, ld=None):
    n2 = F.shape[0]
    Ft = torch.from_numpy(np.ascontiguousarray(F, np.float32)).cuda()
    D = None
    if ld is not None:
        D = torch.full((n2, ld), -1, dtype=torch.int32, device="cuda")
    D, c = emo.emo_dominance_ws(Ft, D=D)
    torch.cuda.synchronize()
    return D.cpu().numpy().view(np.uint32), c.cpu().numpy()


@pytest.mark.parametrize("n2,m,q", [(1, 2, None), (33, 3, None), (1025, 3, 8.0), (2100, 2, 16.0),
                                    (3001, 4, None), (2600, 5, 4.0), (1500, 6, 8.0)])
def test_matches_the_pairwise_definition(n2, m, q):
    F = wl.population(n2, m, m + 5, "sphere", seed=5000 + n2 + m, quantize=q)
    D, c = _run(F)
    assert np.array_equal(D, oracle.dominance_bits(F))
    assert np.array_equal(c, oracle.domination_counts(F))


def test_duplicates_and_signed_zeros():
    F = np.array([[0.0, 1.0, 2.0], [-0.0, 1.0, 2.0], [0.0, 1.0, 2.0], [0.5, 1.0, 2.0], [-0.0, 0.5, 2.0],
                  [1.0, 1.0, 3.0]], dtype=np.float32)
    F = np.concatenate([F] * 300)  # long runs of identical points across column blocks
    D, c = _run(F)
    assert np.array_equal(D, oracle.dominance_bits(F))
    assert np.array_equal(c, oracle.domination_counts(F))


@pytest.mark.parametrize("extra", [1, 45])
def test_padded_and_odd_leading_dimension(extra):
    F = wl.population(1500, 3, 8, "linear", seed=6)
    ld = (1500 + 31) // 32 + extra
    D, _ = _run(F, ld=ld)
    assert np.array_equal(D, oracle.dominance_bits(F, ld=ld))


def test_equals_the_direct_kernel_at_20000():
    F = wl.config(1).F
    Ft = torch.from_numpy(F).cuda()
    D1, c1 = emo.emo_dominance(Ft)
    D2, c2 = emo.emo_dominance_ws(Ft)
    torch.cuda.synchronize()
    assert torch.equal(D1, D2) and torch.equal(c1, c2)
