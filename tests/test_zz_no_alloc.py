"""The allocation-free selection entry point (emo_nsga3_select_noalloc).

Callers that cannot allocate device memory use the library's built-in
scratch instead of a workspace. This file is collected last so that a run
stopping at the first failure has already run every other test; it passes
both alone in a fresh process and after the others. Two calls in a row, on
different populations, check that the shared scratch carries nothing over
from the previous call: their survivors and info must equal those of
emo_nsga3_select with its own workspace (survivors are integers, compared
exactly, the tolerance of every survivor comparison in this suite).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2503_20286_gb300 import _binding as emo  # noqa: E402
from paper_2503_20286_gb300 import build as _build  # noqa: E402
from paper_2503_20286_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu


def _run_both(F, R, n_keep, seed, gen):
    dev = torch.device("cuda")
    Ft, Rt = torch.from_numpy(F).to(dev), torch.from_numpy(R).to(dev)
    s_ws = torch.empty(n_keep, dtype=torch.int32, device=dev)
    s_na = torch.full((n_keep,), -1, dtype=torch.int32, device=dev)
    i_ws = torch.zeros(8, dtype=torch.int32, device=dev)
    i_na = torch.full((8,), -1, dtype=torch.int32, device=dev)
    emo.emo_nsga3_select(Ft, Rt, n_keep, seed, gen, survivors=s_ws, info=i_ws)
    emo.emo_nsga3_select_noalloc(Ft, Rt, n_keep, seed, gen, survivors=s_na, info=i_na)
    torch.cuda.synchronize()
    return s_ws.cpu().numpy(), s_na.cpu().numpy(), i_ws.cpu().numpy(), i_na.cpu().numpy()


def test_noalloc_matches_workspace_entry_on_two_calls_in_a_row():
    _build.build()
    emo.lib()
    cases = [(wl.population(8000, 3, 12, "sphere", seed=501), wl.das_dennis(60, 3), 4000, 17, 3),
             (wl.population(2500, 5, 14, "linear", seed=502, quantize=32.0), wl.das_dennis(6, 5), 1300, 99, 4)]
    for F, R, n_keep, seed, gen in cases:
        s_ws, s_na, i_ws, i_na = _run_both(F, R, n_keep, seed, gen)
        assert i_ws[0] == 0 and i_na[0] == 0
        assert np.array_equal(s_na, s_ws)
        assert np.array_equal(i_na, i_ws)


def test_noalloc_rejects_populations_beyond_the_scratch():
    dev = torch.device("cuda")
    F = torch.from_numpy(wl.population(20000, 3, 12, "sphere", seed=503)).to(dev)
    R = torch.from_numpy(wl.das_dennis(140, 3)).to(dev)
    with pytest.raises(emo.EmoError) as e:
        emo.emo_nsga3_select_noalloc(F, R, 10000, 1, 0)
    assert e.value.status == 3  # EMO_ERR_WORKSPACE
