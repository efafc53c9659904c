"""CPU checks of the C ABI: the library builds, loads and exports every entry
point declared in include/emo.h; host-side argument checks reject bad calls
before anything is launched. No compute call runs here."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "emo.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(emo_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2503_20286_gb300 import build, _binding
    build.build()
    return _binding.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("emo_dominance", "emo_nd_rank", "emo_nsga3_select", "emo_nsga3_select_batch",
                 "emo_workspace_size", "emo_batch_workspace_size"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2503_20286_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(emo_[a-z0-9_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_status_strings_and_version(lib):
    from paper_2503_20286_gb300 import _binding as b
    assert b.emo_version() >= 100
    for code in range(7):
        assert b.emo_status_string(code)
    assert b.emo_status_string(99) == "unknown status"


def test_host_argument_checks_reject_before_launch(lib):
    L = lib
    # null pointers / bad sizes are refused on the host (no CUDA call)
    assert L.emo_dominance(None, 10, 3, None, 1, None, None) == 1
    assert L.emo_dominance(ctypes.c_void_p(256), 10, 1, ctypes.c_void_p(256), 1, None, None) == 1
    assert L.emo_dominance(ctypes.c_void_p(256), 100, 3, ctypes.c_void_p(256), 3, None, None) == 1  # ld < 4
    assert L.emo_nsga3_select(None, 10, 3, None, 5, 5, 0, 0, None, None, None, 0, None) == 1
    p = ctypes.c_void_p(256)
    assert L.emo_nsga3_select(p, 10, 3, p, 5, 11, 0, 0, p, None, p, 1 << 20, None) == 1  # n_keep > n2
    assert L.emo_nsga3_select(p, 10, 17, p, 5, 5, 0, 0, p, None, p, 1 << 20, None) == 1  # m > 16
    assert L.emo_nsga3_select(p, 10, 3, p, 0, 5, 0, 0, p, None, p, 1 << 20, None) == 1   # no references
    assert L.emo_nd_rank(p, 0, 3, 0, p, None, p, 1 << 20, None) == 1                      # n2 = 0
    assert L.emo_nd_rank(p, 10, 3, 11, p, None, p, 1 << 20, None) == 1                    # n_keep > n2
    assert L.emo_nsga3_select_batch(None, 1, p, 1 << 20, None) == 1
    assert L.emo_nsga3_select_ex(p, 10, 3, p, 5, 5, 0, 0, 2, p, None, None, p, 1 << 20, None) == 1  # niche mode
    assert L.emo_hype_select(p, 10, 3, p, None, 100, 5, p, None, None, p, 1 << 20, None) == 1        # no samples
    assert L.emo_autotune(3, 10, None) == 1                                                          # n2 < 64
    assert L.emo_autotune(1, 1000, None) == 1                                                        # m < 2
    assert L.emo_launch_shape(3, 1000, None) == 1                                                    # no output
    assert L.emo_launch_shape(17, 1000, p) == 1                                                      # m > 16
    assert L.emo_dominance_cols(p, 3000, 3, 1000, 2000, p, 40, None, None) == 1        # col_lo not a block start
    assert L.emo_dominance_cols(p, 3000, 3, 1024, 3001, p, 40, None, None) == 1        # col_hi > n2
    assert L.emo_dominance_cols(p, 3000, 3, 1024, 2048, p, 31, None, None) == 1        # ld < 32 words
    assert L.emo_front_counts(p, 4, 100, None, 5, p, p, None) == 1                     # rows missing
    assert L.emo_front_counts(p, 3, 100, p, 5, p, p, None) == 1                        # ld < 4 words
    assert L.emo_nsga3_select_ranked(p, 10, 3, p, 5, 5, 0, 0, None, p, None, p, 1 << 20, None) == 1  # no ranks
    assert L.emo_workspace_size(6, 1000, 3, 0) == 0                                    # ranked: no directions
    assert L.emo_get_last_device_status(None, None) == 1
    assert L.emo_hype_select(p, 10, 3, p, p, 0, 5, p, None, None, p, 1 << 20, None) == 1           # s = 0
    assert L.emo_workspace_size(2, 0, 3, 5) == 0
    assert L.emo_workspace_size(2, 10, 1, 5) == 0
    assert L.emo_workspace_size(7, 10, 3, 5) == 0
    assert L.emo_workspace_size(0, 10, 3, 5) == 0    # dominance needs no workspace
    assert L.emo_workspace_status(None, None, None) == 1
    # TensorMOEA/D selection: X, F1, O, F2, n, d, m, z, W, I_nb, T, theta, X_next, F_next, winner, status, ws
    mo = lambda n, d, m, T, theta, ws, nbytes: L.emo_moead_select(p, p, p, p, n, d, m, p, p, p, T, theta, p, p,
                                                                 None, None, ws, nbytes, None)
    assert L.emo_moead_select(None, p, p, p, 10, 4, 3, p, p, p, 2, 5.0, p, p, None, None, p, 1 << 20, None) == 1
    assert mo(10, 4, 3, 11, 5.0, p, 1 << 20) == 1                       # T > n
    assert mo(10, 4, 3, 0, 5.0, p, 1 << 20) == 1                        # T = 0
    assert mo(10, 0, 3, 2, 5.0, p, 1 << 20) == 1                        # d = 0
    assert mo(10, 4, 17, 2, 5.0, p, 1 << 20) == 1                       # m > 16
    assert mo(10, 4, 3, 2, -1.0, p, 1 << 20) == 1                       # theta < 0
    assert mo(10, 4, 3, 2, float("nan"), p, 1 << 20) == 1               # theta NaN
    assert mo(10, 4, 3, 2, 5.0, ctypes.c_void_p(128), 1 << 20) == 1     # workspace not 256-byte aligned
    assert mo(100, 4, 3, 10, 5.0, p, 14079) == 3                        # one byte short
    # regions: status + z_min keys (256), best value 8n, lowest index 4n, pair values 8nT, per-subproblem
    # ||w||, own value and unit weights 8n(m + 2), each 256-aligned
    assert L.emo_workspace_size(4, 100, 3, 10) == 14080
    assert L.emo_workspace_size(4, 100, 3, 0) == 0
    assert L.emo_workspace_size(4, 100, 3, 101) == 0
    # generation operators
    assert L.emo_variation(None, 10, 4, None, None, 10, 0, 0, 20.0, 20.0, 1.0, 0.25, p, None, None) == 1
    assert L.emo_variation(p, 10, 4, p, None, 10, 0, 0, 20.0, 20.0, 1.0, 0.25, p, None, None) == 1   # lo without hi
    assert L.emo_variation(p, 10, 4, None, None, 0, 0, 0, 20.0, 20.0, 1.0, 0.25, p, None, None) == 1  # no offspring
    assert L.emo_variation(p, 10, 4, None, None, 10, 0, 0, -1.0, 20.0, 1.0, 0.25, p, None, None) == 1  # eta_c < 0
    assert L.emo_variation(p, 10, 1 << 24, None, None, 10, 0, 0, 20.0, 20.0, 1.0, 0.25, p, None, None) == 1
    assert L.emo_standin_objectives(p, 10, 2, 3, 1, p, None) == 1                        # d < m
    assert L.emo_standin_objectives(p, 10, 12, 3, 7, p, None) == 1                       # unknown shape
    assert L.emo_igd(p, 10, 3, p, 5, p, p, 39, None) == 3                                 # 8 bytes per reference
    assert L.emo_igd(p, 10, 3, p, 0, p, p, 1 << 20, None) == 1
    assert L.emo_workspace_size(5, 1000, 3, 0) == 8000
    assert L.emo_generation_workspace_size(100, 2, 3, 91) == 0                            # d < m
    assert L.emo_generation_workspace_size(100, 12, 3, 0) == 0                            # no directions
    assert L.emo_generation_workspace_size(100, (1 << 20) + 1, 3, 91) == 0
    assert L.emo_nsga3_generation(p, p, 100, 2, 3, p, 91, 1, 0, 0, 20.0, 20.0, 1.0, 0.1, 0, None, p, 1 << 30,
                                  None) == 1                                              # d < m
    assert L.emo_nsga3_generation(p, p, 100, 12, 3, p, 91, 1, 0, 0, 20.0, 20.0, 1.0, 0.1, 0, None,
                                  ctypes.c_void_p(128), 1 << 30, None) == 1               # workspace alignment
