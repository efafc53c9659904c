"""Offline autotuning of launch shapes and the sticky device status."""
import pytest
import torch

import oracle
from paper_2503_20286_gb300 import _binding as emo
from paper_2503_20286_gb300 import workloads as wl

from . import _gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def test_autotune_writes_and_reuses_the_cache_and_keeps_results(tmp_path):
    path = str(tmp_path / "tune.txt")
    emo.emo_autotune(3, 20000, path)
    lines = open(path).read().split()
    major, minor = torch.cuda.get_device_capability()
    assert len(lines) == 4 and lines[0] == str(10 * major + minor) and lines[1:3] == ["3", "14"]
    assert int(lines[3]) in (2, 4, 8, 16, 32)
    emo.emo_autotune(3, 20000, path)               # found in the cache: nothing appended
    assert open(path).read().split() == lines
    p = wl.config(1)                                # 2N = 20,000, M = 3: runs with the tuned shape
    _gpu.compare_select(p.F, p.R, p.n_keep, p.seed, p.generation)


def test_sticky_status_reports_the_first_device_failure_once():
    emo.emo_get_last_device_status()              # clear anything earlier tests left
    F = wl.population(600, 3, 9, "sphere", seed=33)
    R = wl.das_dennis(8, 3)
    R[5, 1] = -0.25                                 # a negative direction is refused on the device
    s, info, _ = _gpu.gpu_select(F, R, 300, seed=1, debug=False)
    assert info["status"] == 1
    assert emo.emo_get_last_device_status() == 1
    assert emo.emo_get_last_device_status() == 0
    p = wl.config(0)                                # a good call leaves the word at zero
    _gpu.compare_select(p.F, p.R, p.n_keep, p.seed, p.generation)
    assert emo.emo_get_last_device_status() == 0
