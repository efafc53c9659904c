"""Offline autotuning of launch shapes and the sticky device status."""
import numpy as np
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
    emo.emo_autotune_reset()
    default = emo.emo_launch_shape(3, 20000)
    path = str(tmp_path / "tune.txt")
    emo.emo_autotune(3, 20000, path)
    lines = open(path).read().split()
    major, minor = torch.cuda.get_device_capability()
    assert len(lines) == 8 and lines[0] == str(10 * major + minor) and lines[1:3] == ["3", "14"]
    assert int(lines[3]) in (2, 4, 8, 16, 32)
    assert int(lines[4]) in (64, 128, 256, 512, 1024)
    G = default["peel_ctas"]
    assert 0 <= int(lines[5]) <= G and 0 <= int(lines[6]) <= G
    shape = emo.emo_launch_shape(3, 20000)
    assert shape["assoc_blocks_per_sm"] == int(lines[3]) and shape["dom_rowblocks_per_item"] == int(lines[4])
    assert shape["other_coop_ctas"] <= shape["peel_ctas"] <= G
    assert shape["peel_wavefront"] == int(lines[7]) in (0, 1)
    emo.emo_autotune(3, 20000, path)               # found in the cache: nothing appended
    assert open(path).read().split() == lines
    p = wl.config(1)                                # 2N = 20,000, M = 3: runs with the tuned shapes
    _gpu.compare_select(p.F, p.R, p.n_keep, p.seed, p.generation)
    emo.emo_autotune_reset()
    assert emo.emo_launch_shape(3, 20000) == default


def test_association_only_cache_lines_still_load(tmp_path):
    """A four-field line (arch m bucket blocks) tunes the association kernel
    only; the other shapes keep their defaults."""
    emo.emo_autotune_reset()
    default = emo.emo_launch_shape(5, 3000)
    assert default["dom_rowblocks_per_item"] in (64, 128, 256, 512, 1024)
    major, minor = torch.cuda.get_device_capability()
    path = tmp_path / "old.txt"
    path.write_text(f"{10 * major + minor} 5 11 16\n")
    try:
        emo.emo_autotune(5, 3000, str(path))       # found in the file: nothing is timed or appended
        assert path.read_text().split() == [str(10 * major + minor), "5", "11", "16"]
        got = emo.emo_launch_shape(5, 3000)
        assert got["assoc_blocks_per_sm"] == 16
        assert got["dom_rowblocks_per_item"] == 1024 and got["peel_ctas"] == default["peel_ctas"]
    finally:
        emo.emo_autotune_reset()


@pytest.mark.parametrize("cap_wide,cap_narrow,chunk", [(1, 1, 64), (3, 2, 128), (7, 7, 1024), (0, 1, 256)])
def test_any_launch_shape_gives_the_same_survivors(tmp_path, cap_wide, cap_narrow, chunk):
    """A single CTA per front (no grid barrier), a few CTAs, or every CTA;
    small or large dominance items: survivors and intermediates stay
    bit-exact with the oracle (2N = 20,000 M = 3 and 2N = 3,000 M = 5)."""
    major, minor = torch.cuda.get_device_capability()
    arch = 10 * major + minor
    path = tmp_path / "shape.txt"
    path.write_text(f"{arch} 3 14 8 {chunk} {cap_wide} {cap_narrow}\n{arch} 5 11 4 {chunk} {cap_wide} {cap_narrow}\n")
    emo.emo_autotune_reset()
    try:
        emo.emo_autotune(3, 20000, str(path))      # loads the file; the entry exists, so nothing is timed
        emo.emo_autotune(5, 3000, str(path))
        sh = emo.emo_launch_shape(3, 20000)
        assert sh["dom_rowblocks_per_item"] == chunk
        if cap_wide:
            assert sh["peel_ctas"] == cap_wide
        p = wl.config(1)
        _gpu.compare_select(p.F, p.R, p.n_keep, p.seed, p.generation)
        F = wl.population(3000, 5, 14, "linear", seed=71, quantize=32.0)
        _gpu.compare_select(F, wl.das_dennis(6, 5), 1500, 5, 2)
        r, last = _gpu.gpu_rank(p.F)
        assert np.array_equal(r, oracle.nd_sort_deb(p.F)) and last == int(r.max())
    finally:
        emo.emo_autotune_reset()


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
