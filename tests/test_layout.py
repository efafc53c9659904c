"""Host-side checks of the dominance-tile layout and workspace carving: the
internal header is compiled with g++ (no GPU) and the tile indexing, work
item decomposition and workspace regions are checked exhaustively for a
range of population sizes."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_tile_layout_and_workspace(tmp_path):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    exe = tmp_path / "layout_check"
    subprocess.check_call([gxx, "-std=c++17", "-O1", os.path.join(HERE, "host", "layout_check.cpp"), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "layout ok" in out.stdout
