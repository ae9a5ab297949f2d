"""Host check of the banded 2D stage's work list (no GPU): tests/band_plan_check.cu
includes the library's own planner and item decoder, builds as a host program and checks,
on grids with ragged tiles, ragged last bands and many bands, that every x and y tile is
listed exactly once in the band that holds its rows, that ring rows stay inside a slot,
and that every wait of the persistent kernel targets items listed before the waiting
one -- the condition under which the launch always completes."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_band_work_list_is_complete_and_ordered():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "band_plan_check")
        r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-x", "cu", "-o", exe,
                            os.path.join(HERE, "band_plan_check.cu")], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
