"""Host check of the step kernels' index arithmetic: row_geometry_check.cu
includes the kernels' own host-and-device row geometry and enumerates every
thread of the step launches on many lattice shapes (periodic and bounded
axes, D2Q9 batches), checking coverage, the unknown links, every population
index read and every block-sum slot.  Runs on the CPU (nvcc builds a host program)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_row_geometry_indices(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "row_geometry_check")
    res = subprocess.run([nvcc, "-O1", "-std=c++17", "-I", os.path.join(ROOT, "include"),
                          "-I", os.path.join(ROOT, "paper_2608_19617_b300", "csrc"),
                          os.path.join(HERE, "row_geometry_check.cu"), "-o", exe],
                         capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-3000:]
    run = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert run.returncode == 0 and run.stdout.strip().endswith("(0 failures)"), run.stdout[-3000:]
