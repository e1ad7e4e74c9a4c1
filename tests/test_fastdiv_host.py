"""The invariant-divisor division of the kernels' node indexing (FastDiv in
albm_node.cuh) against plain integer division, compiled for and run on the
host (nvcc, no GPU needed)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_fastdiv_matches_integer_division(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "fastdiv_check")
    subprocess.run([nvcc, "-std=c++17", "-O2", os.path.join(HERE, "fastdiv_check.cu"), "-o", exe],
                   check=True, capture_output=True, text=True)
    res = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stdout + res.stderr
    assert "mismatches 0" in res.stdout
