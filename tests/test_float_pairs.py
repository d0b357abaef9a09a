"""The library converts between doubles, floats and (hi, lo) float pairs in
integer arithmetic, so that its element, Galerkin and float32-copy kernels
issue no double-pipe instruction (GB300 runs double arithmetic at 1/61 of the
float rate).  These conversions must give bitwise what the IEEE conversions
give: checked on the host on a few million values, with the edge cases
(powers of two, exact ties, zeros, random bit patterns)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_integer_conversions_match_ieee(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "float_pairs_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-x", "cu", os.path.join(HERE, "float_pairs_check.cu"),
                    "-o", exe], check=True, capture_output=True)
    r = subprocess.run([exe, "3000000"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
