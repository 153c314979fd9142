"""The integer-pipe binary32 <-> binary64 conversions used by the transforms
(fpconv.cuh), compiled for the host and compared bit for bit with the
compiler's conversions (round to nearest even, subnormals, overflow, NaN)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_conversions_match_ieee_rounding(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = tmp_path / "fpconv_check"
    subprocess.run([nvcc, "-std=c++17", "-O2", "-o", str(exe), os.path.join(HERE, "host", "fpconv_check.cu")],
                   check=True, capture_output=True, timeout=300)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=300).stdout
    last = out.strip().split("\n")[-1].split()
    assert last[0] == "mismatches" and int(last[3]) > 5_000_000, out
    assert int(last[1]) == 0, out
