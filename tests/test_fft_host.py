"""The register FFT of the fused transforms (fft_reg.cuh), compiled for the
host and checked against the dense DFT sums for every supported N (8, 12, 16,
24, 32), both signs, plain and centred (the phases of Sec. 3.2's transform)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_register_fft_matches_dense_sums(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = tmp_path / "fft_check"
    subprocess.run([nvcc, "-std=c++17", "-O2", "-o", str(exe), os.path.join(HERE, "host", "fft_check.cu")],
                   check=True, capture_output=True, timeout=300)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout.split("\n")
    rows = [r.split() for r in out if r.strip()]
    assert len(rows) == 20
    for n, s, kind, err in rows:
        # FP32 butterflies: a few ulps times log2 N
        assert float(err) < 5e-7, (n, s, kind, err)
