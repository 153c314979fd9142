"""The library's radial integrals (csrc/radial.h: closed forms for lambda = 0, 1
and the Clenshaw-Curtis quadrature used for other lambda, Sec. 2.2), compiled
for the host and checked against 30-digit quadrature (mpmath), including the
small-argument case that inelastic weights reach (b near 0)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
L = 6.0


def test_radial_integrals_match_high_precision_quadrature(tmp_path):
    mpmath = pytest.importorskip("mpmath")
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not found")
    exe = tmp_path / "radial_check"
    subprocess.run([gxx, "-std=c++17", "-O2", "-o", str(exe), os.path.join(HERE, "host", "radial_check.cpp")],
                   check=True, capture_output=True, timeout=300)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout.split("\n")
    mpmath.mp.dps = 30
    nI = 0
    for row in (r.split() for r in out if r.strip()):
        if row[0] == "P":
            assert float(row[2]) < 1e-14, row  # CC rule exact on polynomials of degree <= 24
            continue
        lam, a, b, cf, q = (float(x) for x in row[1:])

        def f(r):
            return r ** (lam + 2) * (mpmath.sinc(a * r) if a else 1) * (mpmath.sinc(b * r) if b else 1)

        ref = float(mpmath.quad(f, [0] + [L * i / 96 for i in range(1, 97)]))
        tol = 1e-13 * abs(ref) + 1e-15
        assert abs(q - ref) <= tol, ("quadrature", lam, a, b, q, ref)
        # the closed form where the library uses it (elsewhere it cancels: quadrature is used)
        if lam in (0.0, 1.0) and (a == 0.0 or b == 0.0 or b * L >= 0.25):
            assert abs(cf - ref) <= tol, ("closed form", lam, a, b, cf, ref)
        nI += 1
    assert nI == 48
