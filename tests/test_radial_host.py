"""The library's radial integrals (csrc/radial.h: closed forms for lambda = 0, 1
and the series-and-panels rule of the tables for other lambda down to the soft
potentials' -3 < lambda, Sec. 2.1-2.2), compiled
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
        lam, a, b, cf, q, sr, sp = (float(x) for x in row[1:])
        s1 = mpmath.mpf(lam) + 3  # s + 1 with s = lambda + 2

        # r = u^(1/(s+1)) turns r^s dr into du/(s+1): no singular factor at 0 for any lambda > -3
        def g(u):
            r = u ** (1 / s1) if u > 0 else mpmath.mpf(0)
            return (mpmath.sinc(a * r) if a else 1) * (mpmath.sinc(b * r) if b else 1)

        ref = float(mpmath.quad(g, [0] + [(mpmath.mpf(L) * i / 96) ** s1 for i in range(1, 97)]) / s1)
        tol = 1e-13 * abs(ref) + 1e-15
        assert abs(sr - ref) <= tol, ("series rule, table omega", lam, a, b, sr, ref)
        assert abs(sp - ref) <= tol, ("series rule, pair omega", lam, a, b, sp, ref)
        if lam in (0.0, 1.0):
            assert abs(q - ref) <= tol, ("panel rule", lam, a, b, q, ref)
            # the closed form where the library uses it (elsewhere it cancels: quadrature is used)
            if a == 0.0 or b == 0.0 or b * L >= 0.25:
                assert abs(cf - ref) <= tol, ("closed form", lam, a, b, cf, ref)
        nI += 1
    assert nI == 96
