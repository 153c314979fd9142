"""Pins for the oracle's quadrature and convolution weights (Sec. 2.2, Eq. GHat_calc).

The oracle evaluates the radial integrals by composite Gauss-Legendre
quadrature. Here they are checked against closed forms for lambda = 0, 1 that
the tests derive on their own (integration by parts; not the oracle's method):
  sinc(ar) sinc(br) r^2 = [cos((a-b) r) - cos((a+b) r)] / (2ab), so
  I_lam(a, b) = [C_lam(a-b) - C_lam(a+b)] / (2ab),  C_lam(k) = int_0^L r^lam cos(kr) dr,
  C_0(k) = sin(kL)/k,  C_1(k) = L sin(kL)/k - 2 sin^2(kL/2)/k^2,
  J_0(c) = (sin cL - cL cos cL)/c^3,  J_1(c) = (2cL sin cL - (c^2L^2 - 2) cos cL - 2)/c^4.
"""
import itertools
import math

import numpy as np
import pytest

import oracle

L = 6.0


def C_lam(lam, k):
    if abs(k) < 1e-12:
        return L ** (lam + 1) / (lam + 1)
    if lam == 0:
        return math.sin(k * L) / k
    return L * math.sin(k * L) / k - 2.0 * math.sin(0.5 * k * L) ** 2 / k ** 2


def I_closed(lam, a, b):
    if a == 0.0:
        return J_closed(lam, b)
    if b == 0.0:
        return J_closed(lam, a)
    return (C_lam(lam, a - b) - C_lam(lam, a + b)) / (2.0 * a * b)


def J_closed(lam, c):
    if c == 0.0:
        return L ** (lam + 3) / (lam + 3)
    x = c * L
    if lam == 0:
        return (math.sin(x) - x * math.cos(x)) / c ** 3
    return (2 * x * math.sin(x) - (x * x - 2) * math.cos(x) - 2) / c ** 4


def test_gauss_legendre_matches_numpy():
    for n in (1, 2, 3, 7, 16, 33):
        x, w = oracle.gauss_legendre(n)
        xr, wr = np.polynomial.legendre.leggauss(n)
        assert np.allclose(x, xr, atol=1e-14, rtol=0)
        assert np.allclose(w, wr, atol=1e-14, rtol=0)


def test_gauss_legendre_exact_on_polynomials():
    n = 9
    x, w = oracle.gauss_legendre(n)
    for deg in range(2 * n):
        exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
        assert abs(np.dot(w, x ** deg) - exact) < 1e-13


@pytest.mark.parametrize("lam", [0.0, 1.0])
def test_radial_integrals_match_closed_forms(lam):
    rng = np.random.default_rng(7)
    hz = 0.5 * math.pi / L
    cases = [(0.0, 0.0), (0.0, 3 * hz), (hz, hz), (hz * math.sqrt(2), hz), (5 * hz, 5.01 * hz)]
    cases += [tuple(rng.uniform(0, 15 * hz, size=2)) for _ in range(20)]
    scale = L ** (lam + 3)
    for a, b in cases:
        assert abs(oracle.radial_I(lam, L, a, b) - I_closed(lam, a, b)) <= 1e-13 * scale
    for c in [0.0, hz, 1.0, 2.5, 7.3, 12.0]:
        assert abs(oracle.radial_J(lam, L, c) - J_closed(lam, c)) <= 1e-13 * scale


@pytest.mark.parametrize("lam", [0.0, 1.0])
def test_ghat_pair_closed_form(lam):
    """Ghat = sqrt(2/pi) [I(|zeta|/2, |xi - zeta/2|) - J(|xi|)] on grid points."""
    N = 8
    dz = math.pi / L
    rng = np.random.default_rng(3)
    for _ in range(25):
        k = rng.integers(0, N, size=3)
        m = rng.integers(0, N, size=3)
        zeta = dz * (k - N // 2)
        xi = dz * (m - N // 2)
        ref = math.sqrt(2 / math.pi) * (
            I_closed(lam, np.linalg.norm(zeta) / 2, np.linalg.norm(xi - zeta / 2))
            - J_closed(lam, np.linalg.norm(xi)))
        assert abs(oracle.ghat_pair(N, L, lam, k, m) - ref) <= 1e-12 * L ** (lam + 3)


def test_ghat_vanishes_at_zeta_zero():
    """Ghat(xi, 0) = 0 exactly: the gain and loss integrands coincide."""
    N = 8
    for m in itertools.product(range(N), repeat=3):
        assert oracle.ghat_pair(N, L, 1.0, [N // 2] * 3, m) == 0.0
        if m[0] == 3 and m[1] == 3:
            break


@pytest.mark.parametrize("lam", [0.0, 1.0, 0.5, -1.5, -2.5])
def test_weight_table_matches_pair_quadrature(lam):
    N = 8
    G = oracle.ghat_dense(N, L, lam)
    rng = np.random.default_rng(11)
    gmax = np.abs(G).max()
    checked = 0
    while checked < 40:
        kk, mm = rng.integers(0, N ** 3, size=2)
        k = np.array(np.unravel_index(kk, (N, N, N)))
        m = np.array(np.unravel_index(mm, (N, N, N)))
        n = k - m + N // 2
        if np.any(n < 0) or np.any(n >= N):
            assert G[kk, mm] == 0.0  # outside the zero-extended support
            continue
        assert abs(G[kk, mm] - oracle.ghat_pair(N, L, lam, k, m)) <= 1e-13 * gmax
        checked += 1
    # row zeta = 0 is identically zero
    k0 = np.ravel_multi_index((N // 2,) * 3, (N, N, N))
    assert np.all(G[k0] == 0.0)


def test_weight_table_symmetries():
    """Ghat depends on |zeta|, |xi - zeta/2|, |xi|: invariant under axis
    permutations and joint sign flips (where the flipped index is on the grid)."""
    N = 8
    h = N // 2
    G = oracle.ghat_dense(N, L, 1.0).reshape((N,) * 6)
    rng = np.random.default_rng(5)
    for _ in range(200):
        kp = rng.integers(-h + 1, h, size=3)
        mp = rng.integers(-h + 1, h, size=3)
        if np.any(np.abs(kp - mp) > h - 1):
            continue  # keep n' = k' - m' (and its sign flip) on the grid
        base = G[tuple(kp + h) + tuple(mp + h)]
        perm = rng.permutation(3)
        assert G[tuple(kp[perm] + h) + tuple(mp[perm] + h)] == base
        s = rng.choice([-1, 1], size=3)
        assert abs(G[tuple(s * kp + h) + tuple(s * mp + h)] - base) <= 1e-15 * abs(base) + 1e-300


@pytest.mark.parametrize("lam", [0.1, 0.3, 0.5, 0.75, -0.5, -1.0, -1.5, -2.0, -2.5, -2.9])
def test_radial_integrals_for_non_integer_lambda_match_high_precision_quadrature(lam):
    """Sec. 2.2: for non-integer lambda the weights are a 1-D integral evaluated by
    quadrature, here also for the soft potentials -3 < lambda < 0 of Sec. 2.1, whose
    factor r^(lambda+2) is singular at 0 for lambda < -2. Reference: mpmath at 30
    digits after r = u^(1/(lambda+3)), which turns r^(lambda+2) dr into
    du/(lambda+3) (64 panels); the oracle's graded composite Gauss-Legendre rule
    must agree to FP64 level."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    s1 = mpmath.mpf(lam) + 3
    for a, b in ((0.0, 0.0), (0.26, 0.26), (1.3, 4.1), (7.2, 13.9), (0.0, 5.0), (3.3, 0.2)):
        def g(u):
            r = u ** (1 / s1) if u > 0 else mpmath.mpf(0)
            return (mpmath.sinc(a * r) if a else 1) * (mpmath.sinc(b * r) if b else 1)
        ref = float(mpmath.quad(g, [0] + [(mpmath.mpf(L) * i / 64) ** s1 for i in range(1, 65)]) / s1)
        if a == 0.0 and b == 0.0:  # int_0^L r^(lambda+2) dr in closed form
            assert abs(ref - L ** (lam + 3) / (lam + 3)) <= 1e-14 * abs(ref)
        got = oracle.radial_I(lam, L, a, b)
        assert abs(got - ref) <= 1e-13 * abs(ref) + 1e-16, (a, b, got, ref)
        if a == 0.0:
            assert abs(oracle.radial_J(lam, L, b) - ref) <= 1e-13 * abs(ref) + 1e-16
