"""Pins for the oracle's transforms, convolution and projection (Sec. 3.2, 3.3).

Each check ties the oracle to something outside itself: numpy's FFT with the
centring shifts, scipy's linear convolution, numpy's least-squares projector,
exact algebraic identities, and a brute-force quadrature of the weak form
(Eq. collision_weakform) that uses a different discretisation altogether.
"""
import math

import numpy as np
import pytest
import scipy.signal

import oracle
from paper_1211_0540_gb300 import inputs

L = 6.0


def centred_fft(N, f):
    """(2pi)^{-3/2} dv^3 sum_j f_j exp(-2 pi i k'j'/N) via numpy's FFT with shifts."""
    dv = 2 * L / N
    F = np.fft.fftshift(np.fft.fftn(np.fft.ifftshift(f.reshape(N, N, N))))
    return (2 * math.pi) ** -1.5 * dv ** 3 * F.reshape(-1)


@pytest.mark.parametrize("N", [4, 6, 8])
def test_forward_dft_matches_numpy_fft(N):
    rng = np.random.default_rng(N)
    f = rng.standard_normal(N ** 3)
    ref = centred_fft(N, f)
    scale = np.abs(ref).max()
    assert np.abs(oracle.dft_forward_direct(N, L, f) - ref).max() <= 1e-13 * scale
    assert np.abs(oracle.dft_forward(N, L, f)[0] - ref).max() <= 1e-13 * scale


@pytest.mark.parametrize("N", [6, 8])
def test_inverse_dft_matches_numpy_and_round_trips(N):
    rng = np.random.default_rng(100 + N)
    qh = rng.standard_normal(N ** 3) + 1j * rng.standard_normal(N ** 3)
    dz = math.pi / L
    ref = (2 * math.pi) ** -1.5 * dz ** 3 * (N ** 3) * np.fft.fftshift(
        np.fft.ifftn(np.fft.ifftshift(qh.reshape(N, N, N)))).reshape(-1)
    out, ratio = oracle.dft_inverse(N, L, qh)
    assert np.abs(out[0] - ref.real).max() <= 1e-13 * np.abs(ref).max()
    assert abs(ratio[0] - np.linalg.norm(ref.imag) / np.linalg.norm(ref.real)) < 1e-12
    # round trip: dv^3 dz^3 / (2 pi)^3 * N^3 = 1
    f = rng.standard_normal((3, N ** 3))
    back, _ = oracle.dft_inverse(N, L, oracle.dft_forward(N, L, f))
    assert np.abs(back - f).max() <= 1e-13


def test_convolution_with_unit_weights_is_linear_convolution():
    """Ghat == 1: Qhat_k = dz^3 sum_m fhat_m fhat_{k-m+N/2}, i.e. the full linear
    convolution (scipy) read at offset N/2: a wrong shift or operand fails."""
    N = 6
    rng = np.random.default_rng(1)
    fh = rng.standard_normal(N ** 3) + 1j * rng.standard_normal(N ** 3)
    G = np.ones((N ** 3, N ** 3))
    # the oracle zeroes invalid pairs itself; a dense table of ones is fine
    got = oracle.convolve_dense(N, L, G, fh)[0].reshape(N, N, N)
    full = scipy.signal.convolve(fh.reshape(N, N, N), fh.reshape(N, N, N), mode="full")
    h = N // 2
    ref = (math.pi / L) ** 3 * full[h:h + N, h:h + N, h:h + N]
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_convolution_weight_roles_with_separable_table():
    """G[k, m] = g1(k) g2(m): Qhat_k = g1(k) * dz^3 * ((g2 fhat) conv fhat)(k + N/2).
    Pins which index of the table is zeta and which is xi."""
    N = 6
    rng = np.random.default_rng(2)
    fh = rng.standard_normal(N ** 3) + 1j * rng.standard_normal(N ** 3)
    g1 = rng.uniform(0.5, 2.0, N ** 3)
    g2 = rng.uniform(0.5, 2.0, N ** 3)
    got = oracle.convolve_dense(N, L, np.outer(g1, g2), fh)[0]
    full = scipy.signal.convolve((g2 * fh).reshape(N, N, N), fh.reshape(N, N, N), mode="full")
    h = N // 2
    ref = g1 * (math.pi / L) ** 3 * full[h:h + N, h:h + N, h:h + N].reshape(-1)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_table_convolution_equals_dense_convolution():
    N = 6
    rng = np.random.default_rng(3)
    fh = rng.standard_normal((2, N ** 3)) + 1j * rng.standard_normal((2, N ** 3))
    a = oracle.convolve(N, L, 1.0, fh)
    b = oracle.convolve_dense(N, L, oracle.ghat_dense(N, L, 1.0), fh)
    assert np.abs(a - b).max() <= 1e-14 * np.abs(b).max()


def test_convolution_invariants():
    N = 8
    f = inputs.homogeneous_cells(N, L, 1, seed=4)
    fh = oracle.dft_forward(N, L, f)
    q = oracle.convolve(N, L, 1.0, fh)
    k0 = np.ravel_multi_index((N // 2,) * 3, (N,) * 3)
    assert q[0, k0] == 0.0  # Ghat(xi, 0) = 0 -> Qhat(0) = 0 exactly
    q3 = oracle.convolve(N, L, 1.0, 3.0 * fh)
    assert np.abs(q3 - 9.0 * q).max() <= 1e-13 * np.abs(q).max()  # bilinear
    # xi <-> zeta - xi: the same sum with the weight moved to the partner index
    G = oracle.ghat_dense(N, L, 1.0)
    h = N // 2
    idx = np.arange(N ** 3)
    k = np.stack(np.unravel_index(idx, (N,) * 3), 1)
    Gs = np.zeros_like(G)
    for kk in range(N ** 3):
        n = k[kk] - k + h
        ok = np.all((n >= 0) & (n < N), axis=1)
        nn = np.ravel_multi_index(n[ok].T, (N,) * 3)
        Gs[kk, idx[ok]] = G[kk, nn]
    qs = oracle.convolve_dense(N, L, Gs, fh)
    assert np.abs(qs - q).max() <= 1e-12 * np.abs(q).max()


def test_gain_plus_loss_is_full():
    N = 6
    f = inputs.homogeneous_cells(N, L, 1, seed=5)
    fh = oracle.dft_forward(N, L, f)
    full = oracle.convolve(N, L, 0.0, fh, part=0)
    gain = oracle.convolve(N, L, 0.0, fh, part=2)
    loss = oracle.convolve(N, L, 0.0, fh, part=1)
    assert np.abs(gain + loss - full).max() <= 1e-13 * np.abs(gain).max()


def weakform_qhat(N, L, lam, f, kk_list):
    """Brute-force quadrature of the weak form (Eq. collision_weakform) with the
    isotropic sphere average done analytically:
    Qhat(zeta) = (2pi)^{-3/2} dv^6 sum_{j,j*} f_j f_j* |u|^lam
                 [sinc(|zeta||u|/2) e^{-i zeta.(v+v*)/2} - e^{-i zeta.v}],  u = v - v*."""
    v1, v2, v3 = inputs.velocity_nodes(N, L)
    V = np.stack([v1.ravel(), v2.ravel(), v3.ravel()], 1)
    f = f.reshape(-1)
    dv = 2 * L / N
    dz = math.pi / L
    U = V[:, None, :] - V[None, :, :]
    nu = np.linalg.norm(U, axis=2)
    ff = f[:, None] * f[None, :] * nu ** lam
    mid = 0.5 * (V[:, None, :] + V[None, :, :])
    out = []
    for kk in kk_list:
        zeta = dz * (np.array(np.unravel_index(kk, (N,) * 3)) - N // 2)
        nz = np.linalg.norm(zeta)
        arg = 0.5 * nz * nu
        sinc = np.where(arg == 0, 1.0, np.sin(arg) / np.where(arg == 0, 1.0, arg))
        gain = np.sum(ff * sinc * np.exp(-1j * mid @ zeta))
        loss = np.sum(ff * np.exp(-1j * V @ zeta)[:, None])
        out.append((2 * math.pi) ** -1.5 * dv ** 6 * (gain - loss))
    return np.array(out)


@pytest.mark.slow
def test_spectral_convolution_agrees_with_weak_form_quadrature():
    """Different discretisations of the same Qhat: the spectral oracle and the
    brute-force weak-form sum agree better as N grows (narrow Maxwellian mix so
    that the |u| <= L cut-off and the Fourier truncation are both harmless)."""
    lam = 1.0
    errs = []
    for N in (12, 16):
        f = (inputs.maxwellian(N, L, 0.6, (0.7, 0, 0), 0.6)
             + inputs.maxwellian(N, L, 0.4, (-0.7, 0.2, 0), 0.8))
        fh = oracle.dft_forward(N, L, f)
        q = oracle.convolve(N, L, lam, fh)[0]
        rng = np.random.default_rng(N)
        h = N // 2
        picks = [np.ravel_multi_index(tuple(rng.integers(h - 2, h + 3, 3)), (N,) * 3)
                 for _ in range(6)]
        ref = weakform_qhat(N, L, lam, f, picks)
        errs.append(np.abs(q[picks] - ref).max() / np.abs(ref).max())
    # measured: 2.8e-2 (N=12), 2.3e-3 (N=16); a wrong constant or sign is O(1)
    assert errs[1] < errs[0] / 5
    assert errs[1] < 5e-3


def test_projection_identities():
    N = 8
    rng = np.random.default_rng(6)
    Q = rng.standard_normal((3, N ** 3))
    P = oracle.project(N, L, Q)
    mom = oracle.moments(N, L, P)
    absmom = oracle.moments(N, L, np.abs(P))  # scale of each moment sum
    v1, v2, v3 = inputs.velocity_nodes(N, L)
    dv3 = (2 * L / N) ** 3
    C = dv3 * np.stack([np.ones(N ** 3), v1.ravel(), v2.ravel(), v3.ravel(),
                        (v1 ** 2 + v2 ** 2 + v3 ** 2).ravel()])
    scale = np.abs(C) @ np.abs(P).T
    assert np.all(np.abs(mom.T) <= 1e-12 * scale)              # C Q = 0
    assert np.abs(oracle.project(N, L, P) - P).max() <= 1e-12  # idempotent
    # equals the orthogonal projector onto null(C) (numpy least squares)
    lam_ls, *_ = np.linalg.lstsq(C.T, Q.T, rcond=None)
    ref = Q - (C.T @ lam_ls).T
    assert np.abs(P - ref).max() <= 1e-11 * np.abs(Q).max()
    del absmom


def test_raw_mass_moment_vanishes_before_projection():
    """Qhat(0) = 0, so the mass of Qt is zero up to roundoff before P_N."""
    N = 8
    f = inputs.homogeneous_cells(N, L, 2, seed=8)
    Q, raw, ratio = oracle.collide(N, L, 1.0, f, want_raw=True)
    m = oracle.moments(N, L, raw)
    scale = oracle.moments(N, L, np.abs(raw))
    assert np.all(np.abs(m[:, 0]) <= 1e-13 * scale[:, 0])
    assert np.all(ratio < 1.0)
