"""Pins of the oracle's inelastic operator (beta in Eq. G_eqn and Eq. GHat_calc,
Sec. 2.2) and of the projection without the energy row (Sec. 3.3).

- beta = 1 through the inelastic tables (gain integrals on (|k'|^2, |m'|^2,
  k'.m')) reproduces the elastic tables (on (|k'|^2, |2m' - k'|^2)).
- Energy: with the rule v' = v + (beta/2)(|u| sigma - u) and isotropic b, the
  sphere average of |v'|^2 + |v*'|^2 - |v|^2 - |v*|^2 is -beta(1-beta)|u|^2, so
  int Q |v|^2 dv = -(beta(1-beta)/2) int int f f* |u|^(lambda+2). For Maxwell
  molecules (lambda = 0) that is -beta(1-beta)(rho E - |P|^2) for any f; for
  hard spheres and a Maxwellian at rest it is -(beta(1-beta)/2) rho^2 (2T)^(3/2)
  E|Z|^3 with E|Z|^3 = 2^(3/2) Gamma(3) / Gamma(3/2) (Z a standard normal in 3-D).
  The discrete operator must converge to both as N grows (a misplaced beta
  gives an O(1) error that does not shrink).
- Weak-form brute force with the inelastic rule (a different discretisation).
- Projection on mass and momentum: CQ = 0 on those rows, idempotence, the
  minimal-norm correction (numpy least squares on the four rows).
"""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_1211_0540_gb300 import inputs

L = 6.0


def moments(N, f):
    v1, v2, v3 = inputs.velocity_nodes(N, L)
    dv3 = (2 * L / N) ** 3
    f = np.asarray(f).reshape(-1)
    rho = f.sum() * dv3
    P = np.array([(f * v.ravel()).sum() * dv3 for v in (v1, v2, v3)])
    E = (f * (v1 ** 2 + v2 ** 2 + v3 ** 2).ravel()).sum() * dv3
    return rho, P, E


def test_beta_one_through_the_inelastic_tables_is_the_elastic_operator():
    N, lam = 8, 1.0
    f = inputs.homogeneous_cells(N, L, 2, seed=71)
    fh = oracle.dft_forward(N, L, f)
    w = oracle.WeightsBeta(N, L, lam, 1.0)
    out = np.zeros(fh.shape, dtype=np.complex128)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    fh64 = np.ascontiguousarray(fh)
    oracle.lib().ora_convolve_beta(N, L, 2, p(w.I3), p(w.J), 0, p(fh64.view(np.float64)), p(out.view(np.float64)))
    ref = oracle.convolve(N, L, lam, fh)
    assert np.abs(out - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("beta", [0.8, 0.6])
def test_energy_dissipation_of_maxwell_molecules(beta):
    errs = []
    for N in (8, 12, 16):
        f = inputs.maxwellian(N, L, 0.6, (0.5, 0, 0), 0.7) + inputs.maxwellian(N, L, 0.4, (-0.6, 0.2, 0), 1.0)
        _, raw, _ = oracle.collide(N, L, 0.0, f[None], beta=beta, want_raw=True)
        rho, P, E = moments(N, f)
        ref = -beta * (1 - beta) * (rho * E - P @ P)
        errs.append(abs(moments(N, raw)[2] - ref) / abs(ref))
    # measured (beta = 0.8): 0.64, 4.4e-2, 9.4e-4
    assert errs[0] > 5 * errs[1] > 25 * errs[2], errs
    assert errs[2] < 5e-3, errs


def test_energy_dissipation_of_hard_spheres_for_a_maxwellian():
    beta, T = 0.8, 1.0
    EZ3 = 2 ** 1.5 * math.gamma(3) / math.gamma(1.5)
    errs = []
    for N in (8, 12, 16):
        f = inputs.maxwellian(N, L, 1.0, (0, 0, 0), T)
        _, raw, _ = oracle.collide(N, L, 1.0, f[None], beta=beta, want_raw=True)
        rho, _, _ = moments(N, f)
        ref = -(beta * (1 - beta) / 2) * rho ** 2 * (2 * T) ** 1.5 * EZ3
        errs.append(abs(moments(N, raw)[2] - ref) / abs(ref))
    # measured: 0.63, 2.0e-2, 7.6e-3
    assert errs[0] > 10 * errs[1] and errs[2] < errs[1], errs
    assert errs[2] < 1e-2, errs


def test_inelastic_projection_conserves_mass_and_momentum_only():
    N, beta = 12, 0.8
    f = inputs.homogeneous_cells(N, L, 2, seed=72)
    Q = oracle.collide(N, L, 1.0, f, beta=beta)
    v1, v2, v3 = inputs.velocity_nodes(N, L)
    dv3 = (2 * L / N) ** 3
    C = dv3 * np.stack([np.ones(N ** 3), v1.ravel(), v2.ravel(), v3.ravel(), (v1 ** 2 + v2 ** 2 + v3 ** 2).ravel()])
    m = Q @ C.T
    scale = np.abs(Q) @ np.abs(C).T
    assert np.all(np.abs(m[:, :4]) <= 1e-12 * scale[:, :4])
    assert np.all(m[:, 4] < -1e-3 * scale[:, 4])  # energy is dissipated, not restored


def test_projection_on_four_rows_identities():
    N = 8
    rng = np.random.default_rng(73)
    Q = rng.standard_normal((3, N ** 3))
    P1 = oracle.project(N, L, Q, rows=4)
    v1, v2, v3 = inputs.velocity_nodes(N, L)
    dv3 = (2 * L / N) ** 3
    C4 = dv3 * np.stack([np.ones(N ** 3), v1.ravel(), v2.ravel(), v3.ravel()])
    assert np.abs(P1 @ C4.T).max() <= 1e-12 * (np.abs(Q) @ np.abs(C4).T).max()
    assert np.abs(oracle.project(N, L, P1, rows=4) - P1).max() <= 1e-13 * np.abs(Q).max()
    lam, *_ = np.linalg.lstsq(C4.T, Q.T, rcond=None)  # minimal correction within the row space
    ref = Q - (C4.T @ lam).T
    assert np.abs(P1 - ref).max() <= 1e-11 * np.abs(Q).max()


def weakform_qhat_beta(N, lam, beta, f, kk_list):
    """Weak form (Eq. collision_weakform) with the inelastic rule, sphere average
    done analytically: e^{-i zeta.v'} averages to
    e^{-i zeta.(v - beta u/2)} sinc(beta |zeta| |u| / 2)."""
    v1, v2, v3 = inputs.velocity_nodes(N, L)
    V = np.stack([v1.ravel(), v2.ravel(), v3.ravel()], 1)
    f = f.reshape(-1)
    dv = 2 * L / N
    dz = math.pi / L
    U = V[:, None, :] - V[None, :, :]
    nu = np.linalg.norm(U, axis=2)
    ff = f[:, None] * f[None, :] * nu ** lam
    shift = V[:, None, :] - 0.5 * beta * U
    out = []
    for kk in kk_list:
        zeta = dz * (np.array(np.unravel_index(kk, (N,) * 3)) - N // 2)
        arg = 0.5 * beta * np.linalg.norm(zeta) * nu
        sinc = np.where(arg == 0, 1.0, np.sin(arg) / np.where(arg == 0, 1.0, arg))
        gain = np.sum(ff * sinc * np.exp(-1j * shift @ zeta))
        loss = np.sum(ff * np.exp(-1j * V @ zeta)[:, None])
        out.append((2 * math.pi) ** -1.5 * dv ** 6 * (gain - loss))
    return np.array(out)


@pytest.mark.slow
def test_inelastic_convolution_agrees_with_weak_form_quadrature():
    lam, beta = 1.0, 0.7
    errs = []
    for N in (12, 16):
        f = inputs.maxwellian(N, L, 0.6, (0.7, 0, 0), 0.6) + inputs.maxwellian(N, L, 0.4, (-0.7, 0.2, 0), 0.8)
        q = oracle.convolve(N, L, lam, oracle.dft_forward(N, L, f), beta=beta)[0]
        rng = np.random.default_rng(N)
        h = N // 2
        picks = [np.ravel_multi_index(tuple(rng.integers(h - 2, h + 3, 3)), (N,) * 3) for _ in range(6)]
        ref = weakform_qhat_beta(N, lam, beta, f, picks)
        errs.append(np.abs(q[picks] - ref).max() / np.abs(ref).max())
    assert errs[1] < errs[0] / 5, errs
    assert errs[1] < 5e-3, errs
