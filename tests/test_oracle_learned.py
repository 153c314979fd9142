"""Pins of the oracle's learned-path indicator (oracle/learned.py).

- SplitMix64 reproduces the published test vector of its reference
  implementation (seed 1234567), so the sampled pencils are the generator's.
- The indicator is evaluated a second, independent way: transforms by numpy's
  FFT with the centring signs of Eq. meshpoints and the weighted convolution as
  an explicit gather over a dense weight table; both must agree to roundoff.
- Scaling: f -> a f, Q -> a^2 Q leaves the indicator unchanged (Q is bilinear).
"""
import math

import numpy as np

import oracle
from oracle import learned as olearned
from paper_1211_0540_gb300 import inputs

L = 6.0


def test_splitmix64_reference_vector():
    g = olearned.splitmix64(1234567)
    got = [next(g) for _ in range(5)]
    assert got == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                   4593380528125082431, 16408922859458223821]


def test_pencils_are_distinct_central_and_counted():
    for N in (8, 12, 16):
        pens = olearned.indicator_pencils(N, seed=12345)
        assert len(pens) == max(1, 64 // N) and len(set(pens)) == len(pens)
        for kk in pens:
            k1, k2 = kk // N - N // 2, kk % N - N // 2
            assert abs(k1) <= N // 4 and abs(k2) <= N // 4


def centred_fft(N, Lv, f):
    """fhat_k = (2 pi)^{-3/2} dv^3 sum_j f_j exp(-2 pi i k'.j'/N) through numpy's FFT:
    exp(-2 pi i (k-h)(j-h)/N) = (-1)^{k+j+h} exp(-2 pi i k j / N) per dimension (h = N/2)."""
    h = N // 2
    dv = 2 * Lv / N
    s = (-1.0) ** np.arange(N)
    sj = s[:, None, None] * s[None, :, None] * s[None, None, :]
    out = np.fft.fftn(f.reshape(-1, N, N, N) * sj, axes=(1, 2, 3)) * sj * ((-1.0) ** (3 * h))
    return (out * (2 * math.pi) ** -1.5 * dv ** 3).reshape(-1, N ** 3)


def dense_convolution(N, Lv, G, fh):
    """Qhat_k = dz^3 sum_m G[k, m] fhat_m fhat_{k-m+N/2}, terms off the grid dropped."""
    h = N // 2
    idx = np.indices((N, N, N)).reshape(3, -1).T
    n = idx[:, None, :] - idx[None, :, :] + h            # [k, m, d]
    valid = np.all((n >= 0) & (n < N), axis=2)
    nflat = np.where(valid, (n[..., 0] * N + n[..., 1]) * N + n[..., 2], 0)
    dz = math.pi / Lv
    out = np.empty_like(fh)
    for c in range(fh.shape[0]):
        prod = fh[c][None, :] * fh[c][nflat] * valid
        out[c] = dz ** 3 * np.sum(G * prod, axis=1)
    return out


def test_indicator_matches_numpy_evaluation():
    N, lam = 8, 1.0
    f = inputs.homogeneous_cells(N, L, 3, seed=41)
    rng = np.random.default_rng(42)
    Q = oracle.collide(N, L, lam, f) * (1.0 + 0.05 * rng.standard_normal((3, N ** 3)))
    pens = olearned.indicator_pencils(N, seed=12345)
    got = olearned.learned_indicator(N, L, lam, f, Q, pens)
    idx = olearned.sampled_modes(N, pens)
    fh = centred_fft(N, L, f)
    qf = dense_convolution(N, L, oracle.ghat_dense(N, L, lam, part=0), fh)[:, idx]
    ql = dense_convolution(N, L, oracle.ghat_dense(N, L, lam, part=1), fh)[:, idx]
    fq = centred_fft(N, L, Q)[:, idx]
    ref = np.linalg.norm(fq - qf, axis=1) / np.linalg.norm(ql, axis=1)
    assert np.all(ref > 1e-3)  # the perturbation makes the residual visible
    assert np.abs(got - ref).max() <= 1e-10 * ref.max()


def test_indicator_is_scale_invariant():
    N, lam = 8, 0.0
    f = inputs.homogeneous_cells(N, L, 2, seed=43)
    Q = oracle.collide(N, L, lam, f) * 1.1
    pens = olearned.indicator_pencils(N, seed=7)
    a = olearned.learned_indicator(N, L, lam, f, Q, pens)
    b = olearned.learned_indicator(N, L, lam, 3.0 * f, 9.0 * Q, pens)
    assert np.abs(a - b).max() <= 1e-12 * a.max()
