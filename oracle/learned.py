"""FP64 definition of the learned path's fallback indicator (test infrastructure).

The paper has no learned component. The library's learned mode replaces the
weighted convolution by a surrogate and checks each cell with a residual
indicator on a few sampled Fourier modes; this module states that indicator in
plain FP64 on top of the oracle's own transform and convolution (Sec. 3.2), so
that the GPU indicator can be compared with it on the same inputs.

Sampled modes. S = max(1, 64 // N) distinct zeta pencils (k1, k2), each with
all N values of k3. The pencil offsets k1' = k1 - N/2 and k2' = k2 - N/2 lie in
[-N/4, N/4] and are drawn from the SplitMix64 generator (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014) started at
`seed`: each offset is (next() mod (2q + 1)) - q with q = N/4, k1' first;
a pencil already drawn is skipped. Both sides implement this generator from
its published definition.

Indicator of one cell with distribution f and candidate operator value Q:
    ind = || F[Q](zeta_s) - Qhat(zeta_s) ||_2 / || Qhat^-(zeta_s) ||_2
over the sampled modes zeta_s, where F is the forward transform of Sec. 3.2,
Qhat = dz^3 sum_m Ghat(xi_m, zeta) fhat_m fhat_{k-m+N/2} is the weighted
convolution with the full weights and Qhat^- the same sum with the loss part
of the weights only (the denominator of the parity metric near equilibrium).
Pinned by a numpy evaluation through FFTs and a dense weight table
(tests/test_oracle_learned.py).
"""
import numpy as np

from . import convolve, dft_forward

MASK64 = (1 << 64) - 1


def splitmix64(seed):
    """Generator of SplitMix64 outputs from the 64-bit state `seed` (published constants)."""
    s = int(seed) & MASK64
    while True:
        s = (s + 0x9E3779B97F4A7C15) & MASK64
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        yield z ^ (z >> 31)


def indicator_pencils(N, seed=12345, modes=64):
    """The sampled pencils as grid indices kk = k1 N + k2, in drawing order."""
    h, q = N // 2, N // 4
    S = max(1, modes // N)
    g = splitmix64(seed)
    out = []
    while len(out) < S:
        k1 = int(next(g) % (2 * q + 1)) - q
        k2 = int(next(g) % (2 * q + 1)) - q
        kk = (k1 + h) * N + (k2 + h)
        if kk not in out:
            out.append(kk)
    return out


def sampled_modes(N, pencils):
    """Flat mode indices (k1 N + k2) N + k3 of the sampled pencils, k3 fastest."""
    return np.array([kk * N + k3 for kk in pencils for k3 in range(N)], dtype=np.int64)


def learned_indicator(N, L, lam, f, Q, pencils):
    """Indicator per cell (see the module docstring); f, Q: (ncells, N^3) FP64."""
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1, N ** 3)
    Q = np.ascontiguousarray(Q, dtype=np.float64).reshape(-1, N ** 3)
    idx = sampled_modes(N, pencils)
    fh = dft_forward(N, L, f)
    qfull = convolve(N, L, lam, fh, part=0)[:, idx]
    qloss = convolve(N, L, lam, fh, part=1)[:, idx]
    fq = dft_forward(N, L, Q)[:, idx]
    return np.linalg.norm(fq - qfull, axis=1) / np.linalg.norm(qloss, axis=1)
