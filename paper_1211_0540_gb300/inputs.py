"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds only input recipes (where the distribution f is sampled and
with which random parameters). It contains none of the method's arithmetic and
imports neither the CUDA library nor the oracle, so both sides can be fed the
same arrays. Random numbers come from numpy's PCG64 generator with an explicit
seed; nothing here depends on the platform.

Velocity nodes follow the paper's mesh (Sec. 3.1, Eq. meshpoints):
v_j = dv (j - N/2), dv = 2L/N, j in [0, N)^3, cell layout k3 fastest.
"""
import math

import numpy as np

__all__ = [
    "velocity_nodes", "maxwellian", "bi_maxwellian", "bkw", "random_bi_maxwellian_params",
    "homogeneous_cells", "wall_heating_initial", "precision_sweep_cells", "uneven_batch",
    "training_states", "surrogate_training_states", "sudden_heating_grid",
]


def velocity_nodes(N, L):
    """(v1, v2, v3) arrays of shape (N, N, N) at the grid nodes."""
    dv = 2.0 * L / N
    g = dv * (np.arange(N) - N // 2)
    return np.meshgrid(g, g, g, indexing="ij")


def maxwellian(N, L, rho=1.0, u=(0.0, 0.0, 0.0), T=1.0):
    v1, v2, v3 = velocity_nodes(N, L)
    r2 = (v1 - u[0]) ** 2 + (v2 - u[1]) ** 2 + (v3 - u[2]) ** 2
    return (rho * (2.0 * math.pi * T) ** -1.5 * np.exp(-r2 / (2.0 * T))).reshape(-1)


def bi_maxwellian(N, L, rho1, u1, T1, rho2, u2, T2):
    return maxwellian(N, L, rho1, u1, T1) + maxwellian(N, L, rho2, u2, T2)


def bkw(N, L, K):
    """Bobylev-Krook-Wu profile at parameter K (density 1, zero mean):
    (2 pi K)^{-3/2} exp(-|v|^2/(2K)) [(5K-3)/(2K) + (1-K)|v|^2/(2K^2)]."""
    v1, v2, v3 = velocity_nodes(N, L)
    r2 = v1 ** 2 + v2 ** 2 + v3 ** 2
    g = (2.0 * math.pi * K) ** -1.5 * np.exp(-r2 / (2.0 * K))
    return (g * ((5.0 * K - 3.0) / (2.0 * K) + (1.0 - K) * r2 / (2.0 * K * K))).reshape(-1)


def random_bi_maxwellian_params(rng, mean_mode="x"):
    """rho1 ~ U(0.3, 0.7), rho2 = 1 - rho1, temperatures ~ U(0.5, 2).
    mean_mode "x": means +-U e_x with U ~ U(0.5, 1.5);
    mean_mode "cube": two independent means ~ U(-1.5, 1.5)^3."""
    rho1 = rng.uniform(0.3, 0.7)
    T1, T2 = rng.uniform(0.5, 2.0, size=2)
    if mean_mode == "x":
        U = rng.uniform(0.5, 1.5)
        u1, u2 = (U, 0.0, 0.0), (-U, 0.0, 0.0)
    else:
        u1 = tuple(rng.uniform(-1.5, 1.5, size=3))
        u2 = tuple(rng.uniform(-1.5, 1.5, size=3))
    return rho1, u1, T1, 1.0 - rho1, u2, T2


def homogeneous_cells(N, L, ncells, seed, mean_mode="x"):
    """ncells seeded bi-Maxwellians, shape (ncells, N^3), float64."""
    rng = np.random.default_rng(seed)
    out = np.empty((ncells, N ** 3))
    for c in range(ncells):
        out[c] = bi_maxwellian(N, L, *random_bi_maxwellian_params(rng, mean_mode))
    return out


def wall_heating_initial(N, L, nx):
    """Gas at rest, rho = 1, T = 1 in every cell (sudden wall heating, Sec. 5)."""
    m = maxwellian(N, L, 1.0, (0.0, 0.0, 0.0), 1.0)
    return np.tile(m, (nx, 1))


def sudden_heating_grid(X=20.0, dx_wall=0.125, wall_len=2.0, dx_bulk=0.5, ratio=1.2):
    """Cell widths of the paper's sudden-heating run (Sec. 5): eight cells per
    mean free path next to the wall, two in the interior (Knudsen number 1, so
    the mean free path is the unit length). Recipe: uniform dx_wall over
    [0, wall_len], then widths growing by `ratio` per cell up to dx_bulk, then
    equal cells no wider than dx_bulk up to X. Returns the widths (sum X)."""
    w = [dx_wall] * int(round(wall_len / dx_wall))
    x = sum(w)
    d = dx_wall * ratio
    while d < dx_bulk and x + d < X:
        w.append(d)
        x += d
        d *= ratio
    n = int(math.ceil((X - x) / dx_bulk - 1e-12))
    w += [(X - x) / n] * n
    return np.array(w)


def precision_sweep_cells(N, L, ncells, seed):
    """Bi-Maxwellians with means ~ U(-1.5, 1.5)^3 and temperatures ~ U(0.5, 2)."""
    return homogeneous_cells(N, L, ncells, seed, mean_mode="cube")


def uneven_batch(ninst, seed, L=6.0, Ns=(12, 16, 24, 32), pN=(0.4, 0.3, 0.2, 0.1),
                 lams=(0.0, 1.0), plam=(0.5, 0.5)):
    """Uneven batch of space-homogeneous instances: per instance N and lambda
    drawn with the given weights; lambda = 0 instances are BKW profiles
    (K ~ U(0.6, 0.95)) with probability 1/2, otherwise bi-Maxwellians.
    Returns a list of (N, lam, f) with f float64 of length N^3."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(ninst):
        N = int(rng.choice(Ns, p=pN))
        lam = float(rng.choice(lams, p=plam))
        if lam == 0.0 and rng.uniform() < 0.5:
            f = bkw(N, L, rng.uniform(0.6, 0.95))
        else:
            f = bi_maxwellian(N, L, *random_bi_maxwellian_params(rng, "x"))
        out.append((N, lam, f))
    return out


def training_states(N, L, nstates, seed, chunk=2048):
    """Seeded bi- and tri-Maxwellians (half each; means ~ U(-1.5, 1.5)^3,
    temperatures ~ U(0.5, 2), weights from a Dirichlet(1) draw), density 1.
    Vectorised over chunks of states."""
    rng = np.random.default_rng(seed)
    nb = np.where(rng.uniform(size=nstates) < 0.5, 2, 3)
    w = rng.dirichlet(np.ones(3), size=nstates)
    w[nb == 2, 2] = 0.0
    w /= w.sum(axis=1, keepdims=True)
    u = rng.uniform(-1.5, 1.5, size=(nstates, 3, 3))
    T = rng.uniform(0.5, 2.0, size=(nstates, 3))
    g1 = 2.0 * L / N * (np.arange(N) - N // 2)
    out = np.empty((nstates, N ** 3))
    for c0 in range(0, nstates, chunk):
        c1 = min(nstates, c0 + chunk)
        Tb = T[c0:c1, :, None, None]  # (n, 3 bumps, 1, 1)
        # the Maxwellian factorises over the three velocity components
        e = np.exp(-(g1[None, None, None, :] - u[c0:c1, :, :, None]) ** 2 / (2.0 * Tb))  # (n, 3, 3, N)
        amp = w[c0:c1] * (2.0 * math.pi * T[c0:c1]) ** -1.5  # (n, 3)
        g = np.einsum("nb,nbi,nbj,nbk->nijk", amp, e[:, :, 0], e[:, :, 1], e[:, :, 2], optimize=True)
        out[c0:c1] = g.reshape(c1 - c0, -1)
    return out


def surrogate_training_states(N, L, nstates, seed, chunk=2048):
    """Training distribution of the learned surrogate, three seeded families
    (density 1 each):
      - 40 %: bi-/tri-Maxwellians as in training_states;
      - 30 %: a Maxwellian (mean ~ U(-1, 1)^3, T ~ U(0.5, 2)) carrying 2-20 %
        of its mass in a second Maxwellian (mean offset ~ U(-1.5, 1.5)^3,
        T ~ U(0.5, 2)) -- states near equilibrium;
      - 30 %: half-range mixtures, a Maxwellian at T1 ~ U(0.5, 2) for v1 < 0 and
        one at T2 ~ U(0.5, 3) for v1 >= 0 (zero mean, masses ~ U(0.3, 0.7)
        of the total): the discontinuous distributions a diffuse wall emits."""
    rng = np.random.default_rng(seed)
    fam = rng.choice(3, size=nstates, p=[0.4, 0.3, 0.3])
    out = np.empty((nstates, N ** 3))
    i0 = np.flatnonzero(fam == 0)
    if i0.size:
        out[i0] = training_states(N, L, i0.size, int(rng.integers(1 << 31)), chunk)
    g1 = 2.0 * L / N * (np.arange(N) - N // 2)

    def maxw(u, T):  # (n, 3), (n,) -> (n, M), unit mass
        e = np.exp(-(g1[None, None, :] - u[:, :, None]) ** 2 / (2.0 * T[:, None, None]))
        a = (2.0 * math.pi * T) ** -1.5
        return np.einsum("n,ni,nj,nk->nijk", a, e[:, 0], e[:, 1], e[:, 2]).reshape(len(T), -1)

    i1 = np.flatnonzero(fam == 1)
    for c0 in range(0, i1.size, chunk):
        idx = i1[c0:c0 + chunk]
        n = idx.size
        u0 = rng.uniform(-1.0, 1.0, size=(n, 3))
        T0 = rng.uniform(0.5, 2.0, size=n)
        eps = rng.uniform(0.02, 0.2, size=n)
        u1 = u0 + rng.uniform(-1.5, 1.5, size=(n, 3))
        T1 = rng.uniform(0.5, 2.0, size=n)
        out[idx] = (1.0 - eps)[:, None] * maxw(u0, T0) + eps[:, None] * maxw(u1, T1)
    i2 = np.flatnonzero(fam == 2)
    v1 = np.repeat(g1, N * N)
    neg, pos = (v1 < 0.0)[None, :], (v1 >= 0.0)[None, :]
    for c0 in range(0, i2.size, chunk):
        idx = i2[c0:c0 + chunk]
        n = idx.size
        z = np.zeros((n, 3))
        T1 = rng.uniform(0.5, 2.0, size=n)
        T2 = rng.uniform(0.5, 3.0, size=n)
        m1 = rng.uniform(0.3, 0.7, size=n)
        A = maxw(z, T1) * neg
        B = maxw(z, T2) * pos
        dv3 = (2.0 * L / N) ** 3
        a = m1 / (A.sum(axis=1) * dv3)
        b = (1.0 - m1) / (B.sum(axis=1) * dv3)
        out[idx] = a[:, None] * A + b[:, None] * B
    return out
