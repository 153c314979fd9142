"""FP64 CPU oracle for the conservative spectral collision operator (arXiv:1211.0540).

TEST INFRASTRUCTURE ONLY. This package is the independent, slow, plain
restatement of the method that the CUDA library is checked against. Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it; the library itself never does, and it shares no code with the
library. The arithmetic lives in ``bte_oracle.c`` (plain C, FP64); this module
only marshals numpy arrays through ctypes.

Every function cites the passage of the paper it restates (section and
equation label). Parity status of each function is listed in ``PINS`` below.
"""
import ctypes
import os

import numpy as np

from . import build as _build

__all__ = [
    "lib", "gauss_legendre", "sinc", "radial_I", "radial_J", "ghat_pair", "weights",
    "ghat_dense", "dft_forward_direct", "dft_forward", "dft_inverse", "convolve",
    "convolve_dense", "moments", "project", "collide", "rk2_homogeneous", "transport",
    "strang_step", "BC_DIFFUSE", "BC_SPECULAR", "BC_NOFLUX", "set_threads", "get_threads", "weights_beta",
]

BC_DIFFUSE = 0
BC_SPECULAR = 1
BC_NOFLUX = 2

# How each function is pinned to something other than itself (tests/test_oracle_*.py).
PINS = {
    "gauss_legendre": "numpy.polynomial.legendre.leggauss; exact on polynomials of degree 2n-1",
    "radial_I/radial_J/ghat_pair": "closed forms of the radial integrals for lambda=0,1 derived "
                                   "independently in the tests; 30-digit mpmath quadrature after "
                                   "r = u^(1/(lambda+3)) for variable hard and soft potentials "
                                   "(lambda in 0.1..0.75 and -0.5..-2.9); Ghat(xi,0)=0; symmetries",
    "weights": "table lookup == per-pair quadrature (lambda = 0, 1, 0.5, -1.5, -2.5)",
    "dft_forward(_direct)": "numpy FFT with centring phases; round trip; direct == separable",
    "dft_inverse": "round trip with dft_forward; numpy inverse FFT",
    "convolve": "Ghat == 1 reduces to scipy linear convolution; bilinearity; xi<->zeta-xi "
                "symmetry; Qhat(0) = 0; weak-form brute force (different discretisation)",
    "project": "CQ=0, P^2=P, minimal-norm (projection onto null(C)) via numpy lstsq",
    "collide": "Q(Maxwellian) -> 0 and BKW closed form, both converging in N",
    "rk2_homogeneous": "explicit Heun stages; conservation over 20 steps; second order in dt "
                       "(successive differences shrink by ~4 per halving)",
    "transport": "constant state, exact mass balance at the walls, second-order convergence",
    "transport(dx)": "uniform widths reproduce the uniform path bit for bit; constant state and "
                     "mass sum(dx f) kept on a stretched grid; second order on a smoothly stretched "
                     "grid; no-flux boundary invariants",
    "weights_beta / collide(beta)": "beta = 1 reproduces the elastic tables; weak-form brute force with the "
                                    "inelastic rule; energy dissipation -beta(1-beta)(rho E - |P|^2) for "
                                    "Maxwell molecules and its hard-sphere Maxwellian value, converging in N",
    "project(rows=4)": "CQ = 0 on the kept rows, idempotence, numpy lstsq on the 4 rows",
    "learned.indicator_pencils": "SplitMix64 published test vector; range and distinctness",
    "learned.learned_indicator": "numpy FFT + dense-weight gather evaluation; scale invariance",
}

_lib = None


def lib():
    """Load (building if needed) the oracle shared library."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    L = ctypes.CDLL(path)
    d = ctypes.c_double
    i = ctypes.c_int
    p = ctypes.c_void_p
    sig = {
        "ora_set_threads": (None, [i]),
        "ora_get_threads": (i, []),
        "ora_gauss_legendre": (i, [i, p, p]),
        "ora_sinc": (d, [d]),
        "ora_radial_I": (d, [d, d, d, d]),
        "ora_radial_J": (d, [d, d, d]),
        "ora_ghat_pair": (d, [i, d, d, p, p]),
        "ora_weights_sizes": (None, [i, p, p, p]),
        "ora_weights_build": (i, [i, d, d, p, p]),
        "ora_ghat_dense": (None, [i, p, p, i, p]),
        "ora_dft_forward_direct": (None, [i, d, p, p]),
        "ora_dft_forward": (None, [i, d, i, p, p]),
        "ora_dft_inverse": (None, [i, d, i, p, p, p]),
        "ora_convolve": (None, [i, d, i, p, p, i, p, p]),
        "ora_convolve_dense": (None, [i, d, i, p, p, p]),
        "ora_moments": (None, [i, d, i, p, p]),
        "ora_project": (None, [i, d, i, p]),
        "ora_collide": (None, [i, d, i, p, p, i, i, p, p, p, p]),
        "ora_rk2_homogeneous": (None, [i, d, i, p, p, d, d, p]),
        "ora_transport": (None, [i, d, i, d, d, i, i, d, d, d, p]),
        "ora_strang_step": (None, [i, d, i, d, d, i, i, d, d, p, p, d, d, p]),
        "ora_project_rows": (None, [i, d, i, i, p]),
        "ora_transport_grid": (None, [i, d, i, p, i, i, d, d, d, p]),
        "ora_strang_step_grid": (None, [i, d, i, p, i, i, d, d, p, p, d, d, p]),
        "ora_weights_sizes_beta": (None, [i, p, p]),
        "ora_weights_build_beta": (i, [i, d, d, d, p, p]),
        "ora_convolve_beta": (None, [i, d, i, p, p, i, p, p]),
        "ora_collide_beta": (None, [i, d, i, p, p, i, i, i, p, p, p, p]),
        "ora_rk2_homogeneous_beta": (None, [i, d, i, p, p, i, d, d, p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n):
    lib().ora_set_threads(int(n))


def get_threads():
    return int(lib().ora_get_threads())


def gauss_legendre(n):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().ora_gauss_legendre(n, _p(x), _p(w))
    return x, w


def sinc(x):
    return lib().ora_sinc(float(x))


def radial_I(lam, L, a, b):
    """int_0^L r^{lam+2} sinc(a r) sinc(b r) dr (Sec. 2.2, Eq. GHat_calc)."""
    return lib().ora_radial_I(float(lam), float(L), float(a), float(b))


def radial_J(lam, L, c):
    """int_0^L r^{lam+2} sinc(c r) dr (Sec. 2.2, Eq. GHat_calc)."""
    return lib().ora_radial_J(float(lam), float(L), float(c))


def ghat_pair(N, L, lam, k, m):
    """Ghat(xi_m, zeta_k) by direct quadrature of Eq. GHat_calc (grid of Eq. meshpoints)."""
    k = np.ascontiguousarray(k, dtype=np.int32)
    m = np.ascontiguousarray(m, dtype=np.int32)
    return lib().ora_ghat_pair(int(N), float(L), float(lam), _p(k), _p(m))


class Weights:
    """Radial integrals tabulated on the integer invariants of the grid."""

    def __init__(self, N, L, lam):
        np_, nq, ns = (ctypes.c_int(), ctypes.c_int(), ctypes.c_int())
        lib().ora_weights_sizes(int(N), ctypes.byref(np_), ctypes.byref(nq), ctypes.byref(ns))
        self.N, self.L, self.lam = int(N), float(L), float(lam)
        self.I = np.zeros((np_.value, nq.value))
        self.J = np.zeros(ns.value)
        rc = lib().ora_weights_build(self.N, self.L, self.lam, _p(self.I), _p(self.J))
        if rc != 0:
            raise ValueError("oracle: bad grid (N must be even and >= 2, L > 0)")


class WeightsBeta:
    """Inelastic weights (restitution parameter beta, Sec. 2.2): gain integrals on
    the invariants (|k'|^2, |m'|^2, k'.m'), loss integrals on |m'|^2 (N <= 16)."""

    def __init__(self, N, L, lam, beta):
        np_, nt = ctypes.c_int(), ctypes.c_int()
        lib().ora_weights_sizes_beta(int(N), ctypes.byref(np_), ctypes.byref(nt))
        self.N, self.L, self.lam, self.beta = int(N), float(L), float(lam), float(beta)
        self.I3 = np.zeros(np_.value * np_.value * nt.value)
        self.J = np.zeros(np_.value)
        rc = lib().ora_weights_build_beta(self.N, self.L, self.lam, self.beta, _p(self.I3), _p(self.J))
        if rc != 0:
            raise ValueError("oracle: bad inelastic grid (N even, 2 <= N <= 16, L > 0, 0 < beta <= 1)")


_weights_cache = {}
_weights_beta_cache = {}


def weights_beta(N, L, lam, beta):
    key = (int(N), float(L), float(lam), float(beta))
    if key not in _weights_beta_cache:
        _weights_beta_cache[key] = WeightsBeta(N, L, lam, beta)
    return _weights_beta_cache[key]


def weights(N, L, lam):
    key = (int(N), float(L), float(lam))
    if key not in _weights_cache:
        _weights_cache[key] = Weights(N, L, lam)
    return _weights_cache[key]


def ghat_dense(N, L, lam, part=0):
    """Dense M x M table G[k, m] = Ghat(xi_m, zeta_k) (small N only)."""
    w = weights(N, L, lam)
    M = N ** 3
    G = np.zeros((M, M))
    lib().ora_ghat_dense(int(N), _p(w.I), _p(w.J), int(part), _p(G))
    return G


def _cells(f, N):
    f = _f64(f)
    M = N ** 3
    if f.size % M:
        raise ValueError("array size is not a multiple of N^3")
    return f.reshape(-1, M), f.size // M


def dft_forward_direct(N, L, f):
    """Full triple sum for one cell (Sec. 3.2). Returns complex (M,)."""
    f = _f64(f).reshape(-1)
    out = np.zeros(2 * N ** 3)
    lib().ora_dft_forward_direct(int(N), float(L), _p(f), _p(out))
    return out.view(np.complex128)


def dft_forward(N, L, f):
    """fhat for each cell (Sec. 3.2); f: (ncells, M) real. Returns complex (ncells, M)."""
    f2, nc = _cells(f, N)
    out = np.zeros(2 * f2.size)
    lib().ora_dft_forward(int(N), float(L), nc, _p(f2), _p(out))
    return out.view(np.complex128).reshape(nc, -1)


def dft_inverse(N, L, qh):
    """Re of the inverse sum (Sec. 3.2). Returns (real (ncells, M), imag ratio (ncells,))."""
    qh = np.ascontiguousarray(qh, dtype=np.complex128).reshape(-1, N ** 3)
    nc = qh.shape[0]
    out = np.zeros((nc, N ** 3))
    ratio = np.zeros(nc)
    lib().ora_dft_inverse(int(N), float(L), nc, _p(qh.view(np.float64)), _p(out), _p(ratio))
    return out, ratio


def convolve(N, L, lam, fh, part=0, beta=1.0):
    """Qhat_k = dz^3 sum_m Ghat(xi_m, zeta_k) fhat_m fhat_{k-m+N/2} (Sec. 3.2);
    beta != 1: the inelastic weights (Sec. 2.2, Eq. GHat_calc with beta)."""
    fh = np.ascontiguousarray(fh, dtype=np.complex128).reshape(-1, N ** 3)
    out = np.zeros(fh.shape, dtype=np.complex128)
    if float(beta) != 1.0:
        w = weights_beta(N, L, lam, beta)
        lib().ora_convolve_beta(int(N), float(L), fh.shape[0], _p(w.I3), _p(w.J), int(part),
                                _p(fh.view(np.float64)), _p(out.view(np.float64)))
        return out
    w = weights(N, L, lam)
    lib().ora_convolve(int(N), float(L), fh.shape[0], _p(w.I), _p(w.J), int(part),
                       _p(fh.view(np.float64)), _p(out.view(np.float64)))
    return out


def convolve_dense(N, L, G, fh):
    fh = np.ascontiguousarray(fh, dtype=np.complex128).reshape(-1, N ** 3)
    G = _f64(G)
    out = np.zeros(fh.shape, dtype=np.complex128)
    lib().ora_convolve_dense(int(N), float(L), fh.shape[0], _p(G), _p(fh.view(np.float64)),
                             _p(out.view(np.float64)))
    return out


def moments(N, L, f):
    """(C f) per cell: mass, momentum (3), energy |v|^2 (Sec. 3.3)."""
    f2, nc = _cells(f, N)
    out = np.zeros((nc, 5))
    lib().ora_moments(int(N), float(L), nc, _p(f2), _p(out))
    return out


def project(N, L, Q, rows=5):
    """P_N Q = Q - C^T (C C^T)^{-1} C Q per cell (Sec. 3.3; sign reading), with the
    first `rows` rows of C: 5 = mass, momentum, energy; 4 = mass and momentum."""
    q2, nc = _cells(Q, N)
    q2 = q2.copy()
    lib().ora_project_rows(int(N), float(L), nc, int(rows), _p(q2))
    return q2


def collide(N, L, lam, f, part=0, project=True, want_raw=False, beta=1.0):
    """Q = P_N Qt(f) per cell. Returns Q (and Qt, imag ratio if want_raw).
    beta != 1: inelastic weights, projection on mass and momentum only (Sec. 3.3)."""
    f2, nc = _cells(f, N)
    Q = np.zeros_like(f2)
    raw = np.zeros_like(f2)
    ratio = np.zeros(nc)
    if float(beta) != 1.0:
        w = weights_beta(N, L, lam, beta)
        lib().ora_collide_beta(int(N), float(L), nc, _p(w.I3), _p(w.J), int(part), 4, int(bool(project)),
                               _p(f2), _p(Q), _p(raw), _p(ratio))
    else:
        w = weights(N, L, lam)
        lib().ora_collide(int(N), float(L), nc, _p(w.I), _p(w.J), int(part), int(bool(project)),
                          _p(f2), _p(Q), _p(raw), _p(ratio))
    if want_raw:
        return Q, raw, ratio
    return Q


def rk2_homogeneous(N, L, lam, f, dt, eps=1.0, beta=1.0):
    f2, nc = _cells(f, N)
    f2 = f2.copy()
    if float(beta) != 1.0:
        w = weights_beta(N, L, lam, beta)
        lib().ora_rk2_homogeneous_beta(int(N), float(L), nc, _p(w.I3), _p(w.J), 4, float(dt), float(eps),
                                       _p(f2))
        return f2
    w = weights(N, L, lam)
    lib().ora_rk2_homogeneous(int(N), float(L), nc, _p(w.I), _p(w.J), float(dt), float(eps),
                              _p(f2))
    return f2


def transport(N, L, f, tau, x0=0.0, x1=1.0, bc_left=BC_DIFFUSE, bc_right=BC_SPECULAR,
              Tw_left=1.0, Tw_right=1.0, dx=None):
    """Heun transport sub-step (Sec. 3.4) on nx uniform cells of [x0, x1], or on
    cells of widths dx (nx values) when given."""
    f2, nx = _cells(f, N)
    f2 = f2.copy()
    if dx is not None:
        dx = _f64(dx)
        if dx.size != nx or nx < 2:
            raise ValueError("dx needs one width per cell (nx >= 2)")
        lib().ora_transport_grid(int(N), float(L), nx, _p(dx), int(bc_left), int(bc_right),
                                 float(Tw_left), float(Tw_right), float(tau), _p(f2))
        return f2
    lib().ora_transport(int(N), float(L), nx, float(x0), float(x1), int(bc_left), int(bc_right),
                        float(Tw_left), float(Tw_right), float(tau), _p(f2))
    return f2


def strang_step(N, L, lam, f, dt, eps, x0=0.0, x1=1.0, bc_left=BC_DIFFUSE,
                bc_right=BC_SPECULAR, Tw_left=1.0, Tw_right=1.0, dx=None):
    f2, nx = _cells(f, N)
    f2 = f2.copy()
    w = weights(N, L, lam)
    if dx is not None:
        dx = _f64(dx)
        if dx.size != nx or nx < 2:
            raise ValueError("dx needs one width per cell (nx >= 2)")
        lib().ora_strang_step_grid(int(N), float(L), nx, _p(dx), int(bc_left), int(bc_right),
                                   float(Tw_left), float(Tw_right), _p(w.I), _p(w.J), float(dt),
                                   float(eps), _p(f2))
        return f2
    lib().ora_strang_step(int(N), float(L), nx, float(x0), float(x1), int(bc_left),
                          int(bc_right), float(Tw_left), float(Tw_right), _p(w.I), _p(w.J),
                          float(dt), float(eps), _p(f2))
    return f2
