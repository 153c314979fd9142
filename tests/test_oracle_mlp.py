"""The FP64 surrogate definition's analytic gradient against central finite
differences on a tiny width (pins the oracle's backward pass)."""
import numpy as np

from oracle import mlp


def test_mlp_gradient_matches_central_differences():
    M, H, B = 8, 6, 5
    rng = np.random.default_rng(0)
    p = rng.standard_normal(mlp.nparams(M, H)) * 0.3
    f = rng.uniform(0.1, 1.0, (B, M))
    Q = rng.standard_normal((B, M)) * 0.1
    dv3, s_in, s_out = 0.7, 2.0, 3.0
    loss, g = mlp.loss_and_grads(p, f, Q, dv3, s_in, s_out, M, H)
    h = 1e-6
    idx = rng.choice(p.size, 40, replace=False)
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        lp, _ = mlp.loss_and_grads(p + e, f, Q, dv3, s_in, s_out, M, H)
        lm, _ = mlp.loss_and_grads(p - e, f, Q, dv3, s_in, s_out, M, H)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, g[i])
    assert loss > 0


def test_gelu_matches_tanh_form_and_derivative():
    z = np.linspace(-5, 5, 101)
    h = 1e-6
    assert np.allclose((mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h), mlp.gelu_grad(z), atol=1e-8)
    assert abs(mlp.gelu(0.0)) == 0.0 and abs(mlp.gelu(10.0) - 10.0) < 1e-12


def test_vacuum_cell_gives_zero_input_and_output():
    """A cell with rho = 0 (f = 0) takes x = 0 instead of 0/0, and its output
    rho^2 y / s_out is exactly 0; the other cells are unaffected (scale
    invariance of x = s_in f / rho is kept for them)."""
    M, H = 8, 6
    rng = np.random.default_rng(1)
    p = rng.standard_normal(mlp.nparams(M, H)) * 0.3
    f = rng.uniform(0.1, 1.0, (3, M))
    f[1] = 0.0
    c = mlp.forward(p, f, 0.7, 2.0, M, H)
    assert np.all(c["x"][1] == 0.0) and np.all(np.isfinite(c["y"]))
    q = mlp.predict(p, f, 0.7, 2.0, 3.0, M, H)
    assert np.all(q[1] == 0.0)
    f2 = f.copy()
    f2[0] *= 5.0  # x is invariant under scaling a cell
    assert np.allclose(mlp.forward(p, f2, 0.7, 2.0, M, H)["x"][0], c["x"][0], rtol=1e-14, atol=0)
