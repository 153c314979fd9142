"""FP64 definition of the learned surrogate network (test infrastructure).

The paper has no learned component; this module states the library's
surrogate (a residual MLP on the normalised distribution) in plain numpy FP64
so that the GPU training and inference kernels can be checked against it:
    x = s_in f / rho (0 for rho = 0),  h1 = GELU(W1 x + b1),  h2 = h1 + GELU(W2 h1 + b2),
    y = W3 h2 + b3,    t = s_out Q / rho^2,   loss = mean((y - t)^2),
rho = sum f dv^3, GELU(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))).
Parameters are one flat vector W1 [H, M], b1, W2 [H, H], b2, W3 [M, H], b3.
Pinned by central finite differences (tests/test_oracle_mlp.py).
"""
import math

import numpy as np

K0 = math.sqrt(2.0 / math.pi)
K1 = 0.044715


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(K0 * (z + K1 * z ** 3)))


def gelu_grad(z):
    t = np.tanh(K0 * (z + K1 * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * K0 * (1.0 + 3.0 * K1 * z * z)


def split(p, M, H):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    out = []
    for shape in ((H, M), (H,), (H, H), (H,), (M, H), (M,)):
        n = int(np.prod(shape))
        out.append(p[o:o + n].reshape(shape))
        o += n
    assert o == p.size
    return out


def nparams(M, H):
    return H * M + H + H * H + H + M * H + M


def forward(p, f, dv3, s_in, M, H):
    W1, b1, W2, b2, W3, b3 = split(p, M, H)
    rho = f.sum(axis=1) * dv3
    # a vacuum cell (rho = 0) gets x = 0 (its output rho^2 y / s_out is 0 whatever y)
    scale = np.divide(s_in, rho, out=np.zeros_like(rho), where=rho != 0)
    x = f * scale[:, None]
    z1 = x @ W1.T + b1
    h1 = gelu(z1)
    z2 = h1 @ W2.T + b2
    h2 = h1 + gelu(z2)
    y = h2 @ W3.T + b3
    return dict(rho=rho, x=x, z1=z1, h1=h1, z2=z2, h2=h2, y=y)


def predict(p, f, dv3, s_in, s_out, M, H):
    c = forward(p, f, dv3, s_in, M, H)
    return c["y"] * (c["rho"] ** 2 / s_out)[:, None]


def loss_and_grads(p, f, Q, dv3, s_in, s_out, M, H):
    W1, b1, W2, b2, W3, b3 = split(p, M, H)
    c = forward(p, f, dv3, s_in, M, H)
    t = s_out * Q / (c["rho"] ** 2)[:, None]
    B = f.shape[0]
    d = c["y"] - t
    loss = float(np.mean(d * d))
    dy = 2.0 * d / (B * M)
    gW3 = dy.T @ c["h2"]
    gb3 = dy.sum(axis=0)
    dh2 = dy @ W3
    dz2 = dh2 * gelu_grad(c["z2"])
    gW2 = dz2.T @ c["h1"]
    gb2 = dz2.sum(axis=0)
    dh1 = dh2 + dz2 @ W2
    dz1 = dh1 * gelu_grad(c["z1"])
    gW1 = dz1.T @ c["x"]
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g
