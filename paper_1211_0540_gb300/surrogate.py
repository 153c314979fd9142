"""Training and evaluation workflow of the learned collision surrogate.

The surrogate (a residual MLP, see bte.h) is trained on (f, Q(f)) pairs that
the FP32 operator of this library produces: seeded bi-/tri-Maxwellians,
near-equilibrium and half-range (wall-like) mixtures, and states partially
relaxed by 1..40 Heun steps of the homogeneous problem. All
arithmetic runs in libbte (operator, training kernels, inference); this module
only chooses the data recipe and calls the C ABI through the binding.
"""
import numpy as np

from . import bte, inputs


def make_training_set(ctx, N, L, n_states, seed, relax_fraction=0.4, dt=0.05, max_steps=40,
                      chunk=8192):
    """Return device tensors (f, Q) with n_states cells each (FP64)."""
    import torch
    M = N ** 3
    f = torch.from_numpy(inputs.surrogate_training_states(N, L, n_states, seed)).cuda().reshape(-1)
    rng = np.random.default_rng(seed + 1)
    n_relax = int(relax_fraction * n_states)
    if n_relax:
        # relax the first n_relax states by a seeded number of Heun steps (in groups of equal count)
        steps = rng.integers(1, max_steps + 1, size=n_relax)
        order = np.argsort(steps, kind="stable")
        f_rel = f[:n_relax * M].view(n_relax, M)
        done = 0
        s = torch.cuda.Stream()
        for k in range(1, max_steps + 1):
            idx = order[steps[order] >= k]
            if idx.size == 0:
                break
            sub = f_rel[torch.from_numpy(idx).cuda()].contiguous().view(-1)
            with torch.cuda.stream(s):
                ctx.step(sub, dt, 1.0, mode=bte.FP32, stream=s)
            s.synchronize()
            f_rel[torch.from_numpy(idx).cuda()] = sub.view(-1, M)
            done += 1
    Q = torch.empty_like(f)
    for c0 in range(0, n_states, chunk):
        c1 = min(n_states, c0 + chunk)
        ctx.collide(f[c0 * M:c1 * M], Q[c0 * M:c1 * M], mode=bte.FP32)
    ctx.sync_status()
    return f, Q


def train(ctx, f, Q, N, L, epochs=20, batch=1024, lr=1e-3, weight_decay=0.0, seed=0, s_in=10.0):
    """Scales fitted by the library (unit-RMS targets), then AdamW training."""
    ctx.mlp_fit_scales(f, Q, s_in)
    return ctx.mlp_train(f, Q, epochs=epochs, batch=batch, lr=lr, weight_decay=weight_decay, seed=seed)


def relative_errors(Q_test, Q_ref, norm):
    """Per-cell ||Q_test - Q_ref|| / norm (norm: per-cell array)."""
    d = (Q_test - Q_ref).reshape(len(norm), -1)
    return np.linalg.norm(d, axis=1) / norm
