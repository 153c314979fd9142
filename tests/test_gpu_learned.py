"""The learned mode against the oracle.

- Indicator parity: the GPU indicator (bte_learned_indicator) and the oracle's
  FP64 statement of it (oracle/learned.py) on the same host-made inputs f and
  Q, at N = 8 and 16; both draw the same pencils (SplitMix64 on each side).
  The indicator is a ratio of FP32 sums at the sampled modes: agreement
  |ind_gpu - ind_oracle| <= 1e-5 ind_oracle + 1e-6 (the FP32 operator's own
  error is ~1e-7 of the loss-term norm).
- Accuracy of the learned mode (the config-5 recipe): a width-1024 surrogate
  trained on 200k pairs the FP32 operator produces (30 epochs), run on 1024
  cells of the wall-heating slab with the fallback at 1e-2: every cell is
  within 1e-2 of the oracle (||Q - Q_oracle|| / ||Q_loss_oracle||) and
  conserves mass, momentum and energy to 1e-12. Measured on GB300: 27 cells
  fall back, max error 8.4e-3; the surrogate alone reaches 0.11, and its full
  error over its indicator has median 1.08 and max 2.3.
- Gain: on the same 1024 cells the learned mode evaluates more cells per
  second than the FP32 operator, each at its stated accuracy.
"""
import time

import numpy as np
import pytest

import oracle
from oracle import learned as olearned
from paper_1211_0540_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

L = 6.0


@pytest.fixture(scope="module")
def bte():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_0540_gb300 import bte as b
    return b


def loss_norm(N, lam, f):
    return np.linalg.norm(oracle.collide(N, L, lam, f, part=1, project=False), axis=1)


def moment_ok(N, Q):
    v1, v2, v3 = inputs.velocity_nodes(N, L)
    dv3 = (2 * L / N) ** 3
    C = dv3 * np.stack([np.ones(N ** 3), v1.ravel(), v2.ravel(), v3.ravel(), (v1 ** 2 + v2 ** 2 + v3 ** 2).ravel()])
    m = Q @ C.T
    return np.all(np.abs(m) <= 1e-12 * (np.abs(Q) @ np.abs(C).T))


@pytest.mark.parametrize("N", [8, 12, 16])
def test_indicator_sample_is_the_published_generator(bte, N):
    c = bte.Context(0)
    c.init_weights([(N, L, 1.0)])
    assert c.learned_sample() == olearned.indicator_pencils(N, seed=12345)
    c.close()


@pytest.mark.parametrize("N,ncells,lam,split", [(8, 40, 1.0, 4), (16, 37, 1.0, 4), (16, 33, 0.0, 4), (12, 35, 1.0, 1),
                                                (16, 38, 1.0, 1), (8, 41, -1.0, 2), (16, 160, 1.0, 4)])
def test_indicator_matches_oracle(bte, N, ncells, lam, split):
    f = inputs.homogeneous_cells(N, L, ncells, seed=600 + N + ncells)
    rng = np.random.default_rng(601 + N)
    Qo = oracle.collide(N, L, lam, f)
    # candidate values: exact, mildly and strongly perturbed, zero
    scale = np.ones((ncells, 1))
    scale[1::4] = 1.0 + 1e-3 * rng.standard_normal((len(scale[1::4]), 1))
    Q = Qo * scale * (1.0 + 0.02 * rng.standard_normal((ncells, N ** 3)) * (np.arange(ncells) % 4 == 2)[:, None])
    Q[3::4] = 0.0
    c = bte.Context(0)
    c.init_weights([(N, L, lam)])
    # the indicator's transform of f runs in the batch's configuration, or with one
    # CTA per cell once the cells fill the SMs (160 cells)
    c.set_option("dft_split", split)
    ind = c.learned_indicator(torch.from_numpy(f).cuda(), torch.from_numpy(np.ascontiguousarray(Q)).cuda())
    c.sync_status()
    got = ind.cpu().numpy()
    ref = olearned.learned_indicator(N, L, lam, f, Q, olearned.indicator_pencils(N, seed=12345))
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - ref) <= 1e-5 * ref + 1e-6), np.abs(got - ref).max()
    c.close()


def test_learned_mode_thresholds_the_indicator(bte):
    """BTE_LEARNED with an unreachable threshold returns P(Q_nn) for every cell
    and reports the indicator of exactly that output."""
    N, H = 8, 128
    c = bte.Context(0)
    c.init_weights([(N, L, 1.0)])
    c.mlp_init(0, H, seed=5)
    c.mlp_set_scales(10.0, 50.0)
    f = torch.from_numpy(inputs.homogeneous_cells(N, L, 40, seed=8)).cuda()
    c.set_option("learned_tol_ppm", 1 << 30)
    c.learned_stats(reset=True)
    Q = c.collide(f, mode=bte.LEARNED)
    st = c.learned_stats(reset=True)
    ind = c.learned_indicator(f, Q)
    c.sync_status()
    assert st["fallbacks"] == 0 and st["cells"] == 40
    assert abs(st["max_indicator"] - float(ind.max())) <= 1e-6 * float(ind.max())
    c.close()


def test_vacuum_cells_give_zero_in_the_learned_mode(bte):
    """Cells with f = 0 (rho = 0) beside ordinary ones: the surrogate takes x = 0
    for them, so Q is exactly 0 with or without the fallback; the ordinary
    cells get the same values as in a batch without vacuum cells."""
    N, H = 8, 128
    c = bte.Context(0)
    c.init_weights([(N, L, 1.0)])
    c.mlp_init(0, H, seed=5)
    c.mlp_set_scales(10.0, 50.0)
    f = inputs.homogeneous_cells(N, L, 40, seed=8)
    fz = f.copy()
    fz[[3, 17, 39]] = 0.0
    ft = torch.from_numpy(fz).cuda().reshape(-1)
    for fallback in (False, True):
        Q = c.collide(ft, mode=bte.LEARNED, fallback=fallback).cpu().numpy().reshape(40, -1)
        c.sync_status()
        assert np.all(Q[[3, 17, 39]] == 0.0), fallback
        assert np.all(np.isfinite(Q))
    Qs = c.collide(ft, mode=bte.LEARNED, fallback=False).cpu().numpy().reshape(40, -1)
    Qref = c.collide(torch.from_numpy(f).cuda().reshape(-1), mode=bte.LEARNED,
                     fallback=False).cpu().numpy().reshape(40, -1)
    keep = [i for i in range(40) if i not in (3, 17, 39)]
    assert np.array_equal(Qs[keep], Qref[keep])
    c.close()


@pytest.fixture(scope="module")
def trained(bte):
    """Width-1024 surrogate at N = 16 trained as config 5 prescribes (200k pairs
    the FP32 operator produces, 30 epochs), and the wall-heating slab of 1024
    cells after 100 Strang steps."""
    from paper_1211_0540_gb300 import surrogate
    N, lam, nx = 16, 1.0, 1024
    c = bte.Context(0)
    c.init_weights([(N, L, lam)])
    c.mlp_init(0, 1024, seed=1)
    t0 = time.perf_counter()
    f_tr, Q_tr = surrogate.make_training_set(c, N, L, 200000, seed=5)
    t1 = time.perf_counter()
    loss = surrogate.train(c, f_tr, Q_tr, N, L, epochs=30, batch=1024, lr=1e-3, seed=0)
    torch.cuda.synchronize()
    print("training set %.1f s, training %.1f s, final loss %.3e" % (t1 - t0, time.perf_counter() - t1, loss))
    del f_tr, Q_tr
    fw = torch.from_numpy(inputs.wall_heating_initial(N, L, nx)).cuda().reshape(-1)
    tr = dict(nx=nx, x0=0.0, x1=1.0, bc_left=bte.BC_DIFFUSE, bc_right=bte.BC_SPECULAR, Tw_left=2.0, Tw_right=1.0)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        for _ in range(100):
            c.step(fw, 0.5 * (1.0 / nx) / L, 0.1, transport=tr, mode=bte.FP32, stream=s)
    c.sync_status(s)
    f = fw.cpu().numpy().reshape(nx, -1)
    Qo = oracle.collide(N, L, lam, f)
    norm = loss_norm(N, lam, f)
    yield c, fw, f, Qo, norm
    c.close()


def test_learned_mode_is_within_1e2_of_the_oracle_on_every_cell(bte, trained):
    c, fw, f, Qo, norm = trained
    # the surrogate alone and its indicator on every cell (how well the sample tracks the full error)
    Qnn = c.collide(fw, mode=bte.LEARNED, fallback=False)
    ind = c.learned_indicator(fw, Qnn).cpu().numpy()
    e_nn = np.linalg.norm(Qnn.cpu().numpy().reshape(f.shape) - Qo, axis=1) / norm
    r = e_nn / ind
    print("surrogate alone: max err %.3e, median %.3e; err/indicator: max %.2f, median %.2f, "
          "cells with err > 1e-2 and indicator <= 1e-2: %d"
          % (e_nn.max(), np.median(e_nn), r.max(), np.median(r), int(np.sum((e_nn > 1e-2) & (ind <= 1e-2)))))
    c.set_option("learned_tol_ppm", 10000)
    c.learned_stats(reset=True)
    Q = c.collide(fw, mode=bte.LEARNED)
    st = c.learned_stats(reset=True)
    c.sync_status()
    Qg = Q.cpu().numpy().reshape(f.shape)
    err = np.linalg.norm(Qg - Qo, axis=1) / norm
    print("learned mode: max err %.3e, median %.3e, fallback %d of %d cells"
          % (err.max(), np.median(err), st["fallbacks"], st["cells"]))
    assert err.max() <= 1e-2, (err.max(), int(err.argmax()), st)
    assert st["fallbacks"] < st["cells"]  # the surrogate serves some cells
    assert moment_ok(16, Qg)


def test_learned_mode_gains_over_the_fp32_operator(bte, trained):
    c, fw, f, Qo, norm = trained
    s = torch.cuda.Stream()
    out = torch.empty_like(fw)

    def rate(mode, reps=20):
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            for _ in range(3):
                c.collide(fw, out, mode=mode, stream=s)
            s.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                c.collide(fw, out, mode=mode, stream=s)
            s.synchronize()
        return reps * f.shape[0] / (time.perf_counter() - t0)

    c.set_option("learned_tol_ppm", 10000)
    r_l = rate(bte.LEARNED)
    e_l = np.linalg.norm(out.cpu().numpy().reshape(f.shape) - Qo, axis=1) / norm
    r_f = rate(bte.FP32)
    e_f = np.linalg.norm(out.cpu().numpy().reshape(f.shape) - Qo, axis=1) / norm
    c.sync_status(s)
    print("learned %.3g evals/s (max err %.2e) vs FP32 %.3g evals/s (max err %.2e): gain %.2fx"
          % (r_l, e_l.max(), r_f, e_f.max(), r_l / r_f))
    assert e_l.max() <= 1e-2 and e_f.max() <= 1e-5
    assert r_l > r_f, (r_l, r_f)
