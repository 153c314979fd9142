"""bte_collide_noalloc: the collision operator for callers that cannot allocate
GPU memory while they run (fixed memory budgets, or loops that must not be
synchronised by cudaMalloc/cudaFree). Its work area is a static device array
shared by all calls, so the test runs two calls in a row with different batch
sizes and data (stale contents of the first call must not leak into the
second) and checks each against bte_collide on the same input, with the
tolerance of the other parity tests (rel-L2 <= 1e-5 against the norm of the
oracle's loss term). This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1211_0540_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

L = 6.0
TOL32 = 1e-5


def test_noalloc_collide_matches_collide_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_0540_gb300 import bte
    lib = bte.load()
    N, lam = 16, 1.0
    ctx = bte.Context(0)
    ctx.init_weights([(N, L, lam)])
    stream = torch.cuda.current_stream()
    for ncells, seed in ((70, 31), (37, 32)):
        fnp = inputs.homogeneous_cells(N, L, ncells, seed=seed)
        f = torch.from_numpy(fnp).cuda()
        ref = ctx.collide(f, mode=bte.FP32)
        ctx.sync_status()
        Q = torch.full_like(f, float("nan"))
        rc = lib.bte_collide_noalloc(ctx._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(Q.data_ptr()),
                                     ncells, ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.bte_last_error(ctx._h)
        ctx.sync_status()
        got, want = Q.cpu().numpy(), ref.cpu().numpy()
        Qm = oracle.collide(N, L, lam, fnp, part=1, project=False)
        err = np.linalg.norm(got - want, axis=1) / np.linalg.norm(Qm, axis=1)
        assert np.all(np.isfinite(got))
        assert err.max() <= TOL32, err.max()
    # a request beyond the static work area is refused with a clear error
    big = torch.zeros((300, N ** 3), dtype=torch.float64, device="cuda")
    out = torch.zeros_like(big)
    rc = lib.bte_collide_noalloc(ctx._h, ctypes.c_void_p(big.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                 300, ctypes.c_void_p(stream.cuda_stream))
    assert rc == -1
    assert b"limit" in lib.bte_last_error(ctx._h)
    ctx.close()
