"""bte_collide_noalloc: the collision operator for callers that cannot allocate
GPU memory while they run (fixed memory budgets, or loops that must not be
synchronised by cudaMalloc/cudaFree). Its work area is a static device array
shared by all calls, so each case runs two calls in a row with different
batch sizes and data (stale contents of the first call must not leak into the
second) and checks each against bte_collide on the same input, with the
tolerance of the other parity tests (rel-L2 <= 1e-5 against the norm of the
oracle's loss term). The second call of each case sits at the documented
maximum for its grid; one 32-cell group more is refused with a clear error;
a warm call changes neither the device's free memory nor the caller's current
device. This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1211_0540_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

L = 6.0
TOL32 = 1e-5
MAX_CELLS = {8: 2016, 12: 576, 16: 224}


@pytest.mark.parametrize("N", [8, 12, 16])
def test_noalloc_collide_matches_collide_on_two_calls(N):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_0540_gb300 import bte
    lib = bte.load()
    lam = 1.0
    ctx = bte.Context(0)
    ctx.init_weights([(N, L, lam)])
    stream = torch.cuda.current_stream()

    def noalloc(f, Q, n):
        return lib.bte_collide_noalloc(ctx._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(Q.data_ptr()), n,
                                       ctypes.c_void_p(stream.cuda_stream))

    for ncells, seed in ((70, 31 + N), (MAX_CELLS[N], 32 + N)):
        fnp = inputs.homogeneous_cells(N, L, ncells, seed=seed)
        f = torch.from_numpy(fnp).cuda()
        ref = ctx.collide(f, mode=bte.FP32)
        ctx.sync_status()
        Q = torch.full_like(f, float("nan"))
        rc = noalloc(f, Q, ncells)
        assert rc == 0, lib.bte_last_error(ctx._h)
        ctx.sync_status()
        got, want = Q.cpu().numpy(), ref.cpu().numpy()
        pick = np.unique(np.linspace(0, ncells - 1, 12).astype(int))
        Qm = oracle.collide(N, L, lam, fnp[pick], part=1, project=False)
        err = np.linalg.norm(got[pick] - want[pick], axis=1) / np.linalg.norm(Qm, axis=1)
        assert np.all(np.isfinite(got))
        assert err.max() <= TOL32, err.max()
        # every cell against bte_collide, relative to its own size
        assert np.abs(got - want).max() <= 1e-4 * np.abs(want).max()

    # a warm call: no device memory taken or given back, current device unchanged
    f = torch.from_numpy(inputs.homogeneous_cells(N, L, 70, seed=40 + N)).cuda()
    Q = torch.empty_like(f)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    dev0 = torch.cuda.current_device()
    assert noalloc(f, Q, 70) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.current_device() == dev0

    # one 32-cell group beyond the static work area is refused with a clear error
    n_big = MAX_CELLS[N] + 32
    big = torch.zeros((n_big, N ** 3), dtype=torch.float64, device="cuda")
    out = torch.zeros_like(big)
    assert noalloc(big, out, n_big) == -1
    assert b"limit" in lib.bte_last_error(ctx._h)
    ctx.close()
