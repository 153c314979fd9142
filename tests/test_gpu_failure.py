"""Failure detection without a GPU fault: every wait of the convolution kernel
is bounded (one second of the global timer); when it runs out the kernel
records BTE_ETIMEOUT in the status word, drains its own copies and returns,
and the context stays usable. The test makes the waits run out through the
test-only option debug_conv_stall (the first block's copies are never
issued, so nothing completes the barrier phase being waited on)."""
import time

import numpy as np
import pytest

import oracle
from paper_1211_0540_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
L = 6.0


@pytest.fixture(scope="module")
def bte():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_0540_gb300 import bte as b
    return b


@pytest.mark.parametrize("impl", [2, 4])  # sums in registers / in shared memory
def test_bounded_wait_reports_timeout_and_context_recovers(bte, impl):
    N, lam = 8, 1.0
    c = bte.Context(0)
    c.init_weights([(N, L, lam)])
    c.set_option("conv_impl", impl)
    f = inputs.homogeneous_cells(N, L, 40, seed=41)
    ft = torch.from_numpy(f).cuda()
    s = torch.cuda.Stream()
    c.set_option("debug_conv_stall", 1)
    t0 = time.time()
    c.collide(ft, stream=s)
    with pytest.raises(bte.BteError) as err:
        c.sync_status(s)
    elapsed = time.time() - t0
    assert err.value.code == -4, str(err.value)  # BTE_ETIMEOUT
    assert elapsed < 60.0, elapsed  # bounded: about two seconds per stalled warp
    c.set_option("debug_conv_stall", 0)
    Q = c.collide(ft, stream=s)
    c.sync_status(s)  # the status word was cleared by the read above
    Qo = oracle.collide(N, L, lam, f)
    Qm = oracle.collide(N, L, lam, f, part=1, project=False)
    rel = np.linalg.norm(Q.cpu().numpy() - Qo, axis=1) / np.linalg.norm(Qm, axis=1)
    assert rel.max() <= 1e-5, rel.max()
    c.close()
