"""Tensor-core BF16 GEMM (tcgen05 + TMA) against an FP64 reference of the same
operation on bf16-representable inputs. Products of bf16 values are exact in
FP32, so the only error is FP32 accumulation: bound 1e-5 relative to the
row-scale of |A||B|^T; bf16 outputs add one bf16 rounding (2^-8)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(math.sqrt(2.0 / math.pi) * (x + 0.044715 * x ** 3)))


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_0540_gb300 import bte
    c = bte.Context(0)
    yield c
    c.close()


def bf16(rng, shape, scale=1.0):
    t = torch.from_numpy(rng.standard_normal(shape).astype(np.float32) * scale).to(torch.bfloat16)
    return t, t.float().numpy().astype(np.float64)


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (300, 256, 512), (77, 64, 128), (1024, 1024, 4096),
                                   (256, 4096, 1024), (1024, 4096, 1024), (896, 4096, 512)])
def test_gemm_matches_fp64(ctx, M, N, K):
    rng = np.random.default_rng(M + N + K)
    A, An = bf16(rng, (M, K))
    B, Bn = bf16(rng, (N, K))
    D, _, _ = ctx.tc_gemm(A.cuda(), B.cuda())
    ctx.sync_status()
    ref = An @ Bn.T
    scale = np.abs(An) @ np.abs(Bn).T
    err = np.abs(D.cpu().numpy().astype(np.float64) - ref) / scale
    assert err.max() <= 1e-5, err.max()


def test_gemm_epilogue_bias_gelu_transposed(ctx):
    M, N, K = 200, 192, 256
    rng = np.random.default_rng(9)
    A, An = bf16(rng, (M, K), 0.1)
    B, Bn = bf16(rng, (N, K), 0.1)
    bias = torch.from_numpy(rng.standard_normal(N).astype(np.float32))
    D, Db, Dt = ctx.tc_gemm(A.cuda(), B.cuda(), bias=bias.cuda(), gelu=True, out_bf16=True, out_bf16_t=True)
    ctx.sync_status()
    pre = An @ Bn.T + bias.numpy().astype(np.float64)
    scale = np.abs(An) @ np.abs(Bn).T + np.abs(pre)
    assert (np.abs(D.cpu().numpy() - pre) / scale).max() <= 1e-5
    act = gelu(pre)
    got = Db.float().cpu().numpy()
    assert np.abs(got - act).max() <= 2.0 ** -7 * np.abs(act).max() + 1e-6
    assert np.array_equal(Dt.float().cpu().numpy().T, got)
