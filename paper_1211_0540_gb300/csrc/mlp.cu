// Learned surrogate of the collision operator: residual MLP trained on (f, Q(f))
// pairs produced by the operator itself, with BF16 tensor-core GEMMs (gemm_tc.cu).
#include <cuda_bf16.h>

#include <string>

#include "gemm_tc.h"
#include "kernels.h"

using namespace bte;

namespace {
bte_status mlp_fail(bte_ctx *c, bte_status s, const std::string &m) {
    cudaGetLastError();
    if (c) c->err = m;
    return s;
}
}  // namespace

extern "C" bte_status bte_tc_gemm(bte_ctx *c, const void *A, const void *B, float *D, int M, int N, int K,
                                  const float *bias, int gelu, void *D_bf16, void *D_bf16_t, int ld_t,
                                  void *stream) {
    if (!c || !A || !B) return BTE_EINVAL;
    cudaSetDevice(c->device);
    cudaError_t e = gemm_bf16_prepare();
    if (e != cudaSuccess) return mlp_fail(c, BTE_ECUDA, std::string("gemm prepare: ") + cudaGetErrorString(e));
    GemmEpi g;
    g.bias = bias;
    g.out_f32 = D;
    g.ld_f32 = N;
    g.act = gelu ? GEMM_ACT_GELU : GEMM_ACT_NONE;
    g.out_bf16 = (__nv_bfloat16 *)D_bf16;
    g.ld_bf16 = N;
    g.out_bf16_t = (__nv_bfloat16 *)D_bf16_t;
    g.ld_t = ld_t;
    if (D_bf16_t && ld_t < M) return mlp_fail(c, BTE_EINVAL, "bte_tc_gemm: ld_t < M");
    int r = gemm_bf16(A, B, M, N, K, g, c->d_status, (cudaStream_t)stream);
    if (r == -1) return mlp_fail(c, BTE_EINVAL, "bte_tc_gemm: need K % 64 == 0 and N % 64 == 0");
    if (r == -2) return mlp_fail(c, BTE_ECUDA, "bte_tc_gemm: tensor map encoding failed");
    if (r != 0) return mlp_fail(c, BTE_ECUDA, "bte_tc_gemm: launch failed");
    return BTE_OK;
}
