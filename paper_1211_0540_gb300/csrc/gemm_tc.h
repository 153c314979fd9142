// BF16 tensor-core GEMM (tcgen05 + TMA) with a fused epilogue (internal).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace bte {

enum { GEMM_ACT_NONE = 0, GEMM_ACT_GELU = 1 };

// Epilogue of D = alpha * A B^T, applied per element (row, col) in this order:
//   v = alpha * D + bias[col];  out_f32 = v;  v = act(v);  v += residual;
//   out_bf16 = bf16(v);  out_bf16_t[col * ld_t + row] = bf16(v).
// Any output pointer may be null.
struct GemmEpi {
    float alpha = 1.f;
    const float *bias = nullptr;
    float *out_f32 = nullptr;
    int ld_f32 = 0;
    int act = GEMM_ACT_NONE;
    const __nv_bfloat16 *residual = nullptr;
    int ld_res = 0;
    __nv_bfloat16 *out_bf16 = nullptr;
    int ld_bf16 = 0;
    __nv_bfloat16 *out_bf16_t = nullptr;
    int ld_t = 0;
};

cudaError_t gemm_bf16_prepare();  // outside stream capture
// 0 on success; -1 bad shape, -2 tensor map, -3 launch error.
int gemm_bf16(const void *A, const void *B, int M, int N, int K, const GemmEpi &g, int *status, cudaStream_t st);

}  // namespace bte
