// Arithmetic-rate probes of the GPU (bte_alu_peak): the denominators that the
// collision operator's FP32 (and FP64) kernels are compared with.
//
// Every thread runs chains of dependent fused multiply-adds on 8 independent
// accumulators (enough to hide the pipe latency at 8 resident warps per SM
// sub-partition), fully unrolled, then stores one value so that the work is
// not removed. kind 0: scalar fma.rn.f32; kind 1: packed fma.rn.f32x2 (two
// FP32 FMAs per instruction); kind 2: fma.rn.f64. Rate = 2 flops per FMA over
// the event-timed duration of the launch.
#include <cuda_runtime.h>

#include <cstdint>

#include "bte_internal.h"

namespace bte {

namespace {

constexpr int kAcc = 8;
constexpr int kInner = 64;  // unrolled FMAs per accumulator per outer iteration

__global__ void __launch_bounds__(256) peak_f32_kernel(float *out, int iters, float a, float b) {
    float x[kAcc];
#pragma unroll
    for (int i = 0; i < kAcc; ++i) x[i] = (float)(threadIdx.x + i) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kInner; ++k)
#pragma unroll
            for (int i = 0; i < kAcc; ++i) x[i] = fmaf(x[i], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kAcc; ++i) s += x[i];
    if (s == 12345.678f) out[blockIdx.x] = s;  // never true for these inputs; keeps the work live
}

__global__ void __launch_bounds__(256) peak_f32x2_kernel(float *out, int iters, float a, float b) {
    uint64_t x[kAcc];
    uint64_t av, bv;
    asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
    for (int i = 0; i < kAcc; ++i) {
        const float v = (float)(threadIdx.x + i) * 1e-3f;
        asm("mov.b64 %0, {%1, %1};" : "=l"(x[i]) : "f"(v));
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kInner; ++k)
#pragma unroll
            for (int i = 0; i < kAcc; ++i) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[i]) : "l"(av), "l"(bv));
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kAcc; ++i) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[i]));
        s += lo + hi;
    }
    if (s == 12345.678f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) peak_f64_kernel(double *out, int iters, double a, double b) {
    double x[kAcc];
#pragma unroll
    for (int i = 0; i < kAcc; ++i) x[i] = (double)(threadIdx.x + i) * 1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kInner; ++k)
#pragma unroll
            for (int i = 0; i < kAcc; ++i) x[i] = fma(x[i], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kAcc; ++i) s += x[i];
    if (s == 12345.678) out[blockIdx.x] = s;
}

}  // namespace

}  // namespace bte

extern "C" bte_status bte_alu_peak(bte_ctx *c, int kind, double *tflops, double *ms_out, void *stream) {
    using namespace bte;
    if (!c || !tflops || kind < 0 || kind > 2) return BTE_EINVAL;
    cudaSetDevice(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int threads = 256, blocks = c->num_sms * 8;  // 2048 threads per SM: 16 warps per sub-partition
    const int iters = kind == 2 ? 40 : 400;
    double *sink = nullptr;
    if (cudaMalloc(&sink, sizeof(double) * blocks) != cudaSuccess) {
        cudaGetLastError();
        c->err = "bte_alu_peak: allocation";
        return BTE_ENOMEM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto launch = [&]() {
        if (kind == 0) peak_f32_kernel<<<blocks, threads, 0, st>>>((float *)sink, iters, 0.999999f, 1e-7f);
        else if (kind == 1) peak_f32x2_kernel<<<blocks, threads, 0, st>>>((float *)sink, iters, 0.999999f, 1e-7f);
        else peak_f64_kernel<<<blocks, threads, 0, st>>>(sink, iters, 0.999999999, 1e-12);
    };
    launch();  // warm-up (clocks, instruction cache)
    cudaEventRecord(e0, st);
    const int reps = 5;
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->err = std::string("bte_alu_peak: ") + cudaGetErrorString(e);
        return BTE_ECUDA;
    }
    const double fmas = (double)reps * blocks * threads * iters * kInner * kAcc * (kind == 1 ? 2.0 : 1.0);
    *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms / reps;
    return BTE_OK;
}
