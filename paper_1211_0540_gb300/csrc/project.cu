// Conservation projection of Sec. 3.3 in FP64:
//   Q <- Q - C^T (C C^T)^{-1} C Q,  C_j = dv^3 (1, v1, v2, v3, |v|^2)_j.
// (The paper prints "Q = Qt + C (C C^T)^{-1} C Qt"; the Lagrange solution of
// its minimisation problem is the form above, which is what is computed.) The
// dv^3 factors cancel, so the kernel uses c_j = (1, v1, v2, v3, |v|^2) and the
// host-inverted 5x5 matrix A^{-1}, A = sum_j c_j c_j^T.
// One CTA per cell: the five moment sums are reduced in a fixed order (warp
// shuffles, then shared memory), so results are deterministic. The kernel can
// fuse the Heun update of the time step that consumes the projected Q.
#include "kernels.h"

namespace bte {

namespace {
constexpr int kProjThreads = 256;

__device__ __forceinline__ void cvec(int j, int N, double dv, double c[5]) {
    const int h = N / 2;
    const double v1 = dv * (j / (N * N) - h), v2 = dv * ((j / N) % N - h), v3 = dv * (j % N - h);
    c[0] = 1.0;
    c[1] = v1;
    c[2] = v2;
    c[3] = v3;
    c[4] = v1 * v1 + v2 * v2 + v3 * v3;
}

// Block-wide deterministic sum of 5 values; result valid in all threads.
__device__ __forceinline__ void block_sum5(double v[5]) {
    __shared__ double red[kProjThreads / 32][5];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 5; ++i)
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    if (lane == 0)
        for (int i = 0; i < 5; ++i) red[warp][i] = v[i];
    __syncthreads();
    for (int i = 0; i < 5; ++i) {
        double s = 0.0;
        for (int w = 0; w < kProjThreads / 32; ++w) s += red[w][i];
        v[i] = s;
    }
    __syncthreads();
}
}  // namespace

__global__ void __launch_bounds__(kProjThreads)
project_kernel(double *__restrict__ Q, const int64_t *__restrict__ slot_off, int s0, ProjArgs pa,
               int mode, const double *__restrict__ X, double *__restrict__ Y,
               const double *__restrict__ Qp, double a) {
    const int64_t off = slot_off[s0 + blockIdx.x];
    if (off < 0) return;
    const int N = pa.N, M = N * N * N;
    double *q = Q + off;
    double mu[5] = {0, 0, 0, 0, 0}, c[5];
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        cvec(j, N, pa.dv, c);
        const double x = q[j];
#pragma unroll
        for (int i = 0; i < 5; ++i) mu[i] += c[i] * x;
    }
    block_sum5(mu);
    double lam[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < 5; ++k) s += pa.ainv[i * 5 + k] * mu[k];
        lam[i] = s;
    }
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        cvec(j, N, pa.dv, c);
        double corr = 0.0;
#pragma unroll
        for (int i = 0; i < 5; ++i) corr += c[i] * lam[i];
        const double v = q[j] - corr;
        q[j] = v;
        if (mode == 1) Y[off + j] = X[off + j] + a * v;
        else if (mode == 2) Y[off + j] += a * (Qp[off + j] + v);
    }
}

__global__ void __launch_bounds__(kProjThreads)
moments_kernel(const double *__restrict__ f, const int64_t *__restrict__ slot_off, int s0, int N,
               double dv, const int64_t *__restrict__ slot_out, double *__restrict__ out) {
    const int64_t off = slot_off[s0 + blockIdx.x];
    if (off < 0) return;
    const int M = N * N * N;
    double mu[5] = {0, 0, 0, 0, 0}, c[5];
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        cvec(j, N, dv, c);
        const double x = f[off + j];
#pragma unroll
        for (int i = 0; i < 5; ++i) mu[i] += c[i] * x;
    }
    block_sum5(mu);
    if (threadIdx.x == 0) {
        const double w = dv * dv * dv;
        const int64_t o = slot_out[s0 + blockIdx.x];
        for (int i = 0; i < 5; ++i) out[5 * o + i] = w * mu[i];
    }
}

void launch_project(double *Q, const int64_t *slot_off, int s0, int nslots, const ProjArgs &pa,
                    int mode, const double *X, double *Y, const double *Qp, double a,
                    cudaStream_t st) {
    project_kernel<<<nslots, kProjThreads, 0, st>>>(Q, slot_off, s0, pa, mode, X, Y, Qp, a);
}

void launch_moments(const double *f, const int64_t *slot_off, int s0, int nslots, int N, double dv,
                    const int64_t *slot_out, double *out, cudaStream_t st) {
    moments_kernel<<<nslots, kProjThreads, 0, st>>>(f, slot_off, s0, N, dv, slot_out, out);
}

}  // namespace bte
