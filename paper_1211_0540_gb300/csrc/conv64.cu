// Plain FP64 weighted convolution (Sec. 3.2), the comparator operator:
//   Qhat(zeta_k) = sum_{m in box(k)} [Ghat(xi_m, zeta_k) dz^3] fhat_m fhat_{k-m+N/2},
// a direct double sum over the valid box of each zeta point with FP64
// weights and FP64 arithmetic. One warp per (32-cell group, zeta point), one
// lane per cell: the weight stream is warp-uniform and the fhat rows of the
// group layout are read coalesced. No symmetry, tiling or compensation.
#include "kernels.h"

namespace bte {

__global__ void conv64_plain_kernel(const double2 *__restrict__ F, double2 *__restrict__ Qh,
                                    const double *__restrict__ W,
                                    const uint64_t *__restrict__ Woff, int N, int64_t eoff) {
    const int lane = threadIdx.x & 31;
    const int M = N * N * N, h = N / 2;
    const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (k >= M) return;
    const int g = blockIdx.y;
    const double2 *Fg = F + eoff + (int64_t)g * M * kLanes;
    const int k1 = k / (N * N), k2 = (k / N) % N, k3 = k % N;
    const int lo1 = max(0, k1 - h + 1), hi1 = min(N - 1, k1 + h);
    const int lo2 = max(0, k2 - h + 1), hi2 = min(N - 1, k2 + h);
    const int lo3 = max(0, k3 - h + 1), hi3 = min(N - 1, k3 + h);
    const double *w = W + Woff[k];
    double re = 0.0, im = 0.0;
    for (int m1 = lo1; m1 <= hi1; ++m1)
        for (int m2 = lo2; m2 <= hi2; ++m2)
            for (int m3 = lo3; m3 <= hi3; ++m3) {
                const double g_ = *w++;
                const double2 a = Fg[(int64_t)((m1 * N + m2) * N + m3) * kLanes + lane];
                const int n = ((k1 - m1 + h) * N + (k2 - m2 + h)) * N + (k3 - m3 + h);
                const double2 b = Fg[(int64_t)n * kLanes + lane];
                re += g_ * (a.x * b.x - a.y * b.y);
                im += g_ * (a.x * b.y + a.y * b.x);
            }
    Qh[eoff + (int64_t)g * M * kLanes + (int64_t)k * kLanes + lane] = make_double2(re, im);
}

void launch_conv64(const double2 *F, double2 *Qh, const double *W, const uint64_t *Woff, int N,
                   int64_t eoff, int ngroups, cudaStream_t st) {
    const int M = N * N * N, warps = 4;
    dim3 grid((M + warps - 1) / warps, ngroups);
    conv64_plain_kernel<<<grid, warps * 32, 0, st>>>(F, Qh, W, Woff, N, eoff);
}

}  // namespace bte
