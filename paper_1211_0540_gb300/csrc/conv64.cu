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

// Few cells (a partly filled group): one warp per (cell, zeta point), the lanes
// split the box sum (term q = lane, lane + 32, ... in the box's m1, m2, m3
// order) and the partial sums are added by a fixed shuffle tree. The same
// plain FP64 sum, with every lane doing useful work when the group is not
// full (one cell would otherwise cost as much as 32).
__global__ void conv64_cells_kernel(const double2 *__restrict__ F, double2 *__restrict__ Qh,
                                    const double *__restrict__ W, const uint64_t *__restrict__ Woff,
                                    const int64_t *__restrict__ slot_off, int s0, int N, int64_t eoff) {
    const int lane = threadIdx.x & 31;
    const int M = N * N * N, h = N / 2;
    const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (k >= M) return;
    const int slot = blockIdx.y;  // slot within the segment
    if (slot_off[s0 + slot] < 0) return;
    const int g = slot / kLanes, cl = slot % kLanes;
    const double2 *Fg = F + eoff + (int64_t)g * M * kLanes + cl;
    const int k1 = k / (N * N), k2 = (k / N) % N, k3 = k % N;
    const int lo1 = max(0, k1 - h + 1), hi1 = min(N - 1, k1 + h);
    const int lo2 = max(0, k2 - h + 1), hi2 = min(N - 1, k2 + h);
    const int lo3 = max(0, k3 - h + 1), hi3 = min(N - 1, k3 + h);
    const int l2 = hi2 - lo2 + 1, l3 = hi3 - lo3 + 1, nt = (hi1 - lo1 + 1) * l2 * l3;
    const double *w = W + Woff[k];
    double re = 0.0, im = 0.0;
    for (int q = lane; q < nt; q += 32) {
        const int m1 = lo1 + q / (l2 * l3), m2 = lo2 + (q / l3) % l2, m3 = lo3 + q % l3;
        const double g_ = w[q];
        const double2 a = Fg[(int64_t)((m1 * N + m2) * N + m3) * kLanes];
        const int n = ((k1 - m1 + h) * N + (k2 - m2 + h)) * N + (k3 - m3 + h);
        const double2 b = Fg[(int64_t)n * kLanes];
        re += g_ * (a.x * b.x - a.y * b.y);
        im += g_ * (a.x * b.y + a.y * b.x);
    }
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) Qh[eoff + (int64_t)g * M * kLanes + (int64_t)k * kLanes + cl] = make_double2(re, im);
}

void launch_conv64_cells(const double2 *F, double2 *Qh, const double *W, const uint64_t *Woff,
                         const int64_t *slot_off, int s0, int nslots, int N, int64_t eoff, cudaStream_t st) {
    const int M = N * N * N, warps = 4;
    dim3 grid((M + warps - 1) / warps, nslots);
    conv64_cells_kernel<<<grid, warps * 32, 0, st>>>(F, Qh, W, Woff, slot_off, s0, N, eoff);
}

void launch_conv64(const double2 *F, double2 *Qh, const double *W, const uint64_t *Woff, int N,
                   int64_t eoff, int ngroups, cudaStream_t st) {
    const int M = N * N * N, warps = 4;
    dim3 grid((M + warps - 1) / warps, ngroups);
    conv64_plain_kernel<<<grid, warps * 32, 0, st>>>(F, Qh, W, Woff, N, eoff);
}

}  // namespace bte
