// Learned collision path (mode BTE_LEARNED): surrogate -> conservation
// projection -> residual indicator -> exact fallback.
//
// Indicator (per cell). The exact operator is evaluated at S sampled Fourier
// modes zeta_k (fixed, seeded, drawn from |k'|_inf <= N/4 without zeta = 0):
//   Qhat(k)  = sum_m Ghat(xi_m, zeta_k) dz^3 fhat_m fhat_{k-m+N/2}     (Sec. 3.2)
//   Qhat-(k) = the same sum with the loss term of Ghat only,
// and compared with the forward transform of the projected surrogate output:
//   ind = ||Fhat[P Q_nn](k) - Qhat(k)||_S / ||Qhat-(k)||_S,
// i.e. the parity metric of the fast path restricted to S modes. Cells with
// ind > tol are recomputed with the FP32 operator. Cost of the check: S
// zeta points out of N^3 of the convolution (64 / 4096 = 1.6 % at N = 16).
#include <algorithm>
#include <cmath>
#include <random>
#include <vector>

#include "kernels.h"
#include "learned.h"

namespace bte {

namespace {

// One warp per (sample, group): lane = cell. Accumulates the exact and loss
// sums at the sampled mode and the squared differences.
__global__ void __launch_bounds__(32) indicator_kernel(const float2 *__restrict__ F, const float2 *__restrict__ QN,
                                                       const float2 *__restrict__ W, const int *__restrict__ woff,
                                                       const int *__restrict__ kidx, int N, int64_t eoff,
                                                       int nslots, float *err2, float *den2) {
    const int s = blockIdx.x, g = blockIdx.y, lane = threadIdx.x;
    const int M = N * N * N, h = N / 2;
    const int k = kidx[s];
    const int k1 = k / (N * N), k2 = (k / N) % N, k3 = k % N;
    const float2 *Fg = F + eoff + (int64_t)g * M * kLanes;
    const float2 *w = W + woff[s];
    float fr = 0.f, fi = 0.f, lr = 0.f, li = 0.f;
    for (int m1 = max(0, k1 - h + 1); m1 <= min(N - 1, k1 + h); ++m1)
        for (int m2 = max(0, k2 - h + 1); m2 <= min(N - 1, k2 + h); ++m2)
            for (int m3 = max(0, k3 - h + 1); m3 <= min(N - 1, k3 + h); ++m3) {
                const float2 ww = *w++;
                const float2 a = Fg[(int64_t)((m1 * N + m2) * N + m3) * kLanes + lane];
                const int n = ((k1 - m1 + h) * N + (k2 - m2 + h)) * N + (k3 - m3 + h);
                const float2 b = Fg[(int64_t)n * kLanes + lane];
                const float pr = a.x * b.x - a.y * b.y, pi = a.x * b.y + a.y * b.x;
                fr = fmaf(ww.x, pr, fr);
                fi = fmaf(ww.x, pi, fi);
                lr = fmaf(ww.y, pr, lr);
                li = fmaf(ww.y, pi, li);
            }
    const float2 q = QN[eoff + (int64_t)g * M * kLanes + (int64_t)k * kLanes + lane];
    const float dr = q.x - fr, di = q.y - fi;
    const int slot = g * kLanes + lane;
    err2[(size_t)s * nslots + slot] = dr * dr + di * di;
    den2[(size_t)s * nslots + slot] = lr * lr + li * li;
}

__global__ void indicator_reduce_kernel(const float *__restrict__ err2, const float *__restrict__ den2, int S,
                                        int nslots, int nvalid, float *ind) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nslots) return;
    float e = 0.f, d = 0.f;
    for (int s = 0; s < S; ++s) {
        e += err2[(size_t)s * nslots + c];
        d += den2[(size_t)s * nslots + c];
    }
    ind[c] = c < nvalid ? sqrtf(e) / fmaxf(sqrtf(d), 1e-30f) : 0.f;
}

}  // namespace

int build_indicator_table(const Table &t, int S, uint64_t seed, IndicatorTable &out) {
    const int N = t.N, h = N / 2, q = N / 4;
    const double dz3 = t.dz * t.dz * t.dz;
    const double c = std::sqrt(2.0 / 3.14159265358979323846);
    std::mt19937_64 rng(seed);
    std::uniform_int_distribution<int> d(-q, q);
    std::vector<int> ks;
    while ((int)ks.size() < S) {
        const int a = d(rng), b = d(rng), e = d(rng);
        if (a == 0 && b == 0 && e == 0) continue;
        const int k = ((a + h) * N + (b + h)) * N + (e + h);
        if (std::find(ks.begin(), ks.end(), k) == ks.end()) ks.push_back(k);
    }
    std::vector<float2> w;
    std::vector<int> off;
    for (int k : ks) {
        off.push_back((int)w.size());
        const int k1 = k / (N * N), k2 = (k / N) % N, k3 = k % N;
        for (int m1 = std::max(0, k1 - h + 1); m1 <= std::min(N - 1, k1 + h); ++m1)
            for (int m2 = std::max(0, k2 - h + 1); m2 <= std::min(N - 1, k2 + h); ++m2)
                for (int m3 = std::max(0, k3 - h + 1); m3 <= std::min(N - 1, k3 + h); ++m3) {
                    const int s = (m1 - h) * (m1 - h) + (m2 - h) * (m2 - h) + (m3 - h) * (m3 - h);
                    const double full = t.ghat(k1, k2, k3, m1, m2, m3) * dz3;
                    const double loss = -c * t.J[s] * dz3;
                    w.push_back(make_float2((float)full, (float)loss));
                }
    }
    out.S = S;
    cudaError_t e = cudaMalloc(&out.d_w, sizeof(float2) * w.size());
    if (e == cudaSuccess) e = cudaMalloc(&out.d_off, sizeof(int) * S);
    if (e == cudaSuccess) e = cudaMalloc(&out.d_k, sizeof(int) * S);
    if (e == cudaSuccess) e = cudaMemcpy(out.d_w, w.data(), sizeof(float2) * w.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(out.d_off, off.data(), sizeof(int) * S, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(out.d_k, ks.data(), sizeof(int) * S, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return 0;
}

void free_indicator_table(IndicatorTable &t) {
    cudaFree(t.d_w);
    cudaFree(t.d_off);
    cudaFree(t.d_k);
    t.d_w = nullptr;
    t.d_off = nullptr;
    t.d_k = nullptr;
}

void launch_indicator(const IndicatorTable &it, const float2 *F, const float2 *QN, int N, int64_t eoff, int nslots,
                      int nvalid, float *err2, float *den2, float *ind, cudaStream_t st) {
    dim3 grid(it.S, nslots / kLanes);
    indicator_kernel<<<grid, 32, 0, st>>>(F, QN, it.d_w, it.d_off, it.d_k, N, eoff, nslots, err2, den2);
    indicator_reduce_kernel<<<(nslots + 255) / 256, 256, 0, st>>>(err2, den2, it.S, nslots, nvalid, ind);
}

}  // namespace bte
