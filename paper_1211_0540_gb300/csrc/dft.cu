// Centred discrete Fourier transforms of Sec. 3.2 on the grid of Eq. meshpoints,
// one dimension per pass:
//   fhat_k = (2 pi)^{-3/2} dv^3 sum_j f_j exp(-i zeta_k . v_j),
//   Qt_j   = Re (2 pi)^{-3/2} dz^3 sum_k Qhat_k exp(+i zeta_k . v_j),
// with zeta_k . v_j = (2 pi / N) sum_d (k_d - N/2)(j_d - N/2): the phase index
// t = (k' j') mod N selects root[t] = exp(2 pi i t / N).
//
// Layouts. f and Qt are the caller's FP64 cell arrays (per-slot element
// offsets, -1 for the padding slots of a 32-cell group). Intermediate passes
// use a cell-major complex scratch [slot][M]. fhat and Qhat use the group
// layout of the convolution kernel: [group][m][lane], lane = slot % 32, so a
// warp reads one grid point of 32 cells as one coalesced 256-byte row.
#include "kernels.h"

namespace bte {

template <typename C> struct CT;
template <> struct CT<float2> { using R = float; static __device__ float2 mk(float a, float b) { return make_float2(a, b); } };
template <> struct CT<double2> { using R = double; static __device__ double2 mk(double a, double b) { return make_double2(a, b); } };

__device__ __forceinline__ int phase_index(int a, int b, int N) {
    int t = (a * b) % N;
    return t < 0 ? t + N : t;
}

// x * exp(sgn * i theta), root = (cos theta, sin theta)
template <typename C, int SGN>
__device__ __forceinline__ void cmac(typename CT<C>::R &re, typename CT<C>::R &im, C x, C w) {
    if (SGN < 0) {
        re += x.x * w.x + x.y * w.y;
        im += x.y * w.x - x.x * w.y;
    } else {
        re += x.x * w.x - x.y * w.y;
        im += x.y * w.x + x.x * w.y;
    }
}

// Pass along j3 (fastest) from the real FP64 cells: T[slot][j1][j2][k3].
template <typename C>
__global__ void dft_fwd_axis3(const double *__restrict__ f, const int64_t *__restrict__ slot_off,
                              DftSeg s, const C *__restrict__ root, C *__restrict__ T,
                              int *status) {
    using R = typename CT<C>::R;
    const int N = s.N, M = N * N * N, h = N / 2;
    const int sl = blockIdx.y;
    const int64_t off = slot_off[s.s0 + sl];
    C *out = T + s.eoff + (int64_t)sl * M;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M; e += gridDim.x * blockDim.x) {
        if (off < 0) {
            out[e] = CT<C>::mk(0, 0);
            continue;
        }
        const int k3 = e % N, row = e - k3;
        R re = 0, im = 0;
        bool bad = false;
        for (int j3 = 0; j3 < N; ++j3) {
            const double x = f[off + row + j3];
            if (k3 == 0 && !isfinite(x)) bad = true;
            C xv = CT<C>::mk((R)x, 0);
            cmac<C, -1>(re, im, xv, root[phase_index(k3 - h, j3 - h, N)]);
        }
        if (bad) atomicOr(status, ST_NONFINITE);
        out[e] = CT<C>::mk(re, im);
    }
}

// Pass along the middle axis: out[slot][j1][k2][k3] = sum_j2 in[slot][j1][j2][k3] w(k2, j2).
template <typename C, int SGN>
__global__ void dft_axis2(const C *__restrict__ in, DftSeg s, const C *__restrict__ root,
                          C *__restrict__ out) {
    using R = typename CT<C>::R;
    const int N = s.N, M = N * N * N, h = N / 2;
    const int sl = blockIdx.y;
    const C *a = in + s.eoff + (int64_t)sl * M;
    C *o = out + s.eoff + (int64_t)sl * M;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M; e += gridDim.x * blockDim.x) {
        const int k3 = e % N, k2 = (e / N) % N, j1 = e / (N * N);
        R re = 0, im = 0;
        for (int j2 = 0; j2 < N; ++j2)
            cmac<C, SGN>(re, im, a[(j1 * N + j2) * N + k3], root[phase_index(k2 - h, j2 - h, N)]);
        o[e] = CT<C>::mk(re, im);
    }
}

// Pass along k1 into the group layout, with the forward scale.
template <typename C>
__global__ void dft_fwd_axis1_group(const C *__restrict__ in, DftSeg s, const C *__restrict__ root,
                                    typename CT<C>::R scale, C *__restrict__ G) {
    using R = typename CT<C>::R;
    const int N = s.N, M = N * N * N, h = N / 2;
    const int sl = blockIdx.y;
    const C *a = in + s.eoff + (int64_t)sl * M;
    C *g = G + s.eoff + (int64_t)(sl / kLanes) * M * kLanes + (sl % kLanes);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M; e += gridDim.x * blockDim.x) {
        const int k1 = e / (N * N), rest = e % (N * N);
        R re = 0, im = 0;
        for (int j1 = 0; j1 < N; ++j1)
            cmac<C, -1>(re, im, a[j1 * N * N + rest], root[phase_index(k1 - h, j1 - h, N)]);
        g[(int64_t)e * kLanes] = CT<C>::mk(scale * re, scale * im);
    }
}

// Inverse pass along k1 out of the group layout: out[slot][j1][k2][k3].
// Threads run lane-fastest so the group rows are read coalesced.
template <typename C>
__global__ void dft_inv_axis1_group(const C *__restrict__ G, DftSeg s, const C *__restrict__ root,
                                    C *__restrict__ out) {
    using R = typename CT<C>::R;
    const int N = s.N, M = N * N * N, h = N / 2;
    const int grp = blockIdx.y;
    const C *g = G + s.eoff + (int64_t)grp * M * kLanes;
    C *o = out + s.eoff + (int64_t)grp * kLanes * M;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)M * kLanes;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int lane = (int)(t % kLanes);
        const int e = (int)(t / kLanes);
        const int j1 = e / (N * N), rest = e % (N * N);
        R re = 0, im = 0;
        for (int k1 = 0; k1 < N; ++k1)
            cmac<C, +1>(re, im, g[((int64_t)k1 * N * N + rest) * kLanes + lane],
                        root[phase_index(k1 - h, j1 - h, N)]);
        o[(int64_t)lane * M + e] = CT<C>::mk(re, im);
    }
}

// Last inverse pass along k3 into the caller's FP64 array (real part, scaled).
template <typename C>
__global__ void dft_inv_axis3_real(const C *__restrict__ in, const int64_t *__restrict__ slot_off,
                                   DftSeg s, const C *__restrict__ root,
                                   typename CT<C>::R scale, double *__restrict__ q) {
    using R = typename CT<C>::R;
    const int N = s.N, M = N * N * N, h = N / 2;
    const int sl = blockIdx.y;
    const int64_t off = slot_off[s.s0 + sl];
    if (off < 0) return;
    const C *a = in + s.eoff + (int64_t)sl * M;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M; e += gridDim.x * blockDim.x) {
        const int j3 = e % N, row = e - j3;
        R re = 0, im = 0;
        for (int k3 = 0; k3 < N; ++k3)
            cmac<C, +1>(re, im, a[row + k3], root[phase_index(k3 - h, j3 - h, N)]);
        q[off + e] = (double)(scale * re);
    }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
namespace {
inline dim3 grid_for(int M, int nslots, int threads) {
    int bx = (M + threads - 1) / threads;
    return dim3(bx, nslots);
}
}  // namespace

template <typename C>
void launch_dft_forward(const double *f, const int64_t *slot_off, const DftSeg &s, const C *root,
                        double scale, C *T1, C *T2, C *G, int *status, cudaStream_t st) {
    const int M = s.N * s.N * s.N, threads = 128;
    dim3 grid = grid_for(M, s.nslots, threads);
    dft_fwd_axis3<C><<<grid, threads, 0, st>>>(f, slot_off, s, root, T1, status);
    dft_axis2<C, -1><<<grid, threads, 0, st>>>(T1, s, root, T2);
    dft_fwd_axis1_group<C><<<grid, threads, 0, st>>>(T2, s, root, (typename CT<C>::R)scale, G);
}

template <typename C>
void launch_dft_inverse(const C *G, const int64_t *slot_off, const DftSeg &s, const C *root,
                        double scale, C *T1, C *T2, double *q, cudaStream_t st) {
    const int M = s.N * s.N * s.N, threads = 128;
    const int ngroups = s.nslots / kLanes;
    int bx = (int)(((int64_t)M * kLanes + threads - 1) / threads);
    dft_inv_axis1_group<C><<<dim3(bx, ngroups), threads, 0, st>>>(G, s, root, T1);
    dim3 grid = grid_for(M, s.nslots, threads);
    dft_axis2<C, +1><<<grid, threads, 0, st>>>(T1, s, root, T2);
    dft_inv_axis3_real<C><<<grid, threads, 0, st>>>(T2, slot_off, s, root, (typename CT<C>::R)scale, q);
}

template void launch_dft_forward<float2>(const double *, const int64_t *, const DftSeg &,
                                         const float2 *, double, float2 *, float2 *, float2 *, int *,
                                         cudaStream_t);
template void launch_dft_forward<double2>(const double *, const int64_t *, const DftSeg &,
                                          const double2 *, double, double2 *, double2 *, double2 *,
                                          int *, cudaStream_t);
template void launch_dft_inverse<float2>(const float2 *, const int64_t *, const DftSeg &,
                                         const float2 *, double, float2 *, float2 *, double *,
                                         cudaStream_t);
template void launch_dft_inverse<double2>(const double2 *, const int64_t *, const DftSeg &,
                                          const double2 *, double, double2 *, double2 *, double *,
                                          cudaStream_t);

}  // namespace bte
