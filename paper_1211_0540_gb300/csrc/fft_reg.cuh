// Mixed-radix FFT on a register array, all indices compile-time.
//
//   y_k = sum_j x_j w^(S j k),  w = exp(2 pi i / n),  S = +1 or -1,
//
// natural order in and out, for n = 2^a 3^b. Decimation in time (Cooley-Tukey):
// with n = R n2 (radix R = 4 if it divides n, else 3, else 2), j = n2 j1 + j2
// and k = k1 + R k2,
//   y_{k1 + R k2} = sum_{j2} w_{n2}^{S j2 k2} [ w_n^{S j2 k1} sum_{j1} x_{n2 j1 + j2} w_R^{S j1 k1} ],
// i.e. n2 transforms of size R, the twiddles w_n^{S j2 k1}, then R transforms
// of size n2. A transform of size 16 takes 160 real operations (128 additions
// in the eight radix-4 butterflies, 8 general twiddles of 4 each) instead of
// the 1024 FMAs of the dense matrix.
//
// Twiddles come from one table of the top-level size NT,
// root[t] = exp(2 pi i t / NT): w_n^t = root[(t NT / n) mod NT]. Indices 0,
// NT/4, NT/2 and 3NT/4 are +-1 and +-i and cost no multiplication; with the
// loops unrolled every index is a compile-time constant, so on the device the
// table (in constant memory) supplies FMA operands directly. Host and device:
// the same code is checked against the dense sum on the CPU.
#pragma once

#include <cuda_runtime.h>

namespace bte {
namespace fftr {

__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cneg(float2 a) { return make_float2(-a.x, -a.y); }
// i s a for s = +1 or -1
template <int S>
__host__ __device__ __forceinline__ float2 cmul_i(float2 a) {
    return S > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// v w_NT^(S t), t >= 0 (compile-time after unrolling)
template <int NT, int S>
__host__ __device__ __forceinline__ float2 twiddle(float2 v, int t, const float2 (&rt)[NT]) {
    const int u = ((S * t) % NT + NT) % NT;
    if (u == 0) return v;
    if (2 * u == NT) return cneg(v);
    if (4 * u == NT) return cmul_i<1>(v);
    if (4 * u == 3 * NT) return cmul_i<-1>(v);
    const float2 w = rt[u];
    return make_float2(fmaf(v.x, w.x, -(v.y * w.y)), fmaf(v.x, w.y, v.y * w.x));
}

// In place: x <- DFT_S(x) of size N inside a top-level transform of size NT.
template <int N, int S, int NT>
__host__ __device__ __forceinline__ void fft(float2 (&x)[N], const float2 (&rt)[NT]) {
    static_assert(NT % N == 0, "sub-transform size");
    if constexpr (N == 1) {
    } else if constexpr (N == 2) {
        const float2 a = x[0], b = x[1];
        x[0] = cadd(a, b);
        x[1] = csub(a, b);
    } else if constexpr (N == 3) {
        // w_3^S = -1/2 + i S sin(2 pi / 3); sin(2 pi / 3) = Im root[NT / 3]
        const float s3 = rt[NT / 3].y;
        const float2 a = x[0], t = cadd(x[1], x[2]), u = csub(x[1], x[2]);
        const float2 m = make_float2(fmaf(-0.5f, t.x, a.x), fmaf(-0.5f, t.y, a.y));
        const float2 r = cmul_i<S>(make_float2(s3 * u.x, s3 * u.y));
        x[0] = cadd(a, t);
        x[1] = cadd(m, r);
        x[2] = csub(m, r);
    } else if constexpr (N == 4) {
        const float2 a = cadd(x[0], x[2]), b = csub(x[0], x[2]);
        const float2 c = cadd(x[1], x[3]), d = cmul_i<S>(csub(x[1], x[3]));
        x[0] = cadd(a, c);
        x[1] = cadd(b, d);
        x[2] = csub(a, c);
        x[3] = csub(b, d);
    } else {
        constexpr int R = N % 4 == 0 ? 4 : (N % 3 == 0 ? 3 : 2);
        constexpr int N2 = N / R;
        float2 A[R][N2];
#pragma unroll
        for (int j2 = 0; j2 < N2; ++j2) {
            float2 v[R];
#pragma unroll
            for (int j1 = 0; j1 < R; ++j1) v[j1] = x[N2 * j1 + j2];
            fft<R, S, NT>(v, rt);
#pragma unroll
            for (int k1 = 0; k1 < R; ++k1) A[k1][j2] = twiddle<NT, S>(v[k1], j2 * k1 * (NT / N), rt);
        }
#pragma unroll
        for (int k1 = 0; k1 < R; ++k1) {
            float2 u[N2];
#pragma unroll
            for (int j2 = 0; j2 < N2; ++j2) u[j2] = A[k1][j2];
            fft<N2, S, NT>(u, rt);
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) x[k1 + R * k2] = u[k2];
        }
    }
}

// Centred transform of one pencil (N/2 even):
//   y_k = sum_j x_j w^(S (k - N/2)(j - N/2)) = (-1)^k sum_j (-1)^j x_j w^(S j k),
// since w^(-N/2 k) = (-1)^k and w^((N/2)^2) = (-1)^(N/2) = 1.
template <int N, int S>
__host__ __device__ __forceinline__ void centred(float2 (&y)[N], const float2 (&rt)[N]) {
    static_assert(N % 4 == 0, "N/2 must be even");
#pragma unroll
    for (int j = 1; j < N; j += 2) y[j] = cneg(y[j]);
    fft<N, S, N>(y, rt);
#pragma unroll
    for (int k = 1; k < N; k += 2) y[k] = cneg(y[k]);
}

}  // namespace fftr
}  // namespace bte
