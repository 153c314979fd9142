// Device routines of the conservation projection (Sec. 3.3), shared by the
// standalone projection kernel and the fused inverse transform.
#pragma once

#include "kernels.h"

namespace bte {

constexpr int kProjThreads = 256;
constexpr int kProjMaxN = 48;

struct ProjShared {
    double red[32][5];  // one row per warp (up to 1024 threads)
    double v[kProjMaxN], v2[kProjMaxN], g[kProjMaxN];
    double lam[5];
    double tot[5];
};

// Double-float ("Df") numbers: hi + lo as an unevaluated sum of two FP32
// values. The building blocks are error-free: TwoSum (Knuth) gives s + e = a + b
// exactly and fmaf(w, x, -p) the exact error of p = w x. The _rn intrinsics
// keep the compiler from contracting a product into a following add.
struct Df {
    float hi, lo;
};

__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// acc += x
__device__ __forceinline__ void df_add(Df &acc, float x) {
    float s, e;
    two_sum_f(acc.hi, x, s, e);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, e);
}

// acc += w x
__device__ __forceinline__ void df_add_prod(Df &acc, float w, float x) {
    const float p = __fmul_rn(w, x);
    const float pe = fmaf(w, x, -p);
    df_add(acc, p);
    acc.lo = __fadd_rn(acc.lo, pe);
}

__device__ __forceinline__ Df df_add(Df a, Df b) {
    float s, e;
    two_sum_f(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    Df r;
    two_sum_f(s, e, r.hi, r.lo);
    return r;
}

// w a for a small integer w (w hi is split exactly, w lo rounds at 2^-48 of the value)
__device__ __forceinline__ Df df_mul_int(Df a, float w) {
    const float p = __fmul_rn(w, a.hi);
    const float pe = fmaf(w, a.hi, -p);
    Df r;
    two_sum_f(p, fmaf(w, a.lo, pe), r.hi, r.lo);
    return r;
}

// sum over the 32 lanes (every lane receives it)
__device__ __forceinline__ Df df_warp_sum(Df v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const Df w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        v = df_add(v, w);
    }
    return v;
}

// Block-wide sum of 5 values in a fixed order; result valid in all threads.
// Only the first `active` threads hold data: the other warps skip the
// shuffles, and five threads add the per-warp partials (FP64 is slow here, so
// no thread repeats the whole sum).
__device__ __forceinline__ void block_sum5(double v[5], ProjShared &sh, int active) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (active + 31) >> 5;
    if (warp < nw) {
#pragma unroll
        for (int i = 0; i < 5; ++i)
            for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
        if (lane == 0)
            for (int i = 0; i < 5; ++i) sh.red[warp][i] = v[i];
    }
    __syncthreads();
    if ((int)threadIdx.x < 5) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += sh.red[w][threadIdx.x];
        sh.tot[threadIdx.x] = s;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 5; ++i) v[i] = sh.tot[i];
}

// Velocity coordinates of the grid in shared memory (first N threads).
__device__ __forceinline__ void fill_velocities(const ProjArgs &pa, ProjShared &sh) {
    const int N = pa.N, h = N / 2;
    if ((int)threadIdx.x < N) {
        const double v = pa.dv * (double)((int)threadIdx.x - h);
        sh.v[threadIdx.x] = v;
        sh.v2[threadIdx.x] = v * v;
    }
    __syncthreads();
}

// mu_i = sum_j c_i(j) q_j (without the dv^3 factor). q may be global or shared.
__device__ __forceinline__ void cell_moments(const double *q, const ProjArgs &pa, double mu[5],
                                             ProjShared &sh) {
    fill_velocities(pa, sh);
    const int N = pa.N, NN = N * N;
    for (int i = 0; i < 5; ++i) mu[i] = 0.0;
    for (int p = threadIdx.x; p < NN; p += blockDim.x) {
        double r = 0.0, u = 0.0, w = 0.0;
        for (int j1 = 0; j1 < N; ++j1) {
            const double x = q[j1 * NN + p];
            r += x;
            u = fma(sh.v[j1], x, u);
            w = fma(sh.v2[j1], x, w);
        }
        const int j2 = p / N, j3 = p % N;
        mu[0] += r;
        mu[1] += u;
        mu[2] = fma(sh.v[j2], r, mu[2]);
        mu[3] = fma(sh.v[j3], r, mu[3]);
        mu[4] += w + (sh.v2[j2] + sh.v2[j3]) * r;
    }
    block_sum5(mu, sh, NN < (int)blockDim.x ? NN : (int)blockDim.x);
}

// Projection of one cell: reads qin (global or shared), writes qout (global),
// optionally fused with the Heun update of the time step:
// mode 0: qout = P q;  1: qout = P q, y = x + a qout;  2: qout = P q, y += a (qp + qout).
__device__ __forceinline__ void project_cell(const double *qin, double *qout, const ProjArgs &pa, int mode,
                                             const double *x, double *y, const double *qp, double a,
                                             ProjShared &sh) {
    double mu[5];
    cell_moments(qin, pa, mu, sh);
    const int N = pa.N, NN = N * N;
    if (threadIdx.x == 0) {
        for (int i = 0; i < 5; ++i) {
            double s = 0.0;
            for (int k = 0; k < 5; ++k) s = fma(pa.ainv[i * 5 + k], mu[k], s);
            sh.lam[i] = s;
        }
    }
    __syncthreads();
    const double l0 = sh.lam[0], l1 = sh.lam[1], l2 = sh.lam[2], l3 = sh.lam[3], l4 = sh.lam[4];
    if ((int)threadIdx.x < N) sh.g[threadIdx.x] = fma(l1, sh.v[threadIdx.x], l4 * sh.v2[threadIdx.x]);
    __syncthreads();
    for (int p = threadIdx.x; p < NN; p += blockDim.x) {
        const int j2 = p / N, j3 = p % N;
        const double base = l0 + fma(l2, sh.v[j2], fma(l3, sh.v[j3], l4 * (sh.v2[j2] + sh.v2[j3])));
        for (int j1 = 0; j1 < N; ++j1) {
            const int e = j1 * NN + p;
            const double v = qin[e] - (base + sh.g[j1]);
            qout[e] = v;
            if (mode == 1) y[e] = fma(a, v, x[e]);
            else if (mode == 2) y[e] = fma(a, qp[e] + v, y[e]);
        }
    }
}

}  // namespace bte
