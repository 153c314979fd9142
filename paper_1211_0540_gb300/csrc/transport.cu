// Transport sub-step of Sec. 3.4 on a 1-D slab of nx cells (uniform, or of
// unequal widths: transport_grid_stage_kernel below):
//   df/dt + v1 df/dx = 0, finite volumes with the second-order upwind flux of
//   Eq. upwind: F_{j+1/2} = v1 (f_j + dx/2 s_j) if v1 >= 0, else
//   v1 (f_{j+1} - dx/2 s_{j+1}), s_j = minmod((f_j - f_{j-1})/dx, (f_{j+1} - f_j)/dx),
// advanced by Heun's method (the paper's second-order Runge-Kutta):
//   f1 = f + tau R(f);  f <- (f + f1 + tau R(f1)) / 2,  R = -(F_{j+1/2} - F_{j-1/2}) / dx.
// Since minmod is positively homogeneous, dx/2 s_j = minmod(f_j - f_{j-1}, f_{j+1} - f_j) / 2:
// the face values need no division. FP64 arithmetic is expensive on this GPU
// (about 1/75 of the FP32 rate), so minmod works on the IEEE bit patterns
// (integer compares), the wall Maxwellians, (tau/dx) v1 and |v1| are tabulated
// on the host, and a sliding stencil window leaves four FP64 operations per
// value in the second Heun stage and five in the first.
// Walls (two ghost cells each side, formed on the fly):
// - diffuse (Sec. 2.1, Eq. BC): components entering the slab take
//   sigma_w M_w(v), M_w = (2 pi T_w)^{-3/2} exp(-|v|^2 / (2 T_w)); sigma_w is the
//   discrete outgoing flux sum |v.n| f over the discrete flux sum |v.n| M_w of
//   the incoming half, so the wall face carries no net mass; components
//   leaving copy the adjacent cell (zero gradient).
// - specular: v1 -> -v1 mirror, index i -> N - i; i = 0 (v1 = -L) has no
//   partner on the grid and its ghost value is 0.
// - no flux for the incoming characteristics (open boundary, Sec. 3.4):
//   incoming components 0, outgoing ones copy the adjacent cell.
// f is [cell][M] FP64, M = N^3, velocity index fastest (coalesced rows).
#include "kernels.h"

namespace bte {

namespace {
constexpr int kTThreads = 128;  // consecutive velocities of one cell chunk
constexpr int kTChunk = 4;      // cells per thread: 1024 CTAs at 128 cells x N = 16 (6.7 per SM)

// minmod(a, b) = 0 if a b <= 0, else the argument of smaller magnitude.
__device__ __forceinline__ double minmod(double a, double b) {
    const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
    const long long ma = ia & 0x7fffffffffffffffll, mb = ib & 0x7fffffffffffffffll;
    if (((ia ^ ib) < 0) || ma == 0 || mb == 0) return 0.0;
    return ma < mb ? a : b;
}

// sigma_w for the wall of `side` (0 left, 1 right), reduced by the whole CTA.
// Outgoing components (v.n < 0 for the inward normal n) are i < N/2 at the
// left wall and i > N/2 at the right wall; |v.n| = |v1_i| is tabulated.
// The outgoing components form one contiguous range of j (i is the slowest
// index); four independent loads per step keep the reduction off the memory
// latency (the wall CTAs would otherwise set the kernel's duration).
__device__ double wall_sigma(const double *__restrict__ f, const TransportArgs &a, int side) {
    __shared__ double red[kTThreads / 32];
    const int M = a.N * a.N * a.N, NN = a.N * a.N, h = a.N / 2;
    const double *fc = f + (int64_t)(side == 0 ? 0 : a.nx - 1) * M;
    const int j0 = side == 0 ? 0 : (h + 1) * NN, j1 = side == 0 ? h * NN : M;
    const int T = blockDim.x;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    int j = j0 + threadIdx.x;
    for (; j + 3 * T < j1; j += 4 * T) {
        double x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = fc[j + u * T];
#pragma unroll
        for (int u = 0; u < 4; ++u) s[u] = fma(a.wv[(j + u * T) / NN], x[u], s[u]);
    }
    for (; j < j1; j += T) s[0] = fma(a.wv[j / NN], fc[j], s[0]);
    double out = (s[0] + s[1]) + (s[2] + s[3]);
    for (int o = 16; o > 0; o >>= 1) out += __shfl_xor_sync(0xffffffffu, out, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = out;
    __syncthreads();
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    __syncthreads();
    return tot * (side == 0 ? a.rden_left : a.rden_right);
}

// Value of the extended array at cell x in [-2, nx + 1], velocity j.
__device__ __forceinline__ double ext(const double *__restrict__ f, int x, int j, int i, const TransportArgs &a,
                                      double sig_l, double sig_r) {
    const int M = a.N * a.N * a.N, NN = a.N * a.N, h = a.N / 2;
    if (x >= 0 && x < a.nx) return f[(int64_t)x * M + j];
    const bool left = x < 0;
    const int bc = left ? a.bc_left : a.bc_right;
    if (bc == BTE_BC_SPECULAR) {
        if (i == 0) return 0.0;
        const int jm = (a.N - i) * NN + (j - i * NN);
        const int src = left ? (-1 - x) : (2 * a.nx - 1 - x);  // -1->0, -2->1, nx->nx-1, nx+1->nx-2
        return f[(int64_t)src * M + jm];
    }
    const bool incoming = left ? (i > h) : (i < h);  // v . n > 0
    if (incoming) {
        if (bc == BTE_BC_NOFLUX) return 0.0;  // nothing enters through an open boundary
        return left ? sig_l * a.mw_left[j] : sig_r * a.mw_right[j];
    }
    return f[(int64_t)(left ? 0 : a.nx - 1) * M + j];
}

// Heun stages of one transport half step, written so that the second stage
// needs one FMA per value:
//   stage 1: f1 = f + tau R(f),  h = f + (tau / 2) R(f)       (src = f)
//   stage 2: f  = h + (tau / 2) R(f1)  (= (f + f1 + tau R(f1)) / 2)   (src = f1)
// With the upwind side fixed by the sign of v1 only four stencil points are
// read, e_0..e_3 = cells c-2..c+1 (v1 >= 0) or c-1..c+2 (v1 < 0), and with
// D_q = e_q - e_{q-1} the two face values of cell c differ by
//   g = f_{c+1/2} - f_{c-1/2} = D_2 +- (minmod(D_2, D_3) - minmod(D_1, D_2)) / 2,
// and tau R = -(tau / dx) v1 g. A thread takes kTChunk consecutive cells of
// one velocity: it loads their kTChunk + 3 stencil points at once, forms each
// difference D and each minmod once, then per value two operations for g and
// one FMA per output (two in stage 1).
template <int STAGE>
__global__ void __launch_bounds__(kTThreads) transport_stage_kernel(const double *__restrict__ src,
                                                                     double *__restrict__ out,
                                                                     double *__restrict__ half,
                                                                     const __grid_constant__ TransportArgs a) {
    const int M = a.N * a.N * a.N, NN = a.N * a.N, h = a.N / 2;
    const int c0 = blockIdx.y * kTChunk, c1 = min(c0 + kTChunk, a.nx);
    // walls: sigma_w only where a diffuse ghost is read for an incoming
    // velocity (i > N/2 at the left wall, i < N/2 at the right), i.e. the
    // chunks next to a wall and CTAs whose velocity range has such an i
    const int ilo = (int)(blockIdx.x * blockDim.x) / NN;
    const int ihi = min((int)((blockIdx.x + 1) * blockDim.x) - 1, M - 1) / NN;
    double sig_l = 0.0, sig_r = 0.0;
    if (c0 < 2 && a.bc_left == BTE_BC_DIFFUSE && ihi > h) sig_l = wall_sigma(src, a, 0);
    if (c1 > a.nx - 2 && a.bc_right == BTE_BC_DIFFUSE && ilo < h) sig_r = wall_sigma(src, a, 1);
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const int i = j / NN;
    const bool pos = i >= h;
    const double sgn = pos ? 0.5 : -0.5, kv = a.kv[i], kvh = a.kvh[i];
    const int x0 = pos ? c0 - 2 : c0 - 1;  // first stencil point of cell c0
    const int ne = c1 - c0 + 3;            // stencil points of the chunk
    // all loads first (independent, in flight together), then the arithmetic
    double e[kTChunk + 3];
#pragma unroll
    for (int d = 0; d < kTChunk + 3; ++d) e[d] = d < ne ? ext(src, x0 + d, j, i, a, sig_l, sig_r) : 0.0;
    double D[kTChunk + 2], m[kTChunk + 1];
#pragma unroll
    for (int d = 0; d < kTChunk + 2; ++d) D[d] = e[d + 1] - e[d];
#pragma unroll
    for (int d = 0; d < kTChunk + 1; ++d) m[d] = minmod(D[d], D[d + 1]);
#pragma unroll
    for (int q = 0; q < kTChunk; ++q) {
        if (c0 + q >= c1) break;
        // cell c = c0 + q: D_1, D_2, D_3 = D[q], D[q + 1], D[q + 2]
        const double g = fma(sgn, m[q + 1] - m[q], D[q + 1]);
        const double own = pos ? e[q + 2] : e[q + 1];  // src at cell c
        const int64_t idx = (int64_t)(c0 + q) * M + j;
        if (STAGE == 1) {
            out[idx] = fma(-kv, g, own);
            half[idx] = fma(-kvh, g, own);
        } else {
            out[idx] = fma(-kvh, g, half[idx]);
        }
    }
}
// Cells of unequal width dx_c (Sec. 3.4). The reconstruction at a face uses
// the upwind cell's width and the minmod slope of divided differences over
// the distances between cell centres, h_{c+1/2} = (dx_c + dx_{c+1}) / 2:
//   dx_c/2 s_c = minmod(alpha_c (f_c - f_{c-1}), gamma_c (f_{c+1} - f_c)),
//   alpha_c = dx_c / (2 h_{c-1/2}),  gamma_c = dx_c / (2 h_{c+1/2})
// (both 1/2 on a uniform grid; minmod commutes with positive factors). With
// mm the coefficient-weighted minmod of each stencil cell, the two face values
// of cell c differ by g = D_{c} +- (mm_upwind - mm_other) as in the uniform
// kernel, and tau R = -(tau / dx_c) v1 g. The ghost cells' widths mirror the
// adjacent interior cells (alpha, gamma of cells -1 and nx use them).
template <int STAGE>
__global__ void __launch_bounds__(kTThreads) transport_grid_stage_kernel(const double *__restrict__ src,
                                                                          double *__restrict__ out,
                                                                          double *__restrict__ half,
                                                                          const __grid_constant__ TransportArgs a,
                                                                          double tau) {
    const int M = a.N * a.N * a.N, NN = a.N * a.N, h = a.N / 2;
    const int c0 = blockIdx.y * kTChunk, c1 = min(c0 + kTChunk, a.nx);
    const int ilo = (int)(blockIdx.x * blockDim.x) / NN;
    const int ihi = min((int)((blockIdx.x + 1) * blockDim.x) - 1, M - 1) / NN;
    double sig_l = 0.0, sig_r = 0.0;
    if (c0 < 2 && a.bc_left == BTE_BC_DIFFUSE && ihi > h) sig_l = wall_sigma(src, a, 0);
    if (c1 > a.nx - 2 && a.bc_right == BTE_BC_DIFFUSE && ilo < h) sig_r = wall_sigma(src, a, 1);
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const int i = j / NN;
    const bool pos = i >= h;
    const double v1 = a.dv * (double)(i - h);
    const int x0 = pos ? c0 - 2 : c0 - 1;  // first stencil point of cell c0
    const int ne = c1 - c0 + 3;
    double e[kTChunk + 3];
#pragma unroll
    for (int d = 0; d < kTChunk + 3; ++d) e[d] = d < ne ? ext(src, x0 + d, j, i, a, sig_l, sig_r) : 0.0;
    double D[kTChunk + 2], mm[kTChunk + 1];
#pragma unroll
    for (int d = 0; d < kTChunk + 2; ++d) D[d] = e[d + 1] - e[d];
#pragma unroll
    for (int d = 0; d < kTChunk + 1; ++d) {
        const int cell = x0 + d + 1;  // in [-1, nx]
        const bool live = d < ne - 2;
        mm[d] = live ? minmod(a.g_alpha[cell + 1] * D[d], a.g_gamma[cell + 1] * D[d + 1]) : 0.0;
    }
#pragma unroll
    for (int q = 0; q < kTChunk; ++q) {
        if (c0 + q >= c1) break;
        const int c = c0 + q;
        const double g = pos ? D[q + 1] + (mm[q + 1] - mm[q]) : D[q + 1] - (mm[q + 1] - mm[q]);
        const double kv = tau * v1 * a.g_rdx[c];
        const double own = pos ? e[q + 2] : e[q + 1];
        const int64_t idx = (int64_t)c * M + j;
        if (STAGE == 1) {
            out[idx] = fma(-kv, g, own);
            half[idx] = fma(-0.5 * kv, g, own);
        } else {
            out[idx] = fma(-0.5 * kv, g, half[idx]);
        }
    }
}
}  // namespace

void launch_transport_half(double *f, double *f1, double *fh, const TransportArgs &ta, double tau,
                           cudaStream_t st) {
    const int M = ta.N * ta.N * ta.N, h = ta.N / 2;
    TransportArgs a = ta;
    const double k = tau / ta.dx;
    for (int i = 0; i < kTransportMaxN; ++i) {
        const double v1 = i < ta.N ? ta.dv * (i - h) : 0.0;
        a.kv[i] = k * v1;
        a.kvh[i] = 0.5 * a.kv[i];
        a.wv[i] = v1 < 0.0 ? -v1 : v1;
    }
    a.rden_left = ta.den_left > 0.0 ? 1.0 / ta.den_left : 0.0;
    a.rden_right = ta.den_right > 0.0 ? 1.0 / ta.den_right : 0.0;
    dim3 grid((M + kTThreads - 1) / kTThreads, (ta.nx + kTChunk - 1) / kTChunk);
    if (ta.g_rdx) {
        transport_grid_stage_kernel<1><<<grid, kTThreads, 0, st>>>(f, f1, fh, a, tau);
        transport_grid_stage_kernel<2><<<grid, kTThreads, 0, st>>>(f1, f, fh, a, tau);
        return;
    }
    transport_stage_kernel<1><<<grid, kTThreads, 0, st>>>(f, f1, fh, a);
    transport_stage_kernel<2><<<grid, kTThreads, 0, st>>>(f1, f, fh, a);
}

}  // namespace bte
