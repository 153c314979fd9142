// Transport sub-step of Sec. 3.4 on a 1-D slab of nx uniform cells:
//   df/dt + v1 df/dx = 0, finite volumes with the second-order upwind flux of
//   Eq. upwind: F_{j+1/2} = v1 (f_j + dx/2 s_j) if v1 >= 0, else
//   v1 (f_{j+1} - dx/2 s_{j+1}), s_j = minmod((f_j - f_{j-1})/dx, (f_{j+1} - f_j)/dx),
// advanced by Heun's method (the paper's second-order Runge-Kutta):
//   f1 = f + tau R(f);  f <- (f + f1 + tau R(f1)) / 2.
// Walls (two ghost cells each side, filled on the fly):
// - diffuse (Sec. 2.1, Eq. BC): components entering the slab take
//   sigma_w M_w(v), M_w = (2 pi T_w)^{-3/2} exp(-|v|^2 / (2 T_w)); sigma_w equals
//   the discrete outgoing flux divided by the discrete flux of M_w, so the face
//   carries no net mass; components leaving copy the adjacent cell.
// - specular: v1 -> -v1 mirror, index i -> N - i; i = 0 (v1 = -L) has no
//   partner on the grid and its ghost value is 0.
// f is [cell][M] FP64, M = N^3 (the velocity index is the fast one, so each
// thread block reads coalesced rows of one cell and its neighbours).
#include "kernels.h"

namespace bte {

namespace {
constexpr int kTThreads = 256;
constexpr double kPi = 3.14159265358979323846;

__device__ __forceinline__ double minmod(double a, double b) {
    if (a * b <= 0.0) return 0.0;
    return a > 0.0 ? fmin(a, b) : fmax(a, b);
}

__device__ __forceinline__ double wall_maxwellian(double Tw, double v1, double v2, double v3) {
    return pow(2.0 * kPi * Tw, -1.5) * exp(-(v1 * v1 + v2 * v2 + v3 * v3) / (2.0 * Tw));
}

// Value of the extended array at cell x in [-2, nx + 1], velocity j.
__device__ __forceinline__ double ext(const double *__restrict__ f, int x, int j,
                                      const TransportArgs &a, const double *__restrict__ wall,
                                      double v1, double v2, double v3) {
    const int M = a.N * a.N * a.N;
    if (x >= 0 && x < a.nx) return f[(int64_t)x * M + j];
    const bool left = x < 0;
    const int bc = left ? a.bc_left : a.bc_right;
    if (bc == BTE_BC_SPECULAR) {
        const int i = j / (a.N * a.N);
        if (i == 0) return 0.0;
        const int jm = (a.N - i) * a.N * a.N + j % (a.N * a.N);
        const int src = left ? (-1 - x) : (2 * a.nx - 1 - x);  // -1->0, -2->1, nx->nx-1, nx+1->nx-2
        return f[(int64_t)src * M + jm];
    }
    const double vn = left ? v1 : -v1;  // component along the inward normal
    if (vn > 0.0) {
        const double Tw = left ? a.Tw_left : a.Tw_right;
        return wall[left ? 0 : 1] * wall_maxwellian(Tw, v1, v2, v3);
    }
    return f[(int64_t)(left ? 0 : a.nx - 1) * M + j];
}

// sigma_w of each diffuse wall: sum_out |v.n| f / sum_in |v.n| M_w.
__global__ void __launch_bounds__(kTThreads) wall_sigma_kernel(const double *__restrict__ f,
                                                                TransportArgs a, double *wall) {
    const int side = blockIdx.x;  // 0 left, 1 right
    const int bc = side == 0 ? a.bc_left : a.bc_right;
    const int M = a.N * a.N * a.N, h = a.N / 2;
    const double Tw = side == 0 ? a.Tw_left : a.Tw_right;
    const double *fc = f + (int64_t)(side == 0 ? 0 : a.nx - 1) * M;
    double out = 0.0, in = 0.0;
    if (bc == BTE_BC_DIFFUSE) {
        for (int j = threadIdx.x; j < M; j += blockDim.x) {
            const double v1 = a.dv * (j / (a.N * a.N) - h), v2 = a.dv * ((j / a.N) % a.N - h),
                         v3 = a.dv * (j % a.N - h);
            const double vn = side == 0 ? v1 : -v1;
            if (vn < 0.0) out += -vn * fc[j];
            else if (vn > 0.0) in += vn * wall_maxwellian(Tw, v1, v2, v3);
        }
    }
    __shared__ double so[kTThreads / 32], si[kTThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        out += __shfl_xor_sync(0xffffffffu, out, o);
        in += __shfl_xor_sync(0xffffffffu, in, o);
    }
    if ((threadIdx.x & 31) == 0) {
        so[threadIdx.x >> 5] = out;
        si[threadIdx.x >> 5] = in;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double O = 0.0, I = 0.0;
        for (int w = 0; w < kTThreads / 32; ++w) {
            O += so[w];
            I += si[w];
        }
        wall[side] = I > 0.0 ? O / I : 0.0;
    }
}

// stage 1: f1 = f + tau R(f)      (src = f)
// stage 2: f  = (f + f1 + tau R(f1)) / 2   (src = f1)
template <int STAGE>
__global__ void __launch_bounds__(kTThreads) transport_stage_kernel(double *__restrict__ f,
                                                                     double *__restrict__ f1,
                                                                     const double *__restrict__ wall,
                                                                     TransportArgs a, double tau) {
    const int M = a.N * a.N * a.N, h = a.N / 2;
    const int c = blockIdx.y;
    const double *src = STAGE == 1 ? f : f1;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
        const double v1 = a.dv * (j / (a.N * a.N) - h), v2 = a.dv * ((j / a.N) % a.N - h),
                     v3 = a.dv * (j % a.N - h);
        double e[5];
#pragma unroll
        for (int d = 0; d < 5; ++d) e[d] = ext(src, c - 2 + d, j, a, wall, v1, v2, v3);
        const double dx = a.dx;
        double F[2];
#pragma unroll
        for (int face = 0; face < 2; ++face) {
            // face between e[1 + face] and e[2 + face]
            const double fl = e[1 + face], fr = e[2 + face];
            if (v1 >= 0.0) {
                const double s = minmod((fl - e[face]) / dx, (fr - fl) / dx);
                F[face] = v1 * (fl + 0.5 * dx * s);
            } else {
                const double s = minmod((fr - fl) / dx, (e[3 + face] - fr) / dx);
                F[face] = v1 * (fr - 0.5 * dx * s);
            }
        }
        const double R = -(F[1] - F[0]) / dx;
        const int64_t idx = (int64_t)c * M + j;
        if (STAGE == 1) f1[idx] = f[idx] + tau * R;
        else f[idx] = 0.5 * (f[idx] + f1[idx] + tau * R);
    }
}
}  // namespace

void launch_transport_half(double *f, double *f1, double *wall, const TransportArgs &ta, double tau,
                           cudaStream_t st) {
    const int M = ta.N * ta.N * ta.N;
    dim3 grid((M + kTThreads - 1) / kTThreads, ta.nx);
    wall_sigma_kernel<<<2, kTThreads, 0, st>>>(f, ta, wall);
    transport_stage_kernel<1><<<grid, kTThreads, 0, st>>>(f, f1, wall, ta, tau);
    wall_sigma_kernel<<<2, kTThreads, 0, st>>>(f1, ta, wall);
    transport_stage_kernel<2><<<grid, kTThreads, 0, st>>>(f, f1, wall, ta, tau);
}

}  // namespace bte
