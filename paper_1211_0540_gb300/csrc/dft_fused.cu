// Fused per-cell transforms for N <= 16 (the whole cell fits in shared memory).
//   forward:  fhat_k = (2 pi)^{-3/2} dv^3 sum_j f_j exp(-i zeta_k . v_j)
//   inverse:  Qt_j = Re (2 pi)^{-3/2} dz^3 sum_k Qhat_k exp(+i zeta_k . v_j)
// (Sec. 3.2, grid of Eq. meshpoints; zeta_k . v_j = 2 pi k'.j' / N.)
// One CTA per cell does the three one-dimensional passes in shared memory with
// the N x N phase matrix held there too (no per-term index arithmetic), so a
// direction costs one launch and one read + one write of the cell. The
// forward kernel writes fhat straight into the group layout of the
// convolution ([group][k][lane]); the inverse kernel reads Qhat from it, keeps
// Qt in shared memory in FP64, and applies the conservation projection of
// Sec. 3.3 (and optionally the Heun update) before the single write of Q.
#include "project.cuh"

namespace bte {

namespace {

template <int N>
struct FusedShape {
    static constexpr int M = N * N * N;
    static constexpr int NT = N == 16 ? 1024 : (N == 12 ? 576 : 512);  // multiple of N and of 32
    static constexpr int WP = N + 1;          // padded phase-matrix row
    static constexpr size_t smem = 2 * sizeof(float2) * M + sizeof(float2) * N * WP;
};

// W[k][j] = exp(sgn * 2 pi i (k - h)(j - h) / N)
template <int N>
__device__ __forceinline__ void fill_phase(float2 *W, const float2 *__restrict__ root, float sgn) {
    const int h = N / 2;
    for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
        const int k = idx / N, j = idx % N;
        int t = ((k - h) * (j - h)) % N;
        if (t < 0) t += N;
        const float2 w = root[t];
        W[k * (N + 1) + j] = make_float2(w.x, sgn * w.y);
    }
}

}  // namespace

template <int N>
__global__ void __launch_bounds__(FusedShape<N>::NT)
dft_fwd_fused_kernel(const double *__restrict__ f, const int64_t *__restrict__ slot_off, DftSeg s,
                     const float2 *__restrict__ root, float scale, float2 *__restrict__ G, int *status) {
    using S = FusedShape<N>;
    constexpr int M = S::M, NN = N * N;
    extern __shared__ __align__(16) char smem_raw[];
    float2 *A = reinterpret_cast<float2 *>(smem_raw);
    float2 *B = A + M;
    float2 *W = B + M;
    const int sl = blockIdx.x;
    const int64_t off = slot_off[s.s0 + sl];
    float2 *g = G + s.eoff + (int64_t)(sl / kLanes) * M * kLanes + (sl % kLanes);
    if (off < 0) {  // padding lane of a group: zero fhat
        for (int e = threadIdx.x; e < M; e += blockDim.x) g[(int64_t)e * kLanes] = make_float2(0.f, 0.f);
        return;
    }
    fill_phase<N>(W, root, -1.f);
    float *R = reinterpret_cast<float *>(B);
    bool bad = false;
    for (int e = threadIdx.x; e < M; e += blockDim.x) {
        const double x = f[off + e];
        bad |= !isfinite(x);
        R[e] = (float)x;
    }
    if (bad) atomicOr(status, ST_NONFINITE);
    __syncthreads();
    // pass along j3 (real input): A[row][k3] = sum_j3 R[row][j3] W[k3][j3]
    {
        const int k3 = threadIdx.x % N, rg = threadIdx.x / N;
        float2 w[N];
#pragma unroll
        for (int j = 0; j < N; ++j) w[j] = W[k3 * S::WP + j];
        for (int row = rg; row < NN; row += S::NT / N) {
            float re = 0.f, im = 0.f;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const float x = R[row * N + j];
                re = fmaf(x, w[j].x, re);
                im = fmaf(x, w[j].y, im);
            }
            A[row * N + k3] = make_float2(re, im);
        }
    }
    __syncthreads();
    // pass along j2: B[j1][k2][k3] = sum_j2 A[j1][j2][k3] W[k2][j2]
    for (int e = threadIdx.x; e < M; e += blockDim.x) {
        const int k3 = e % N, k2 = (e / N) % N, j1 = e / NN;
        const float2 *a = A + j1 * NN + k3;
        const float2 *w = W + k2 * S::WP;
        float re = 0.f, im = 0.f;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const float2 x = a[j * N], ww = w[j];
            re = fmaf(x.x, ww.x, fmaf(-x.y, ww.y, re));
            im = fmaf(x.y, ww.x, fmaf(x.x, ww.y, im));
        }
        B[e] = make_float2(re, im);
    }
    __syncthreads();
    // pass along j1 into the group layout, scaled
    for (int e = threadIdx.x; e < M; e += blockDim.x) {
        const int k1 = e / NN, rest = e % NN;
        const float2 *b = B + rest;
        const float2 *w = W + k1 * S::WP;
        float re = 0.f, im = 0.f;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const float2 x = b[j * NN], ww = w[j];
            re = fmaf(x.x, ww.x, fmaf(-x.y, ww.y, re));
            im = fmaf(x.y, ww.x, fmaf(x.x, ww.y, im));
        }
        g[(int64_t)e * kLanes] = make_float2(scale * re, scale * im);
    }
}

// mode: 0 raw Qt; 1 P Qt; 2 P Qt and y = x + a Q; 3 P Qt and y += a (qp + Q)
template <int N>
__global__ void __launch_bounds__(FusedShape<N>::NT)
dft_inv_fused_kernel(const float2 *__restrict__ G, const int64_t *__restrict__ slot_off, DftSeg s,
                     const float2 *__restrict__ root, float scale, double *__restrict__ q, ProjArgs pa,
                     int mode, const double *__restrict__ x, double *__restrict__ y,
                     const double *__restrict__ qp, double a) {
    using S = FusedShape<N>;
    constexpr int M = S::M, NN = N * N;
    extern __shared__ __align__(16) char smem_raw[];
    float2 *A = reinterpret_cast<float2 *>(smem_raw);
    float2 *B = A + M;
    float2 *W = B + M;
    __shared__ ProjShared psh;
    const int sl = blockIdx.x;
    const int64_t off = slot_off[s.s0 + sl];
    if (off < 0) return;
    fill_phase<N>(W, root, 1.f);
    const float2 *g = G + s.eoff + (int64_t)(sl / kLanes) * M * kLanes + (sl % kLanes);
    for (int e = threadIdx.x; e < M; e += blockDim.x) A[e] = g[(int64_t)e * kLanes];
    __syncthreads();
    // along k1: B[j1][k2][k3] = sum_k1 A[k1][k2][k3] W[j1][k1]
    for (int e = threadIdx.x; e < M; e += blockDim.x) {
        const int j1 = e / NN, rest = e % NN;
        const float2 *b = A + rest;
        const float2 *w = W + j1 * S::WP;
        float re = 0.f, im = 0.f;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const float2 xx = b[k * NN], ww = w[k];
            re = fmaf(xx.x, ww.x, fmaf(-xx.y, ww.y, re));
            im = fmaf(xx.y, ww.x, fmaf(xx.x, ww.y, im));
        }
        B[e] = make_float2(re, im);
    }
    __syncthreads();
    // along k2: A[j1][j2][k3] = sum_k2 B[j1][k2][k3] W[j2][k2]
    for (int e = threadIdx.x; e < M; e += blockDim.x) {
        const int k3 = e % N, j2 = (e / N) % N, j1 = e / NN;
        const float2 *b = B + j1 * NN + k3;
        const float2 *w = W + j2 * S::WP;
        float re = 0.f, im = 0.f;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const float2 xx = b[k * N], ww = w[k];
            re = fmaf(xx.x, ww.x, fmaf(-xx.y, ww.y, re));
            im = fmaf(xx.y, ww.x, fmaf(xx.x, ww.y, im));
        }
        A[e] = make_float2(re, im);
    }
    __syncthreads();
    // along k3, real part, into FP64 (reusing B's storage: 8 bytes per value)
    double *D = reinterpret_cast<double *>(B);
    {
        const int j3 = threadIdx.x % N, rg = threadIdx.x / N;
        float2 w[N];
#pragma unroll
        for (int k = 0; k < N; ++k) w[k] = W[j3 * S::WP + k];
        for (int row = rg; row < NN; row += S::NT / N) {
            float re = 0.f;
#pragma unroll
            for (int k = 0; k < N; ++k) {
                const float2 xx = A[row * N + k];
                re = fmaf(xx.x, w[k].x, fmaf(-xx.y, w[k].y, re));
            }
            D[row * N + j3] = (double)(scale * re);
        }
    }
    __syncthreads();
    double *qo = q + off;
    if (mode == 0) {
        for (int e = threadIdx.x; e < M; e += blockDim.x) qo[e] = D[e];
        return;
    }
    project_cell(D, qo, pa, mode - 1, x ? x + off : nullptr, y ? y + off : nullptr,
                 qp ? qp + off : nullptr, a, psh);
}

namespace {
template <int N>
void fwd_launch(const double *f, const int64_t *slot_off, const DftSeg &s, const float2 *root, double scale,
                float2 *G, int *status, cudaStream_t st) {
    using S = FusedShape<N>;
    dft_fwd_fused_kernel<N><<<s.nslots, S::NT, S::smem, st>>>(f, slot_off, s, root, (float)scale, G, status);
}
template <int N>
void inv_launch(const float2 *G, const int64_t *slot_off, const DftSeg &s, const float2 *root, double scale,
                double *q, const ProjArgs &pa, int mode, const double *x, double *y, const double *qp, double a,
                cudaStream_t st) {
    using S = FusedShape<N>;
    dft_inv_fused_kernel<N><<<s.nslots, S::NT, S::smem, st>>>(G, slot_off, s, root, (float)scale, q, pa, mode, x,
                                                                y, qp, a);
}
}  // namespace

bool fused_dft_supported(int N) { return N == 8 || N == 12 || N == 16; }

void fused_dft_prepare(int N) {
    // sets the shared-memory attributes (must happen outside stream capture)
    switch (N) {
        case 8: {
            using S = FusedShape<8>;
            cudaFuncSetAttribute(dft_fwd_fused_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem);
            cudaFuncSetAttribute(dft_inv_fused_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem);
            break;
        }
        case 12: {
            using S = FusedShape<12>;
            cudaFuncSetAttribute(dft_fwd_fused_kernel<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem);
            cudaFuncSetAttribute(dft_inv_fused_kernel<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem);
            break;
        }
        case 16: {
            using S = FusedShape<16>;
            cudaFuncSetAttribute(dft_fwd_fused_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem);
            cudaFuncSetAttribute(dft_inv_fused_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem);
            break;
        }
        default: break;
    }
}

void launch_dft_forward_fused(const double *f, const int64_t *slot_off, const DftSeg &s, const float2 *root,
                              double scale, float2 *G, int *status, cudaStream_t st) {
    switch (s.N) {
        case 8: fwd_launch<8>(f, slot_off, s, root, scale, G, status, st); break;
        case 12: fwd_launch<12>(f, slot_off, s, root, scale, G, status, st); break;
        case 16: fwd_launch<16>(f, slot_off, s, root, scale, G, status, st); break;
        default: break;
    }
}

void launch_dft_inverse_fused(const float2 *G, const int64_t *slot_off, const DftSeg &s, const float2 *root,
                              double scale, double *q, const ProjArgs &pa, int mode, const double *x, double *y,
                              const double *qp, double a, cudaStream_t st) {
    switch (s.N) {
        case 8: inv_launch<8>(G, slot_off, s, root, scale, q, pa, mode, x, y, qp, a, st); break;
        case 12: inv_launch<12>(G, slot_off, s, root, scale, q, pa, mode, x, y, qp, a, st); break;
        case 16: inv_launch<16>(G, slot_off, s, root, scale, q, pa, mode, x, y, qp, a, st); break;
        default: break;
    }
}

}  // namespace bte
