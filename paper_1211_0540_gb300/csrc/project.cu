// Conservation projection of Sec. 3.3 in FP64:
//   Q <- Q - C^T (C C^T)^{-1} C Q,  C_j = dv^3 (1, v1, v2, v3, |v|^2)_j.
// (The paper prints "Q = Qt + C (C C^T)^{-1} C Qt"; the Lagrange solution of
// its minimisation problem is the form above, which is what is computed.) The
// dv^3 factors cancel, so the kernel uses c_j = (1, v1, v2, v3, |v|^2) and the
// host-inverted 5x5 matrix A^{-1}, A = sum_j c_j c_j^T.
//
// FP64 is slow on this GPU, so the moments use the tensor structure of c_j:
// with r = sum over j1 of Q, u = sum of v1 Q, w = sum of v1^2 Q taken along the
// j1 line through each (j2, j3),
//   mu0 = sum r, mu1 = sum u, mu2 = sum v2 r, mu3 = sum v3 r,
//   mu4 = sum (w + (v2^2 + v3^2) r),
// three FP64 operations per value; the correction c_j . lambda splits into a
// per-(j2, j3) base plus a per-j1 term, two operations per value. One CTA per
// cell; sums are reduced in a fixed order (deterministic). The same routine
// runs inside the fused inverse transform (dft_fused.cu).
#include "project.cuh"

namespace bte {

__global__ void __launch_bounds__(kProjThreads)
project_kernel(double *__restrict__ Q, const int64_t *__restrict__ slot_off, int s0, ProjArgs pa,
               int mode, const double *__restrict__ X, double *__restrict__ Y,
               const double *__restrict__ Qp, double a) {
    const int64_t off = slot_off[s0 + blockIdx.x];
    if (off < 0) return;
    __shared__ ProjShared sh;
    project_cell(Q + off, Q + off, pa, mode, X ? X + off : nullptr, Y ? Y + off : nullptr,
                 Qp ? Qp + off : nullptr, a, sh);
}

__global__ void __launch_bounds__(kProjThreads)
moments_kernel(const double *__restrict__ f, const int64_t *__restrict__ slot_off, int s0, ProjArgs pa,
               const int64_t *__restrict__ slot_out, double *__restrict__ out) {
    const int64_t off = slot_off[s0 + blockIdx.x];
    if (off < 0) return;
    __shared__ ProjShared sh;
    double mu[5];
    cell_moments(f + off, pa, mu, sh);
    if (threadIdx.x == 0) {
        const double w = pa.dv * pa.dv * pa.dv;
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
    ProjArgs pa{};
    pa.N = N;
    pa.dv = dv;
    moments_kernel<<<nslots, kProjThreads, 0, st>>>(f, slot_off, s0, pa, slot_out, out);
}

}  // namespace bte
