// Fused per-cell transforms (N = 8, 12, 16, 24, 32): a cell's slabs live in the
// shared memory of a thread-block cluster.
//   forward:  fhat_k = (2 pi)^{-3/2} dv^3 sum_j f_j exp(-i zeta_k . v_j)
//   inverse:  Qt_j = Re (2 pi)^{-3/2} dz^3 sum_k Qhat_k exp(+i zeta_k . v_j)
// (Sec. 3.2, grid of Eq. meshpoints; zeta_k . v_j = 2 pi k'.j' / N.)
// A cell is one CTA or a cluster of C CTAs, one thread per pencil: each of
// the three one-dimensional passes loads the N values of a pencil into
// registers and applies the phases exp(+-2 pi i (k - N/2)(j - N/2) / N) by a
// mixed-radix FFT (fft_reg.cuh: the centred phases are the plain DFT with
// the signs (-1)^j on the input and (-1)^k on the output). All indices are
// compile-time constants, so the roots of unity come from constant memory as
// FMA operands; shared memory is touched once per value and pass (rows
// padded to N + 1 against bank conflicts). The forward kernel writes fhat
// straight into the group layout of the convolution ([group][k][lane]); the
// inverse kernel reads Qhat from it and applies the conservation projection
// of Sec. 3.3 (and optionally the Heun update) before the single write of Q.
//
// FP64 runs at about 1/70 of the FP32 rate here, so the five moments of Qt
// are accumulated in double-float arithmetic (pairs of FP32 numbers combined
// by error-free TwoSum / TwoProduct steps, relative error ~1e-13 over the
// reduction tree) and only the final correction Q = Qt - C^T lambda and the
// time update run in FP64.
#include <cooperative_groups.h>

#include <cmath>
#include <map>
#include <mutex>

#include "fft_reg.cuh"
#include "fpconv.cuh"
#include "project.cuh"

namespace cg = cooperative_groups;

namespace bte {

namespace {

template <int N, int C_ = 4>
struct FusedShape {
    static constexpr int M = N * N * N, NN = N * N, H = N / 2;
    static constexpr int C = C_;         // CTAs per cell (one thread-block cluster)
    static constexpr int JR = N / C;     // slab rows (j1 or k2 values) per CTA
    static constexpr int NP = NN / C;    // pencils per CTA and pass
    static constexpr int NT = (NP + 31) / 32 * 32;
    static constexpr int NW = NT / 32;
    static constexpr int P = N + 1;      // padded pencil stride
    // forward: A (own pencils, padded) + B (own slab, read by the cluster)
    static constexpr size_t smem_fwd = sizeof(float2) * (NP * P + JR * NN);
    // inverse: A (own slab, read by the cluster) + B (own pencils, padded) + R (FP32 Qt, padded) + base
    static constexpr size_t smem_inv = sizeof(float2) * (JR * NN + NP * P) + sizeof(float) * NP * P +
                                       sizeof(double) * NP;
    static_assert(N % C == 0, "slabs must split evenly");
};

// Roots of unity exp(2 pi i t / N) in constant memory, one array per N: with
// the unrolled loops the index is a compile-time constant and every use is a
// constant-bank operand of the FMA (no registers, no loads).
__constant__ float2 c_root8[8], c_root12[12], c_root16[16], c_root24[24], c_root32[32];

template <int N> struct CRoot;
template <> struct CRoot<8> { static __device__ const float2 (&get())[8] { return c_root8; } };
template <> struct CRoot<12> { static __device__ const float2 (&get())[12] { return c_root12; } };
template <> struct CRoot<16> { static __device__ const float2 (&get())[16] { return c_root16; } };
template <> struct CRoot<24> { static __device__ const float2 (&get())[24] { return c_root24; } };
template <> struct CRoot<32> { static __device__ const float2 (&get())[32] { return c_root32; } };

// y_k = sum_j x_j W[k][j], W[k][j] = root[((k - N/2)(j - N/2)) mod N]
// (CONJ: conjugated), complex in and out,
// by the register FFT (the centred phases are a sign modulation of the
// plain DFT, see fft_reg.cuh).
template <int N, bool CONJ>
__device__ __forceinline__ void pencil_cc(const float2 (&x)[N], float2 (&y)[N], const float2 (&rt)[N]) {
#pragma unroll
    for (int j = 0; j < N; ++j) y[j] = x[j];
    fftr::centred<N, CONJ ? -1 : 1>(y, rt);
}

// real input, conjugated phases (forward first pass)
template <int N>
__device__ __forceinline__ void pencil_rc(const float (&x)[N], float2 (&y)[N], const float2 (&rt)[N]) {
#pragma unroll
    for (int j = 0; j < N; ++j) y[j] = make_float2(x[j], 0.f);
    fftr::centred<N, -1>(y, rt);
}

// real part of the output (inverse last pass)
template <int N>
__device__ __forceinline__ void pencil_cr(const float2 (&x)[N], float (&y)[N], const float2 (&rt)[N]) {
    float2 z[N];
#pragma unroll
    for (int j = 0; j < N; ++j) z[j] = x[j];
    fftr::centred<N, 1>(z, rt);
#pragma unroll
    for (int k = 0; k < N; ++k) y[k] = z[k].x;
}

// Cluster barrier without memory ordering: only keeps every CTA of the
// cluster resident until all of them got here (their remote reads of this
// CTA's shared memory have completed, since the values were consumed).
__device__ __forceinline__ void cluster_barrier_relaxed() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
}

// Barrier over the CTAs of a cell: a block barrier when the cell is one CTA
// (a cluster barrier would add a memory fence for nothing).
template <int C>
__device__ __forceinline__ void cell_sync(cg::cluster_group &cl) {
    if constexpr (C == 1) __syncthreads();
    else cl.sync();
}
template <int C, class T>
__device__ __forceinline__ T *cell_smem(cg::cluster_group &cl, T *p, int rank) {
    if constexpr (C == 1) return p;
    else return cl.map_shared_rank(p, rank);
}

// The N consecutive FP64 values of a pencil, narrowed to FP32 (integer pipes),
// with 16-byte loads when the pencil is 16-byte aligned; `bad` collects
// non-finite inputs.
template <int N>
__device__ __forceinline__ void load_pencil_f64(const double *__restrict__ fp, float (&x)[N], bool &bad) {
    if ((reinterpret_cast<uintptr_t>(fp) & 15u) == 0) {
        const double2 *f2 = reinterpret_cast<const double2 *>(fp);
#pragma unroll
        for (int j = 0; j < N / 2; ++j) {
            const double2 d = f2[j];
            bad |= !fpc::finite64(d.x) || !fpc::finite64(d.y);
            x[2 * j] = fpc::narrow(d.x);
            x[2 * j + 1] = fpc::narrow(d.y);
        }
    } else {
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const double d = fp[j];
            bad |= !fpc::finite64(d);
            x[j] = fpc::narrow(d);
        }
    }
}

}  // namespace

// Cell = cluster of C CTAs; CTA r owns the slab j1 in [r JR, (r+1) JR) of the
// first two passes and the slab k2 in [r JR, (r+1) JR) of the last one, whose
// pencils it reads from the owners' shared memory (distributed shared memory).
// SECTOR: fhat in the sector order of the group (sector_index) instead of the
// convolution's group layout.
template <int N, int C_, bool SECTOR = false>
__global__ void __cluster_dims__(C_, 1, 1) __launch_bounds__(FusedShape<N, C_>::NT)
dft_fwd_fused_kernel(const double *__restrict__ f, const int64_t *__restrict__ slot_off, DftSeg s,
                     const float2 *__restrict__ root, float scale, float2 *__restrict__ G, int *status) {
    using S = FusedShape<N, C_>;
    constexpr int M = S::M, NN = S::NN, P = S::P, JR = S::JR, C = S::C;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) char smem_raw[];
    float2 *A = reinterpret_cast<float2 *>(smem_raw);  // [jl][j2] rows of P, index k3
    float2 *B = A + S::NP * P;                          // [jl][k2][k3]
    const int r = (int)cl.block_rank(), sl = blockIdx.x / C, t = threadIdx.x;
    const int64_t off = slot_off[s.s0 + sl];
    if (off == -2) return;  // a slot of a group that holds no cell this call (nothing reads it)
    float2 *g = G + s.eoff + (int64_t)(sl / kLanes) * M * kLanes;
    const int ln = sl % kLanes;
    auto gi = [ln](int e) -> int64_t { return SECTOR ? sector_index(e, ln) : (int64_t)e * kLanes + ln; };
    if (off < 0) {  // padding lane of a group (the whole cluster leaves here): zero fhat
        for (int e = r * (M / C) + t; e < (r + 1) * (M / C); e += S::NT) g[gi(e)] = make_float2(0.f, 0.f);
        return;
    }
    const float2(&rt)[N] = CRoot<N>::get();
    const bool act = t < S::NP;
    bool bad = false;
    if (act) {  // along j3, pencil (j1, j2), real input
        const int jl = t / N, j2 = t % N;
        float x[N];
        load_pencil_f64<N>(f + off + (int64_t)((r * JR + jl) * N + j2) * N, x, bad);
        float2 y[N];
        pencil_rc<N>(x, y, rt);
#pragma unroll
        for (int k = 0; k < N; ++k) A[t * P + k] = y[k];
    }
    if (bad) atomicOr(status, ST_NONFINITE);
    __syncthreads();
    if (act) {  // along j2, pencil (j1, k3)
        const int jl = t / N, k3 = t % N;
        float2 x[N], y[N];
#pragma unroll
        for (int j = 0; j < N; ++j) x[j] = A[(jl * N + j) * P + k3];
        pencil_cc<N, true>(x, y, rt);
#pragma unroll
        for (int k = 0; k < N; ++k) B[(jl * N + k) * N + k3] = y[k];
    }
    cell_sync<C>(cl);
    if (act) {  // along j1, pencil (k2, k3), rows from every CTA of the cluster, into the group layout
        const int k2 = r * JR + t / N, k3 = t % N;
        const float2 *src[C];
#pragma unroll
        for (int o = 0; o < C; ++o) src[o] = cell_smem<C>(cl, B, o);
        float2 x[N], y[N];
#pragma unroll
        for (int j = 0; j < N; ++j) x[j] = src[j / JR][((j % JR) * N + k2) * N + k3];
        pencil_cc<N, true>(x, y, rt);
        const int pk = k2 * N + k3;
#pragma unroll
        for (int k = 0; k < N; ++k) g[gi(k * NN + pk)] = make_float2(scale * y[k].x, scale * y[k].y);
    }
    if constexpr (C > 1) cluster_barrier_relaxed();  // no CTA leaves while its slab may still be read
}

// Forward transform of a cell at the modes of a few zeta pencils only (the
// sampled pencils of the learned path's indicator): the pass along j3 for every
// (j1, j2) pencil, then for each sampled pencil (k1, k2) and each k3 the double
// sum over (j1, j2) with phase conj(root(k1', j1') root(k2', j2')). Writes the
// group layout at those modes only. One CTA per cell (N <= 16).
template <int N>
__global__ void __launch_bounds__(FusedShape<N, 1>::NT)
dft_fwd_pencils_kernel(const double *__restrict__ f, const int64_t *__restrict__ slot_off, DftSeg s, float scale,
                       const int *__restrict__ kks, int npen, float2 *__restrict__ G, int *status) {
    using S = FusedShape<N, 1>;
    constexpr int M = S::M, NN = S::NN, P = S::P, H = S::H;
    extern __shared__ __align__(16) char smem_raw[];
    float2 *A = reinterpret_cast<float2 *>(smem_raw);  // [j1][j2] rows of P, index k3
    const int sl = blockIdx.x, t = threadIdx.x;
    const int64_t off = slot_off[s.s0 + sl];
    if (off < 0) return;
    float2 *g = G + s.eoff + (int64_t)(sl / kLanes) * M * kLanes + (sl % kLanes);
    const float2(&rt)[N] = CRoot<N>::get();
    bool bad = false;
    if (t < NN) {  // along j3, pencil (j1, j2) = t, real input
        float x[N];
        load_pencil_f64<N>(f + off + (int64_t)t * N, x, bad);
        float2 y[N];
        pencil_rc<N>(x, y, rt);
#pragma unroll
        for (int k = 0; k < N; ++k) A[t * P + k] = y[k];
    }
    if (bad) atomicOr(status, ST_NONFINITE);
    __syncthreads();
    for (int o = t; o < npen * N; o += S::NT) {
        const int kk = kks[o / N], k3 = o % N, k1 = kk / N, k2 = kk % N;
        float re = 0.f, im = 0.f;
        for (int j1 = 0; j1 < N; ++j1) {
            const float2 r1 = rt[(((k1 - H) * (j1 - H)) % N + N) % N];
#pragma unroll
            for (int j2 = 0; j2 < N; ++j2) {
                const float2 r2 = rt[(((k2 - H) * (j2 - H)) % N + N) % N];
                // w = conj(r1 r2)
                const float wr = r1.x * r2.x - r1.y * r2.y, wi = -(r1.x * r2.y + r1.y * r2.x);
                const float2 a = A[(j1 * N + j2) * P + k3];
                re = fmaf(a.x, wr, fmaf(-a.y, wi, re));
                im = fmaf(a.x, wi, fmaf(a.y, wr, im));
            }
        }
        g[(int64_t)(kk * N + k3) * kLanes] = make_float2(scale * re, scale * im);
    }
}

// mode: 0 raw Qt; 1 P Qt; 2 P Qt and y = x + a Q; 3 P Qt and y += a (qp + Q)
// CTA r owns the slab k2 in [r JR, (r+1) JR) of the first pass and j1 in
// [r JR, (r+1) JR) of the other two; the second pass reads the first pass's
// rows from the whole cluster, and the moment partials of the CTAs are added
// in rank order by every CTA (the same lambda everywhere).
// FWD (mode 2 only): the first Heun stage's state f* = x + a Q is not written;
// its own slab, narrowed to FP32, is the input of the next stage's forward
// transform, which the cluster then runs as dft_fwd_fused_kernel would
// (the same passes on the same values: fhat of f* into Gout, scaled by
// fscale), in the inverse's shared memory.
template <int N, int C_, bool FWD = false>
__global__ void __cluster_dims__(C_, 1, 1) __launch_bounds__(FusedShape<N, C_>::NT)
dft_inv_fused_kernel(const float2 *__restrict__ G, const int64_t *__restrict__ slot_off, DftSeg s,
                     const float2 *__restrict__ root, float scale, double *__restrict__ q, ProjArgs pa,
                     int mode, const double *__restrict__ x, double *__restrict__ y,
                     const double *__restrict__ qp, double a, float2 *__restrict__ Gout = nullptr,
                     float fscale = 0.f, int *status = nullptr) {
    using S = FusedShape<N, C_>;
    constexpr int M = S::M, NN = S::NN, P = S::P, H = S::H, JR = S::JR, C = S::C, NP = S::NP;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) char smem_raw[];
    float2 *A = reinterpret_cast<float2 *>(smem_raw);  // [kl][j1][k3], read by the cluster
    float2 *B = A + JR * NN;                            // [jl][j2] rows of P, index k3
    float *R = reinterpret_cast<float *>(B + NP * P);   // Qt, [jl][j2] rows of P, index j3
    double *base = reinterpret_cast<double *>(R + NP * P);
    __shared__ float red[32][10];
    __shared__ float part[10];
    __shared__ double sg[N], lam[5];
    const int r = (int)cl.block_rank(), sl = blockIdx.x / C, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t off = slot_off[s.s0 + sl];
    if (off < 0) return;  // the whole cluster leaves
    // the time-update operands of the own slab are loaded first, so that their
    // memory latency overlaps the three passes
    constexpr int MS = M / C, IT = (MS + S::NT - 1) / S::NT;
    constexpr bool PF = IT <= 16;  // prefetch while the operands fit in registers
    const double *xo = x ? x + off + (int64_t)r * MS : nullptr;
    double *yo = y ? y + off + (int64_t)r * MS : nullptr;
    const double *qpo = qp ? qp + off + (int64_t)r * MS : nullptr;
    double u[PF ? IT : 1], w[PF ? IT : 1];
    if (!PF) {
    } else if (mode == 2) {
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            const int e = t + i * S::NT;
            u[i] = e < MS ? xo[e] : 0.0;
        }
    } else if (mode == 3) {
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            const int e = t + i * S::NT;
            u[i] = e < MS ? yo[e] : 0.0;
            w[i] = e < MS ? qpo[e] : 0.0;
        }
    }
    const float2(&rt)[N] = CRoot<N>::get();
    const bool act = t < NP;
    const float2 *g = G + s.eoff + (int64_t)(sl / kLanes) * M * kLanes + (sl % kLanes);
    if (act) {  // along k1, pencil (k2, k3), from the group layout
        const int pk = (r * JR + t / N) * N + t % N;
        float2 xx[N], yy[N];
#pragma unroll
        for (int k = 0; k < N; ++k) xx[k] = g[(int64_t)(k * NN + pk) * kLanes];
        pencil_cc<N, false>(xx, yy, rt);
        const int kl = t / N, k3 = t % N;
#pragma unroll
        for (int j = 0; j < N; ++j) A[(kl * N + j) * N + k3] = yy[j];
    }
    cell_sync<C>(cl);
    if (act) {  // along k2, pencil (j1, k3), rows from every CTA of the cluster
        const int j1 = r * JR + t / N, k3 = t % N;
        const float2 *src[C];
#pragma unroll
        for (int o = 0; o < C; ++o) src[o] = cell_smem<C>(cl, A, o);
        float2 xx[N], yy[N];
#pragma unroll
        for (int k = 0; k < N; ++k) xx[k] = src[k / JR][((k % JR) * N + j1) * N + k3];
        pencil_cc<N, false>(xx, yy, rt);
        const int jl = t / N;
#pragma unroll
        for (int j = 0; j < N; ++j) B[(jl * N + j) * P + k3] = yy[j];
    }
    cell_sync<C>(cl);  // all remote reads of A are done (no CTA may leave earlier)
    // along k3, real part, pencil (j1, j2); per-pencil moment sums in double-float
    Df mom[5];
    if (act) {
        float2 xx[N];
        float rr[N];
#pragma unroll
        for (int k = 0; k < N; ++k) xx[k] = B[t * P + k];
        pencil_cr<N>(xx, rr, rt);
        Df s0{0.f, 0.f}, s1{0.f, 0.f}, s2{0.f, 0.f};
#pragma unroll
        for (int j = 0; j < N; ++j) {
            rr[j] *= scale;
            R[t * P + j] = rr[j];
            df_add(s0, rr[j]);
            df_add_prod(s1, (float)(j - H), rr[j]);
            df_add_prod(s2, (float)((j - H) * (j - H)), rr[j]);
        }
        const int w1 = r * JR + t / N - H, w2 = t % N - H;
        mom[0] = s0;
        mom[1] = df_mul_int(s0, (float)w1);
        mom[2] = df_mul_int(s0, (float)w2);
        mom[3] = s1;
        mom[4] = df_add(df_mul_int(s0, (float)(w1 * w1 + w2 * w2)), s2);
    } else {
#pragma unroll
        for (int i = 0; i < 5; ++i) mom[i] = Df{0.f, 0.f};
    }
    if (mode != 0) {
        // moments: warp trees, warp 0 over the CTA's warps, then the cluster's partials in rank order
#pragma unroll
        for (int i = 0; i < 5; ++i) mom[i] = df_warp_sum(mom[i]);
        if (S::NW > 1) {
            if (lane == 0)
#pragma unroll
                for (int i = 0; i < 5; ++i) {
                    red[warp][2 * i] = mom[i].hi;
                    red[warp][2 * i + 1] = mom[i].lo;
                }
            __syncthreads();
            if (warp == 0) {
#pragma unroll
                for (int i = 0; i < 5; ++i)
                    mom[i] = lane < S::NW ? Df{red[lane][2 * i], red[lane][2 * i + 1]} : Df{0.f, 0.f};
#pragma unroll
                for (int i = 0; i < 5; ++i) mom[i] = df_warp_sum(mom[i]);
            }
        }
        if (t == 0)
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                part[2 * i] = mom[i].hi;
                part[2 * i + 1] = mom[i].lo;
            }
        cell_sync<C>(cl);
        if (warp == 0) {
            double mu = 0.0;
            if (lane < 5) {
                Df m{0.f, 0.f};
#pragma unroll
                for (int o = 0; o < C; ++o) {
                    const float *po = cell_smem<C>(cl, part, o);
                    m = df_add(m, Df{po[2 * lane], po[2 * lane + 1]});
                }
                // mu = (sum q, dv sum w_d q (d = 1..3), dv^2 sum |w|^2 q), w = j - N/2
                const double sc = lane == 0 ? 1.0 : (lane == 4 ? pa.dv * pa.dv : pa.dv);
                mu = ((double)m.hi + (double)m.lo) * sc;
            }
            double m5[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) m5[i] = __shfl_sync(0xffffffffu, mu, i);
            if (lane < 5) {
                double l = 0.0;
#pragma unroll
                for (int k = 0; k < 5; ++k) l = fma(pa.ainv[lane * 5 + k], m5[k], l);
                lam[lane] = l;
            }
        }
        cell_sync<C>(cl);  // every CTA has read the partials before any leaves; lambda is visible
        // correction C^T lambda = base(j1, j2) + g(j3)
        const double dv = pa.dv;
        if (t < N) {
            const double v = dv * (double)(t - H);
            sg[t] = fma(lam[3], v, lam[4] * v * v);
        }
        if (act) {
            const double v1 = dv * (double)(r * JR + t / N - H), v2 = dv * (double)(t % N - H);
            base[t] = lam[0] + fma(lam[1], v1, fma(lam[2], v2, lam[4] * fma(v1, v1, v2 * v2)));
        }
    }
    __syncthreads();
    // coalesced output of the own slab: local value e = (pencil p, j3)
    double *qo = q + off + (int64_t)r * MS;
    if (mode == 0) {
        for (int e = t; e < MS; e += S::NT) qo[e] = fpc::widen(R[(e / N) * P + e % N]);
        return;
    }
    bool bad = false;  // FWD: a non-finite f*
    if constexpr (PF) {
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            const int e = t + i * S::NT;
            if (e < MS) {
                const int p = e / N, j3 = e % N;
                const double v = fpc::widen(R[p * P + j3]) - (base[p] + sg[j3]);
                qo[e] = v;
                if constexpr (FWD) {
                    const double fs = fma(a, v, u[i]);
                    bad |= !fpc::finite64(fs);
                    R[p * P + j3] = fpc::narrow(fs);  // each value is read and rewritten by this thread only
                } else if (mode == 2) {
                    yo[e] = fma(a, v, u[i]);
                } else if (mode == 3) {
                    yo[e] = fma(a, w[i] + v, u[i]);
                }
            }
        }
    } else {
#pragma unroll 4
        for (int e = t; e < MS; e += S::NT) {
            const int p = e / N, j3 = e % N;
            const double v = fpc::widen(R[p * P + j3]) - (base[p] + sg[j3]);
            qo[e] = v;
            if constexpr (FWD) {
                const double fs = fma(a, v, xo[e]);
                bad |= !fpc::finite64(fs);
                R[p * P + j3] = fpc::narrow(fs);
            } else if (mode == 2) {
                yo[e] = fma(a, v, xo[e]);
            } else if (mode == 3) {
                yo[e] = fma(a, qpo[e] + v, yo[e]);
            }
        }
    }
    (void)bad;
    if constexpr (FWD) {
        // the next stage's forward transform of f*: the passes of dft_fwd_fused_kernel
        // with its regions in this kernel's (same sizes): pencil rows in B, own slab in A
        if (bad) atomicOr(status, ST_NONFINITE);
        __syncthreads();
        float2 *Af = B;  // [jl][j2] rows of P, index k3
        float2 *Bf = A;  // [jl][k2][k3], read by the cluster (A's remote reads ended several cluster barriers ago)
        if (act) {  // along j3, pencil (j1, j2) = own pencil t, real input
            float xr[N];
#pragma unroll
            for (int j = 0; j < N; ++j) xr[j] = R[t * P + j];
            float2 yv[N];
            pencil_rc<N>(xr, yv, rt);
#pragma unroll
            for (int k = 0; k < N; ++k) Af[t * P + k] = yv[k];
        }
        __syncthreads();
        if (act) {  // along j2, pencil (j1, k3)
            const int jl = t / N, k3 = t % N;
            float2 xx[N], yy[N];
#pragma unroll
            for (int j = 0; j < N; ++j) xx[j] = Af[(jl * N + j) * P + k3];
            pencil_cc<N, true>(xx, yy, rt);
#pragma unroll
            for (int k = 0; k < N; ++k) Bf[(jl * N + k) * N + k3] = yy[k];
        }
        cell_sync<C>(cl);
        if (act) {  // along j1, pencil (k2, k3), rows from every CTA of the cluster, into the group layout
            const int k2 = r * JR + t / N, k3 = t % N;
            const float2 *src[C];
#pragma unroll
            for (int o = 0; o < C; ++o) src[o] = cell_smem<C>(cl, Bf, o);
            float2 xx[N], yy[N];
#pragma unroll
            for (int j = 0; j < N; ++j) xx[j] = src[j / JR][((j % JR) * N + k2) * N + k3];
            pencil_cc<N, true>(xx, yy, rt);
            float2 *go = Gout + s.eoff + (int64_t)(sl / kLanes) * M * kLanes + (sl % kLanes);
            const int pk = k2 * N + k3;
#pragma unroll
            for (int k = 0; k < N; ++k)
                go[(int64_t)(k * NN + pk) * kLanes] = make_float2(fscale * yy[k].x, fscale * yy[k].y);
        }
        if constexpr (C > 1) cluster_barrier_relaxed();  // no CTA leaves while its slab may still be read
    }
}

namespace {
template <int N, int C>
void fwd_launch(const double *f, const int64_t *slot_off, const DftSeg &s, const float2 *root, double scale,
                float2 *G, int *status, cudaStream_t st, bool sector) {
    using S = FusedShape<N, C>;
    if constexpr (N <= 16) {
        if (sector) {
            dft_fwd_fused_kernel<N, C, true><<<s.nslots * C, S::NT, S::smem_fwd, st>>>(f, slot_off, s, root,
                                                                                      (float)scale, G, status);
            return;
        }
    }
    dft_fwd_fused_kernel<N, C><<<s.nslots * C, S::NT, S::smem_fwd, st>>>(f, slot_off, s, root, (float)scale, G,
                                                                        status);
}
template <int N, int C>
void inv_launch(const float2 *G, const int64_t *slot_off, const DftSeg &s, const float2 *root, double scale,
                double *q, const ProjArgs &pa, int mode, const double *x, double *y, const double *qp, double a,
                cudaStream_t st) {
    using S = FusedShape<N, C>;
    dft_inv_fused_kernel<N, C><<<s.nslots * C, S::NT, S::smem_inv, st>>>(G, slot_off, s, root, (float)scale, q, pa,
                                                                        mode, x, y, qp, a);
}
template <int N, int C>
void inv_fwd_launch(const float2 *G, const int64_t *slot_off, const DftSeg &s, const float2 *root, double scale,
                    double *q, const ProjArgs &pa, const double *x, double a, double fscale, float2 *Gout,
                    int *status, cudaStream_t st) {
    using S = FusedShape<N, C>;
    dft_inv_fused_kernel<N, C, true><<<s.nslots * C, S::NT, S::smem_inv, st>>>(
        G, slot_off, s, root, (float)scale, q, pa, 2, x, nullptr, nullptr, a, Gout, (float)fscale, status);
}
template <int N, int C>
void prepare_one() {
    using S = FusedShape<N, C>;
    cudaFuncSetAttribute(dft_fwd_fused_kernel<N, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem_fwd);
    if constexpr (N <= 16)
        cudaFuncSetAttribute(dft_fwd_fused_kernel<N, C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)S::smem_fwd);
    cudaFuncSetAttribute(dft_inv_fused_kernel<N, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem_inv);
    cudaFuncSetAttribute(dft_inv_fused_kernel<N, C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)S::smem_inv);
}
template <int N>
void prepare_n() {
    prepare_one<N, 1>();
    prepare_one<N, 2>();
    prepare_one<N, 4>();
}
int norm_split(int split) { return split == 1 || split == 2 ? split : 4; }
template <int N>
void upload_roots(const float2 (&sym)[N]) {
    float2 h[N];
    for (int t = 0; t < N; ++t) {
        const double th = 2.0 * 3.14159265358979323846 * t / N;
        h[t] = make_float2((float)std::cos(th), (float)std::sin(th));
    }
    cudaMemcpyToSymbol(sym, h, sizeof(h));
}
}  // namespace

bool fused_dft_supported(int N) { return N == 8 || N == 12 || N == 16 || N == 24 || N == 32; }

void fused_dft_prepare(int N) {
    // roots of unity (constant memory is per device) and shared-memory
    // attributes; must happen outside stream capture
    static std::map<int, unsigned> done;  // device -> bit N of the uploaded root tables
    static std::mutex mu;                   // contexts on several host threads share the map
    std::lock_guard<std::mutex> lock(mu);
    int dev = 0;
    cudaGetDevice(&dev);
    if (N < 0 || N > 32 || (done[dev] >> N) & 1u) return;
    switch (N) {
        case 8: upload_roots<8>(c_root8); prepare_n<8>(); break;
        case 12: upload_roots<12>(c_root12); prepare_n<12>(); break;
        case 16: upload_roots<16>(c_root16); prepare_n<16>(); break;
        case 24: upload_roots<24>(c_root24); prepare_one<24, 4>(); break;
        case 32: upload_roots<32>(c_root32); prepare_one<32, 8>(); break;
        default: return;
    }
    done[dev] |= 1u << N;
}

#define BTE_SPLIT_DISPATCH(FN, N, ...)                 \
    switch (norm_split(split)) {                       \
        case 1: FN<N, 1>(__VA_ARGS__); break;          \
        case 2: FN<N, 2>(__VA_ARGS__); break;          \
        default: FN<N, 4>(__VA_ARGS__); break;         \
    }

void launch_dft_forward_pencils(const double *f, const int64_t *slot_off, const DftSeg &s, double scale,
                                const int *kks, int npen, float2 *G, int *status, cudaStream_t st) {
    switch (s.N) {
        case 8: dft_fwd_pencils_kernel<8><<<s.nslots, FusedShape<8, 1>::NT, sizeof(float2) * 64 * 9, st>>>(
                    f, slot_off, s, (float)scale, kks, npen, G, status);
            break;
        case 12: dft_fwd_pencils_kernel<12><<<s.nslots, FusedShape<12, 1>::NT, sizeof(float2) * 144 * 13, st>>>(
                    f, slot_off, s, (float)scale, kks, npen, G, status);
            break;
        case 16: dft_fwd_pencils_kernel<16><<<s.nslots, FusedShape<16, 1>::NT, sizeof(float2) * 256 * 17, st>>>(
                    f, slot_off, s, (float)scale, kks, npen, G, status);
            break;
        default: break;
    }
}

void launch_dft_forward_fused(const double *f, const int64_t *slot_off, const DftSeg &s, const float2 *root,
                              double scale, float2 *G, int *status, cudaStream_t st, int split, bool sector) {
    switch (s.N) {
        case 8: BTE_SPLIT_DISPATCH(fwd_launch, 8, f, slot_off, s, root, scale, G, status, st, sector) break;
        case 12: BTE_SPLIT_DISPATCH(fwd_launch, 12, f, slot_off, s, root, scale, G, status, st, sector) break;
        case 16: BTE_SPLIT_DISPATCH(fwd_launch, 16, f, slot_off, s, root, scale, G, status, st, sector) break;
        case 24: fwd_launch<24, 4>(f, slot_off, s, root, scale, G, status, st, false); break;
        case 32: fwd_launch<32, 8>(f, slot_off, s, root, scale, G, status, st, false); break;
        default: break;
    }
}

void launch_dft_inverse_fused(const float2 *G, const int64_t *slot_off, const DftSeg &s, const float2 *root,
                              double scale, double *q, const ProjArgs &pa, int mode, const double *x, double *y,
                              const double *qp, double a, cudaStream_t st, int split) {
    switch (s.N) {
        case 8: BTE_SPLIT_DISPATCH(inv_launch, 8, G, slot_off, s, root, scale, q, pa, mode, x, y, qp, a, st) break;
        case 12: BTE_SPLIT_DISPATCH(inv_launch, 12, G, slot_off, s, root, scale, q, pa, mode, x, y, qp, a, st) break;
        case 16: BTE_SPLIT_DISPATCH(inv_launch, 16, G, slot_off, s, root, scale, q, pa, mode, x, y, qp, a, st) break;
        case 24: inv_launch<24, 4>(G, slot_off, s, root, scale, q, pa, mode, x, y, qp, a, st); break;
        case 32: inv_launch<32, 8>(G, slot_off, s, root, scale, q, pa, mode, x, y, qp, a, st); break;
        default: break;
    }
}
bool inverse_forward_fused_supported(int N, int) { return fused_dft_supported(N); }

void launch_dft_inverse_forward_fused(const float2 *G, const int64_t *slot_off, const DftSeg &s,
                                      const float2 *root, double scale, double *q, const ProjArgs &pa,
                                      const double *x, double a, double fscale, float2 *Gout, int *status,
                                      cudaStream_t st, int split) {
    switch (s.N) {
        case 8:
        case 12:
        case 16:
            switch (norm_split(split)) {
                case 1:
                    if (s.N == 8) inv_fwd_launch<8, 1>(G, slot_off, s, root, scale, q, pa, x, a, fscale, Gout, status, st);
                    else if (s.N == 12) inv_fwd_launch<12, 1>(G, slot_off, s, root, scale, q, pa, x, a, fscale, Gout, status, st);
                    else inv_fwd_launch<16, 1>(G, slot_off, s, root, scale, q, pa, x, a, fscale, Gout, status, st);
                    break;
                case 2:
                    if (s.N == 8) inv_fwd_launch<8, 2>(G, slot_off, s, root, scale, q, pa, x, a, fscale, Gout, status, st);
                    else if (s.N == 12) inv_fwd_launch<12, 2>(G, slot_off, s, root, scale, q, pa, x, a, fscale, Gout, status, st);
                    else inv_fwd_launch<16, 2>(G, slot_off, s, root, scale, q, pa, x, a, fscale, Gout, status, st);
                    break;
                default:
                    if (s.N == 8) inv_fwd_launch<8, 4>(G, slot_off, s, root, scale, q, pa, x, a, fscale, Gout, status, st);
                    else if (s.N == 12) inv_fwd_launch<12, 4>(G, slot_off, s, root, scale, q, pa, x, a, fscale, Gout, status, st);
                    else inv_fwd_launch<16, 4>(G, slot_off, s, root, scale, q, pa, x, a, fscale, Gout, status, st);
                    break;
            }
            break;
        case 24: inv_fwd_launch<24, 4>(G, slot_off, s, root, scale, q, pa, x, a, fscale, Gout, status, st); break;
        case 32: inv_fwd_launch<32, 8>(G, slot_off, s, root, scale, q, pa, x, a, fscale, Gout, status, st); break;
        default: break;
    }
}
#undef BTE_SPLIT_DISPATCH

}  // namespace bte
