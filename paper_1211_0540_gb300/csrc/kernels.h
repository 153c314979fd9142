// Launch interfaces of the CUDA kernels (internal).
#pragma once

#include "bte_internal.h"

namespace bte {

// One segment of a batch: slots [s0, s0 + nslots) that share a weight table
// (hence N). nslots is a multiple of 32 (padding slots have offset -1).
struct DftSeg {
    int N;
    int s0;        // first slot of the segment (global slot index)
    int nslots;    // slots in the segment (multiple of 32)
    int64_t eoff;  // complex-element offset of slot s0 in scratch / group buffers
};

// Projection (Sec. 3.3), optionally fused with the RK2 update:
// mode 0: Q <- P Q;  mode 1: Q <- P Q, Y <- X + a Q;  mode 2: Q <- P Q, Y <- Y + a (Qp + Q).
struct ProjArgs {
    int N;
    double dv;
    double ainv[25];
};

template <typename C>
void launch_dft_forward(const double *f, const int64_t *slot_off, const DftSeg &s, const C *root,
                        double scale, C *T1, C *T2, C *G, int *status, cudaStream_t st);
template <typename C>
void launch_dft_inverse(const C *G, const int64_t *slot_off, const DftSeg &s, const C *root,
                        double scale, C *T1, C *T2, double *q, cudaStream_t st);

// FP32 convolution (persistent, work queue of ConvItems).
constexpr int kMaxTables = 16;
struct ConvParams {
    const ConvItem *items;
    int nitems;
    const int *nitems_dev = nullptr;  // variants 4, 5: item count read from the device when set
    unsigned *counter;
    const float2 *F;
    float2 *Qh;
    const float *W[kMaxTables];
    const uint32_t *D[kMaxTables];
    int *status;
    int stages;     // pipeline depth per warp (1..4)
    int merge;      // blocks per TwoSum merge
    int warp_smem;  // bytes of ring per warp
    int stall;      // testing the timeout path: each warp never issues its first block
    // Items split into two block ranges (conv_impl 4 only; null: no splits).
    // split[i] = -1, or 2 sid + half: the two halves write their reduced sums to
    // part[(2 sid + half) * kSplitFloats ...]; the CTA that finishes second
    // (split_cnt[sid], zeroed before the launch) adds half 0 and half 1 in that
    // order and writes Q.
    const int *split;
    float *part;
    unsigned *split_cnt;
    // Weights built on the fly (conv_impl 5): per table the FP32 radial tables
    // I32[p * nq + q] and J32[s] (already times sqrt(2/pi) dz^3) and per block
    // entry (consumption order) the third components of the invariants,
    // E + 4 (tile * estride + e): k3'^2, (2m3' - k3')^2, m3'^2, n3'^2.
    const float *I32[kMaxTables];
    const float *J32[kMaxTables];
    const uint16_t *E[kMaxTables];
    int nq[kMaxTables];
    int estride[kMaxTables];
};
constexpr int kSplitFloats = 16 * 4 * 32;  // per half: T <= 16 outputs x (hi, lo) x (re, im) x 32 lanes
int conv_stage_bytes(int kind);
struct ConvLaunch {
    void (*fn)(ConvParams);
    int grid, threads, stages, warp_smem, impl;
    size_t smem;
};
// kinds_mask: bit i set when items of kind i are present. Sets the kernel's
// shared-memory attribute: call outside stream capture.
// impl: 0 = one warp per item, 1 = CTA-cooperative items, 2 = cooperative + packed f32x2,
// 3 = as 2 at 2 CTAs per SM, 4 = as 2 with the compensated sums in shared memory,
// 5 = as 4 with every block's weights built on the fly from the radial tables.
cudaError_t conv32_configure(unsigned kinds_mask, int num_sms, int warps_per_cta, int stages, int impl,
                             ConvLaunch *out);
cudaError_t conv32_launch(const ConvLaunch &L, const ConvParams &p, cudaStream_t st);

// Plain FP64 convolution of one segment.
void launch_conv64(const double2 *F, double2 *Qh, const double *W, const uint64_t *Woff, int N,
                   int64_t eoff, int ngroups, cudaStream_t st);
// the same for a segment with few valid cells: one warp per (valid slot, zeta)
void launch_conv64_cells(const double2 *F, double2 *Qh, const double *W, const uint64_t *Woff,
                         const int64_t *slot_off, int s0, int nslots, int N, int64_t eoff, cudaStream_t st);

void launch_project(double *Q, const int64_t *slot_off, int s0, int nslots, const ProjArgs &pa,
                    int mode, const double *X, double *Y, const double *Qp, double a,
                    cudaStream_t st);
void launch_moments(const double *f, const int64_t *slot_off, int s0, int nslots, int N, double dv,
                    const int64_t *slot_out, double *out, cudaStream_t st);

// Fused single-kernel transforms for N in {8, 12, 16} (dft_fused.cu).
// Inverse mode: 0 raw Qt; 1 P Qt; 2 P Qt and y = x + a Q; 3 P Qt and y += a (qp + Q).
bool fused_dft_supported(int N);
void fused_dft_prepare(int N);  // outside stream capture
// forward transform of N <= 16 cells at the modes of npen zeta pencils kks[] (k1 N + k2) only
void launch_dft_forward_pencils(const double *f, const int64_t *slot_off, const DftSeg &s, double scale,
                                const int *kks, int npen, float2 *G, int *status, cudaStream_t st);
// Sector order of a group of fhat (the fallback indicator's input, N <= 16):
// mode e of lane l at (e / 4) 128 + 4 l + e mod 4, so that four consecutive
// modes of one cell fill one 32-byte sector and the forward transform, which
// holds one cell per CTA, stores whole sectors (the group layout of the
// convolution, 32 e + l, takes one 8-byte piece of a sector per store).
__host__ __device__ __forceinline__ int64_t sector_index(int64_t e, int lane) {
    return ((e >> 2) << 7) + ((int64_t)lane << 2) + (e & 3);
}
// split: CTAs (a thread-block cluster) per cell, 1, 2 or 4 (other values: 4);
// sector: fhat in the sector order (N <= 16) instead of the convolution's
// group layout
void launch_dft_forward_fused(const double *f, const int64_t *slot_off, const DftSeg &s, const float2 *root,
                              double scale, float2 *G, int *status, cudaStream_t st, int split = 4,
                              bool sector = false);
void launch_dft_inverse_fused(const float2 *G, const int64_t *slot_off, const DftSeg &s, const float2 *root,
                              double scale, double *q, const ProjArgs &pa, int mode, const double *x, double *y,
                              const double *qp, double a, cudaStream_t st, int split = 4);
// The first Heun stage's inverse (mode 2: Q = P Qt into q) fused with the second
// stage's forward transform: f* = x + a Q is not stored; fhat(f*) (times fscale)
// goes to Gout in the group layout. Same results as the inverse (mode 2) followed
// by launch_dft_forward_fused on f*. Supported wherever the fused transforms are.
bool inverse_forward_fused_supported(int N, int split);
void launch_dft_inverse_forward_fused(const float2 *G, const int64_t *slot_off, const DftSeg &s,
                                      const float2 *root, double scale, double *q, const ProjArgs &pa,
                                      const double *x, double a, double fscale, float2 *Gout, int *status,
                                      cudaStream_t st, int split = 4);

// Transport (Sec. 3.4) on nx uniform cells of M values. mw_*: wall Maxwellians
// per velocity (device, M doubles), den_*: sum over the incoming half of |v.n| M_w.
constexpr int kTransportMaxN = 32;
struct TransportArgs {
    int N, nx;
    double dv, dx;
    int bc_left, bc_right;
    const double *mw_left, *mw_right;
    double den_left, den_right;
    // cells of unequal width (null: uniform dx): device arrays alpha, gamma
    // (cells -1 .. nx, index c + 1) and 1/dx (cells 0 .. nx-1); see transport.cu
    const double *g_alpha = nullptr, *g_gamma = nullptr, *g_rdx = nullptr;
    // filled per sub-step by launch_transport_half:
    double rden_left, rden_right;   // 1 / den (0 when den is 0)
    double kv[kTransportMaxN];      // (tau / dx) v1_i,  v1_i = dv (i - N/2)
    double kvh[kTransportMaxN];     // kv / 2
    double wv[kTransportMaxN];      // |v1_i|
};
// One transport half step of the slab f (in place); f1 and fh are scratch of f's size.
void launch_transport_half(double *f, double *f1, double *fh, const TransportArgs &ta, double tau,
                           cudaStream_t st);

}  // namespace bte
