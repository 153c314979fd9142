// Residual indicator of the learned path (internal).
#pragma once

#include <cstdint>
#include <vector>

#include "kernels.h"

namespace bte {

// Sampled pencils of the indicator: for pencil i, the kept (m1, m2) blocks of
// zeta pencil kk = k1 N + k2 (descriptors and full weights of the FP32 table)
// and the loss-term weights of the same blocks (d_wloss + wofs_loss).
struct IndPencil {
    int kk, desc_off, nblocks, pad;
    uint64_t wofs_full, wofs_loss;
};

struct IndicatorTable {
    int S = 0;                     // sampled pencils (S x N sampled modes)
    std::vector<int> kks;          // host copy of the sampled pencils (k1 N + k2), drawing order
    float *d_wloss = nullptr;      // loss weights of the sampled pencils (pair-symmetrised, times dz^3)
    IndPencil *d_pen = nullptr;
    int *d_kk = nullptr;           // the sampled pencils' k1 N + k2
};

// modes: about this many sampled modes (pencils = modes / N, at least 1)
int build_indicator_table(const Table &t, int modes, uint64_t seed, IndicatorTable &out);
void free_indicator_table(IndicatorTable &t);
// Q = P_N(rho^2 Y / s_out) for B contiguous cells of N^3 values (N <= 16).
void launch_post_project(const float *Y, const double *rho, int B, int N, float s_out, const ProjArgs &pa, double *Q,
                         cudaStream_t st);
// ind[slot] for the slots of one segment (eoff: its offset in the group buffers;
// F: fhat of f in the sector order of each group (sector_index), QN: fhat of
// the projected surrogate output at the sampled pencils, group layout);
// err2, den2: S * nslots floats of scratch each, ind: nslots floats followed by
// the kernel's own scratch (indicator_scratch_floats counts all of it).
size_t indicator_scratch_floats(const IndicatorTable &it, int N, int nslots);
// out[i] = (double) in[i], i < n
void launch_widen(const float *in, double *out, int n, cudaStream_t st);
// The learned mode's fallback batch on the device (learned.cu): flagged cells
// (ind > tol), offsets (-1 padding lanes, -2 unused groups), work list, its
// length, the zeroed queue counter; statistics (cells, fallbacks, max ind bits).
void launch_fallback_setup(const float *ind, int ncells, double tol, int64_t M, const ConvItem *tmpl, int ntmpl,
                           int nslots_cap, int64_t *off, ConvItem *items, int *nitems, unsigned *counter,
                           unsigned long long *stats, cudaStream_t st);
// Heun stage update with a given Q: mode 1 y = x + a Q, mode 2 y += a (qp + Q).
void launch_stage_update(const double *Q, const double *x, double *y, const double *qp, double a, int64_t n,
                         int mode, cudaStream_t st);
void launch_indicator(const IndicatorTable &it, const Table &t, const float2 *F, const float2 *QN, int64_t eoff,
                      int nslots, int nvalid, float *err2, float *den2, float *ind, cudaStream_t st);

}  // namespace bte
