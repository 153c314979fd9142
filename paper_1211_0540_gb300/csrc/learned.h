// Residual indicator of the learned path (internal).
#pragma once

#include <cstdint>

#include "bte_internal.h"

namespace bte {

struct IndicatorTable {
    int S = 0;
    float2 *d_w = nullptr;  // per sample: (full, loss) weights times dz^3 over the valid box of k
    int *d_off = nullptr;   // first weight of each sample
    int *d_k = nullptr;     // sampled zeta indices
};

int build_indicator_table(const Table &t, int S, uint64_t seed, IndicatorTable &out);
void free_indicator_table(IndicatorTable &t);
// ind[slot] for the slots of one segment (eoff: its offset in the group buffers).
void launch_indicator(const IndicatorTable &it, const float2 *F, const float2 *QN, int N, int64_t eoff, int nslots,
                      int nvalid, float *err2, float *den2, float *ind, cudaStream_t st);

}  // namespace bte
