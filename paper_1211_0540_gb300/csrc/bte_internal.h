// Internal declarations of libbte (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/bte.h"

namespace bte {

// Device status bits (atomicOr'ed by kernels, read by bte_sync_status).
enum : int { ST_TIMEOUT = 1, ST_NONFINITE = 2, ST_BADDESC = 4 };

constexpr int kLanes = 32;  // cells per group: one warp lane per cell

// ----------------------------------------------------------------------------
// Convolution kernel variants: N, k3-tile size T and tile origin K0.
// ----------------------------------------------------------------------------
struct ConvKind {
    int N, T, K0;
};
constexpr int kNumKinds = 10;
// kind ids: 0:(8,8,0) 1:(12,12,0) 2:(16,16,0) 3:(24,12,0) 4:(24,12,12) 5:(32,16,0) 6:(32,16,16)
//           7:(48,16,0) 8:(48,16,16) 9:(48,16,32)
inline ConvKind conv_kind(int id) {
    static const ConvKind k[kNumKinds] = {{8, 8, 0},    {12, 12, 0},  {16, 16, 0}, {24, 12, 0},  {24, 12, 12},
                                          {32, 16, 0},  {32, 16, 16}, {48, 16, 0}, {48, 16, 16}, {48, 16, 32}};
    return k[id];
}
int first_kind_for_N(int N);  // -1 if unsupported
int tiles_for_N(int N);
constexpr int kMaxTiles = 3;

// One warp-sized unit of convolution work: cell group g (32 lanes), pencil
// (k1, k2), k3 tile. Sorted by cost (descending) before upload.
struct ConvItem {
    uint64_t fofs;       // float2 offset of the group's fhat ([m][lane]) == qhat offset
    uint64_t wofs;       // float offset of the first weight block
    uint32_t desc_off;   // first (m1, m2) descriptor of the pencil
    uint32_t nblocks;    // kept (m1, m2) blocks of the pencil
    uint16_t k1, k2;
    uint16_t kind;       // ConvKind id
    uint16_t table;      // weight table index
};
static_assert(sizeof(ConvItem) == 32, "ConvItem layout");

// Per-grid weight table and constants.
struct Table {
    int N = 0;
    double L = 0, lam = 0;
    double beta = 1.0;  // restitution parameter of the collision rule (1: elastic)
    int ntiles = 0;
    int kind0 = 0;
    double dv = 0, dz = 0;
    // FP32 pair-symmetrised weights (times dz^3): [tile][k1][k2][block][cpad]
    std::vector<uint64_t> wofs;          // per (tile, k1, k2)
    std::vector<uint32_t> desc_off;      // per (k1, k2)
    std::vector<uint32_t> nblocks;       // per (k1, k2)
    int cpad[kMaxTiles] = {0, 0, 0};
    size_t n_w32 = 0, n_desc = 0;
    float *d_w32 = nullptr;
    uint32_t *d_desc = nullptr;          // m1 | (m2 << 16)
    // FP64 plain table (times dz^3), valid boxes, zeta-major; built lazily.
    double *d_w64 = nullptr;
    uint64_t *d_w64_off = nullptr;       // per k (M + 1 entries)
    size_t n_w64 = 0;
    // On-the-fly weights (beta = 1): I and J in FP32 times sqrt(2/pi) dz^3, and
    // per k3 tile and block entry (kernel order) the third components of the
    // weight invariants as four 16-bit fields (estride entries per tile)
    float *d_I32 = nullptr, *d_J32 = nullptr;
    uint16_t *d_etab = nullptr;
    int estride = 0;
    // Work items of one 32-cell group (fofs 0, table 0), every k3 tile and
    // pencil with kept blocks, costliest first: the set-up-time template from
    // which bte_collide_noalloc expands its work list on the device.
    ConvItem *d_tmpl = nullptr;
    int n_tmpl = 0;
    // DFT roots exp(2 pi i t / N), t in [0, N)
    float2 *d_root32 = nullptr;
    double2 *d_root64 = nullptr;
    // Projection: (C C^T)^{-1}, row-major 5x5 (C without the dv^3 factor folded in)
    double ainv[25];
    // Host FP64 radial tables on integer invariants (kept for the lazy FP64 table)
    std::vector<double> I, J;            // I[p * nq + q], J[s]
    int np = 0, nq = 0, ns = 0;
    // the convolution kinds of this table's k3 tiles (bit kind0 + tile)
    unsigned kinds_mask() const {
        unsigned m = 0;
        for (int i = 0; i < ntiles; ++i) m |= 1u << (kind0 + i);
        return m;
    }
    std::vector<uint32_t> desc_host;     // block descriptors (host copy, for the lazy FP32 table)
    double ghat(int k1, int k2, int k3, int m1, int m2, int m3) const;  // FP64, no dz^3
    double gain_inelastic(double a, double b) const;                    // I(a, b) off the lattice
};

struct GraphKey {
    int64_t ninst;
    int table, mode, transport;
    double dt, eps;
    const void *f;
    void *stream;
    bool operator<(const GraphKey &o) const;
};

// One configuration of the FP32 path (convolution variant and launch shape,
// compensated-merge interval, CTAs per cell of the fused transforms).
struct ConvCfg {
    int impl = 4, warps = 4, stages = 0, merge = 16, split = 4;
    int csplit = 1;   // variant 4: run the batch's split item list (the costliest pencils in two halves)
    double ms = 0.0;  // measured time of one collide of the batch when tuned
};

struct Batch;  // device-side description of one instance layout (defined in api.cu)
struct Mlp;    // learned surrogate (mlp.h)
struct IndicatorTable;

enum ProfKernel { PK_CONV32 = 0, PK_CONV64 = 1, PK_COLLIDE = 2, PK_FORWARD = 3, PK_INVERSE = 4, PK_TRANSPORT = 5 };
struct ProfEntry {
    int kernel;
    cudaEvent_t a, b;
};
struct WallTable {
    double *d = nullptr;       // device M_w per velocity
    std::vector<double> host;  // same values on the host
};
struct GraphRec {
    cudaGraphExec_t exec = nullptr;
    uint64_t last_use = 0;        // context tick of the latest replay (least recently used is evicted first)
    std::vector<ProfEntry> prof;  // events baked into the graph
    int64_t launches = 0;         // kernels per replay
    std::vector<bte_instance> inst;  // the instance list the graph was captured for (the key holds a hash)
    std::vector<double> trdesc;      // the slab it was captured for (walls, temperatures, widths; hashed in the key)
};

}  // namespace bte

struct bte_ctx {
    int device = 0;
    int num_sms = 0;
    std::string err;
    std::vector<bte::Table *> tables;
    int *d_status = nullptr;
    unsigned *d_counter = nullptr;
    // grow-only scratch
    static constexpr int kScratch = 16;
    void *scratch[kScratch] = {nullptr};
    size_t scratch_bytes[kScratch] = {0};
    std::map<std::string, bte::Batch *> batches;  // per instance layout, at most batch_cache_max
    int batch_cache_max = 64;
    uint64_t batch_tick = 0;
    std::map<bte::GraphKey, bte::GraphRec> graphs;  // at most graph_cache_max
    int graph_cache_max = 32;
    uint64_t graph_tick = 0;
    // Per stream the context has enqueued work on: an event recorded after that
    // work. Waiting on these (instead of the whole device) lets the context free
    // or rebuild what its own kernels may still read.
    std::map<cudaStream_t, cudaEvent_t> fence;
    // profiling / launch accounting
    bool prof = false;
    int prof_mask = 63;        // bit k: record events around ProfKernel k
    bool capturing = false;
    std::vector<bte::ProfEntry> pending;       // direct launches and replays not yet read
    std::vector<bte::ProfEntry> cap_prof;      // entries of the graph being captured
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_free;
    int64_t launches = 0, cap_launches = 0;
    double *d_wall = nullptr;  // unused scratch word pair
    std::map<std::tuple<int, double, double>, bte::WallTable> walls;  // (N, dv, T_w) -> M_w
    // transport coefficients of slabs with cells of unequal width, per width list:
    // device array [alpha (nx + 2) | gamma (nx + 2) | 1/dx (nx)]
    std::map<std::vector<double>, double *> grids;
    int conv_warps = 4;        // warps per CTA of the convolution kernel
    int conv_stages = 0;       // pipeline depth (blocks in flight per warp); 0 = automatic
    int conv_merge = 16;       // blocks per compensated (TwoSum) merge
    int conv_impl = 4;         // 0 warp items, 1 CTA-cooperative, 2 cooperative + packed f32x2,
                               // 3 as 2 at 2 CTAs/SM, 4 as 2 with the compensated sums in shared memory
    int dft_split = 4;         // CTAs per cell of the fused transforms (N <= 16)
    int conv_split = 1;        // variant 4: split the costliest pencil items in two
    int dft_fuse_stages = 1;   // FP32 Heun step: stage 1's inverse transform also forms stage 2's forward
    int debug_conv_stall = 0;  // testing only: make the convolution's waits run out
    std::string gpu_name;      // device name (key of saved tuning caches)
    std::map<std::string, bte::ConvCfg> tuned;  // autotuned configuration per batch shape
    bte::Mlp *mlp = nullptr;   // learned surrogate (bte_mlp_init)
    bte::IndicatorTable *ind = nullptr;  // sampled modes of the fallback indicator
    int learned_tol_ppm = 10000;         // fallback when the indicator exceeds 1e-6 * this
    int learned_samples = 64;
    // learned-mode statistics, accumulated on the device by every call and
    // step: cells seen, cells recomputed, the largest indicator (FP32 bits)
    unsigned long long *d_lstats = nullptr;
};

namespace bte {

// tables.cpp
int build_table(Table &t, std::string &err);
int build_table_fp32(Table &t, std::string &err);  // the stored FP32 weights (built by build_table for N <= 32)
int build_table_fp64(Table &t, std::string &err);
void free_table(Table &t);

}  // namespace bte
