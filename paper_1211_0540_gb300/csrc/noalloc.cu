// bte_collide_noalloc: the FP32 collision operator for callers that must not
// allocate device memory. See include/bte.h for the contract.
//
// Everything a call needs beyond the caller's f and Q and the context's weight
// tables (built earlier, at set-up) lives in one file-scope device array of
// fixed size: the work-queue counter, the per-cell offsets, the convolution
// work list and the two complex work arrays (fhat and Qhat in the group
// layout). The call launches the same kernels as bte_collide (fused forward
// transform, convolution, fused inverse transform with the projection); it
// only points them at that array instead of the context's scratch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "kernels.h"

namespace {

constexpr size_t kNoAllocBytes = (size_t)BTE_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;
constexpr double kPi = 3.14159265358979323846;

// The device array. In host code `g_noalloc_scratch` names a host-side stand-in,
// not device memory: the kernels get the address from cudaGetSymbolAddress.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_mutex;                         // guards the tables below
void *g_scratch_addr[kMaxDevices] = {nullptr};  // device address of the array, per device
// Host staging for the offsets and the work list (static: no host allocation either).
constexpr int kMaxSlots = 1 << 16;
constexpr int kMaxItems = 1 << 16;
int64_t g_slot_off[kMaxSlots];
bte::ConvItem g_items[kMaxItems];
bte::ConvItem g_sorted[kMaxItems];
uint64_t g_cost[kMaxItems];
int g_order[kMaxItems];

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bte_status set_err(bte_ctx *c, bte_status s, const std::string &m) {
    c->err = m;
    return s;
}

}  // namespace

extern "C" bte_status bte_collide_noalloc(bte_ctx *c, const double *f, double *Q, int64_t ncells, void *stream) {
    using namespace bte;
    if (!c) return BTE_EINVAL;
    if (!f || !Q || f == Q) return set_err(c, BTE_EINVAL, "bte_collide_noalloc: bad f or Q");
    if (c->tables.empty()) return set_err(c, BTE_ESTATE, "bte_collide_noalloc: no weight tables");
    const Table *t = c->tables[0];
    if (t->N > 16 || !fused_dft_supported(t->N))
        return set_err(c, BTE_EINVAL, "bte_collide_noalloc: table 0 must have N = 8, 12 or 16");
    if (ncells <= 0) return set_err(c, BTE_EINVAL, "bte_collide_noalloc: ncells must be > 0");
    const int N = t->N;
    const int64_t M = (int64_t)N * N * N;
    const int64_t nslots = (ncells + kLanes - 1) / kLanes * kLanes;
    const int64_t ngroups = nslots / kLanes;
    const int64_t nitems = ngroups * t->ntiles * N * N;
    // layout of the array: counter | offsets | work list | fhat | qhat
    const size_t o_cnt = 0;
    const size_t o_off = 256;
    const size_t o_items = align256(o_off + sizeof(int64_t) * (size_t)nslots);
    const size_t o_f = align256(o_items + sizeof(ConvItem) * (size_t)nitems);
    const size_t o_q = align256(o_f + sizeof(float2) * (size_t)(nslots * M));
    const size_t need = o_q + sizeof(float2) * (size_t)(nslots * M);
    if (need > kNoAllocBytes || nslots > kMaxSlots || nitems > kMaxItems) {
        return set_err(c, BTE_EINVAL,
                       "bte_collide_noalloc: " + std::to_string(ncells) + " cells of N=" + std::to_string(N) +
                           " need " + std::to_string(need) + " bytes of static scratch; the limit is " +
                           std::to_string(kNoAllocBytes) + " bytes");
    }
    if (cudaSetDevice(c->device) != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, BTE_ECUDA, "bte_collide_noalloc: cudaSetDevice failed");
    }
    if (c->device < 0 || c->device >= kMaxDevices) return set_err(c, BTE_EINVAL, "device index too large");
    std::lock_guard<std::mutex> lock(g_mutex);
    // once per device, with that device current: the array's device address
    if (!g_scratch_addr[c->device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return set_err(c, BTE_ECUDA, std::string("bte_collide_noalloc: cudaGetSymbolAddress: ") +
                                             cudaGetErrorString(e));
        }
        g_scratch_addr[c->device] = p;
    }
    unsigned char *base = (unsigned char *)g_scratch_addr[c->device];
    unsigned *d_counter = (unsigned *)(base + o_cnt);
    int64_t *d_off = (int64_t *)(base + o_off);
    ConvItem *d_items = (ConvItem *)(base + o_items);
    float2 *d_F = (float2 *)(base + o_f);
    float2 *d_Q = (float2 *)(base + o_q);

    // per-cell offsets (padding lanes: -1) and the work list, costliest first
    for (int64_t s = 0; s < nslots; ++s) g_slot_off[s] = s < ncells ? s * M : -1;
    int64_t n = 0;
    for (int64_t g = 0; g < ngroups; ++g)
        for (int tile = 0; tile < t->ntiles; ++tile)
            for (int kk = 0; kk < N * N; ++kk) {
                if (t->nblocks[kk] == 0) continue;
                ConvItem &ci = g_items[n];
                ci.fofs = (uint64_t)(g * M * kLanes);
                ci.wofs = t->wofs[(size_t)tile * N * N + kk];
                ci.desc_off = t->desc_off[kk];
                ci.nblocks = t->nblocks[kk];
                ci.k1 = (uint16_t)(kk / N);
                ci.k2 = (uint16_t)(kk % N);
                ci.kind = (uint16_t)(t->kind0 + tile);
                ci.table = 0;
                g_cost[n] = (uint64_t)ci.nblocks * t->cpad[tile];
                g_order[n] = (int)n;
                ++n;
            }
    std::sort(g_order, g_order + n, [](int a, int b) {
        return g_cost[a] != g_cost[b] ? g_cost[a] > g_cost[b] : a < b;
    });
    for (int64_t i = 0; i < n; ++i) g_sorted[i] = g_items[g_order[i]];

    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d_counter, 0, sizeof(unsigned), st);  // the queue starts at 0
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, g_slot_off, sizeof(int64_t) * nslots, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_items, g_sorted, sizeof(ConvItem) * n, cudaMemcpyHostToDevice, st);
    // the staging arrays are reused by the next call: finish the copies first
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, BTE_ECUDA, std::string("bte_collide_noalloc: upload: ") + cudaGetErrorString(e));
    }

    fused_dft_prepare(N);
    ConvLaunch L;
    e = conv32_configure(1u << t->kind0 | (t->ntiles > 1 ? 1u << (t->kind0 + 1) : 0u), c->num_sms, c->conv_warps,
                         c->conv_stages, c->conv_impl, &L);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, BTE_ECUDA, std::string("bte_collide_noalloc: configuration: ") + cudaGetErrorString(e));
    }
    DftSeg ds{N, 0, (int)nslots, 0};
    const double sf = std::pow(2.0 * kPi, -1.5) * t->dv * t->dv * t->dv;
    const double si = std::pow(2.0 * kPi, -1.5) * t->dz * t->dz * t->dz;
    launch_dft_forward_fused(f, d_off, ds, t->d_root32, sf, d_F, c->d_status, st, c->dft_split);
    ConvParams p{};
    p.items = d_items;
    p.nitems = (int)n;
    p.counter = d_counter;
    p.F = d_F;
    p.Qh = d_Q;
    p.W[0] = t->d_w32;
    p.D[0] = t->d_desc;
    p.status = c->d_status;
    p.merge = c->conv_merge;
    e = conv32_launch(L, p, st);
    if (e == cudaSuccess) {
        ProjArgs pa;
        pa.N = N;
        pa.dv = t->dv;
        std::memcpy(pa.ainv, t->ainv, sizeof(pa.ainv));
        launch_dft_inverse_fused(d_Q, d_off, ds, t->d_root32, si, Q, pa, 1, nullptr, nullptr, nullptr, 0.0, st,
                                 c->dft_split);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, BTE_ECUDA, std::string("bte_collide_noalloc: launch: ") + cudaGetErrorString(e));
    }
    return BTE_OK;
}
