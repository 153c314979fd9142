// bte_collide_noalloc: the FP32 collision operator for callers that must not
// allocate device memory. See include/bte.h for the contract.
//
// Everything a call needs beyond the caller's f and Q and the context's
// set-up-time state (weight tables, the one-group work-item template, kernel
// configurations) lives in one file-scope device array of fixed size: the
// work-queue counter, the per-cell offsets, the convolution work list and the
// two complex work arrays (fhat and Qhat in the group layout). A small kernel
// writes the offsets, the counter and the work list (the template repeated
// for every 32-cell group) into that array, so the call copies nothing from
// the host and never waits for the stream; it then launches the same kernels
// as bte_collide (fused forward transform, convolution, fused inverse
// transform with the projection), pointed at the array.
#include <cmath>
#include <cstdio>
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

std::mutex g_mutex;                             // guards g_scratch_addr
void *g_scratch_addr[kMaxDevices] = {nullptr};  // device address of the array, per device

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Work list, per-cell offsets and queue counter of one call: item i is the
// template's item i / ngroups for group i % ngroups (all groups of the
// costliest pencil first: a longest-first order for the atomic queue).
__global__ void noalloc_setup_kernel(const bte::ConvItem *__restrict__ tmpl, int ntmpl, int ngroups, int64_t M,
                                     int64_t ncells, int64_t nslots, bte::ConvItem *__restrict__ items,
                                     int64_t *__restrict__ off, unsigned *__restrict__ counter) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < (int64_t)ntmpl * ngroups) {
        bte::ConvItem it = tmpl[i / ngroups];
        it.fofs = (uint64_t)((i % ngroups) * M * bte::kLanes);
        items[i] = it;
    }
    if (i < nslots) off[i] = i < ncells ? i * M : -1;
    if (i == 0) *counter = 0u;
}

// Sets the caller's device back when the call returns.
struct DeviceRestore {
    int prev = -1;
    DeviceRestore() {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
    }
    ~DeviceRestore() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Error message into the context (storing it may allocate, on this error path only).
bte_status set_err(bte_ctx *c, bte_status s, const char *msg) {
    c->err = msg;
    return s;
}

}  // namespace

extern "C" bte_status bte_collide_noalloc(bte_ctx *c, const double *f, double *Q, int64_t ncells, void *stream) {
    using namespace bte;
    if (!c) return BTE_EINVAL;
    if (!f || !Q || f == Q) return set_err(c, BTE_EINVAL, "bte_collide_noalloc: bad f or Q");
    if (c->tables.empty())
        return set_err(c, BTE_ESTATE, "bte_collide_noalloc: no weight tables");
    const Table *t = c->tables[0];
    if (t->N > 16 || !fused_dft_supported(t->N))
        return set_err(c, BTE_EINVAL, "bte_collide_noalloc: table 0 must have N = 8, 12 or 16");
    if (ncells <= 0) return set_err(c, BTE_EINVAL, "bte_collide_noalloc: ncells must be > 0");
    if (c->device < 0 || c->device >= kMaxDevices)
        return set_err(c, BTE_EINVAL, "bte_collide_noalloc: device index too large");
    const int N = t->N;
    const int64_t M = (int64_t)N * N * N;
    const int64_t nslots = (ncells + kLanes - 1) / kLanes * kLanes;
    const int64_t ngroups = nslots / kLanes;
    const int64_t nitems = ngroups * t->n_tmpl;
    // layout of the array: counter | offsets | work list | fhat | qhat
    const size_t o_cnt = 0;
    const size_t o_off = 256;
    const size_t o_items = align256(o_off + sizeof(int64_t) * (size_t)nslots);
    const size_t o_f = align256(o_items + sizeof(ConvItem) * (size_t)nitems);
    const size_t o_q = align256(o_f + sizeof(float2) * (size_t)(nslots * M));
    const size_t need = o_q + sizeof(float2) * (size_t)(nslots * M);
    if (need > kNoAllocBytes || nitems > (int64_t)1 << 30) {
        char msg[256];
        std::snprintf(msg, sizeof msg,
                      "bte_collide_noalloc: %lld cells of N=%d need %llu bytes of static scratch; the limit is "
                      "%llu bytes (BTE_NOALLOC_SCRATCH_BYTES)",
                      (long long)ncells, N, (unsigned long long)need, (unsigned long long)kNoAllocBytes);
        return set_err(c, BTE_EINVAL, msg);
    }

    DeviceRestore restore;
    if (cudaSetDevice(c->device) != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, BTE_ECUDA, "bte_collide_noalloc: cudaSetDevice failed");
    }
    void *addr = nullptr;
    {
        // once per device, with that device current: the array's device address
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch_addr[c->device]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return set_err(c, BTE_ECUDA, "bte_collide_noalloc: cudaGetSymbolAddress failed");
            }
            g_scratch_addr[c->device] = p;
        }
        addr = g_scratch_addr[c->device];
    }
    unsigned char *base = (unsigned char *)addr;
    unsigned *d_counter = (unsigned *)(base + o_cnt);
    int64_t *d_off = (int64_t *)(base + o_off);
    ConvItem *d_items = (ConvItem *)(base + o_items);
    float2 *d_F = (float2 *)(base + o_f);
    float2 *d_Q = (float2 *)(base + o_q);

    // configuration: the autotuned one for this batch shape (split items are
    // not used here), else the context's options; both were configured at
    // set-up (bte_init_weights, bte_set_option, bte_autotune), so this is a
    // cache lookup
    ConvCfg g;
    g.impl = c->conv_impl;
    g.warps = c->conv_warps;
    g.stages = c->conv_stages;
    g.merge = c->conv_merge;
    g.split = c->dft_split;
    const unsigned mask = t->kinds_mask();
    {
        char key[48];
        std::snprintf(key, sizeof key, "k%u:s%lld", mask, (long long)nslots);
        auto it = c->tuned.find(key);  // a key this short stays in the string's inline buffer
        if (it != c->tuned.end()) g = it->second;
    }
    fused_dft_prepare(N);
    ConvLaunch L;
    cudaError_t e = conv32_configure(mask, c->num_sms, g.warps, g.stages, g.impl, &L);
    if (e != cudaSuccess) {
        cudaGetLastError();
        char msg[256];
        std::snprintf(msg, sizeof msg, "bte_collide_noalloc: configuration: %s", cudaGetErrorString(e));
        return set_err(c, BTE_ECUDA, msg);
    }
    if (g.impl == 5 && !t->d_I32)
        return set_err(c, BTE_EINVAL, "bte_collide_noalloc: conv_impl 5 needs an elastic table 0 (beta = 1)");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nth = nitems > nslots ? nitems : nslots;
    noalloc_setup_kernel<<<(unsigned)((nth + 255) / 256), 256, 0, st>>>(t->d_tmpl, t->n_tmpl, (int)ngroups, M, ncells,
                                                                        nslots, d_items, d_off, d_counter);
    DftSeg ds{N, 0, (int)nslots, 0};
    const double sf = std::pow(2.0 * kPi, -1.5) * t->dv * t->dv * t->dv;
    const double si = std::pow(2.0 * kPi, -1.5) * t->dz * t->dz * t->dz;
    launch_dft_forward_fused(f, d_off, ds, t->d_root32, sf, d_F, c->d_status, st, g.split);
    ConvParams p{};
    p.items = d_items;
    p.nitems = (int)nitems;
    p.counter = d_counter;
    p.F = d_F;
    p.Qh = d_Q;
    p.W[0] = t->d_w32;
    p.D[0] = t->d_desc;
    p.I32[0] = t->d_I32;
    p.J32[0] = t->d_J32;
    p.E[0] = t->d_etab;
    p.nq[0] = t->nq;
    p.estride[0] = t->estride;
    p.status = c->d_status;
    p.merge = g.merge;
    e = conv32_launch(L, p, st);
    if (e == cudaSuccess) {
        ProjArgs pa;
        pa.N = N;
        pa.dv = t->dv;
        std::memcpy(pa.ainv, t->ainv, sizeof(pa.ainv));
        launch_dft_inverse_fused(d_Q, d_off, ds, t->d_root32, si, Q, pa, 1, nullptr, nullptr, nullptr, 0.0, st,
                                 g.split);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        char msg[256];
        std::snprintf(msg, sizeof msg, "bte_collide_noalloc: launch: %s", cudaGetErrorString(e));
        return set_err(c, BTE_ECUDA, msg);
    }
    return BTE_OK;
}
