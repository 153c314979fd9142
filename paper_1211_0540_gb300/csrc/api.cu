// C ABI of libbte (include/bte.h): contexts, weight tables, batches and the
// orchestration of the collision operator, projection and time steps.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <queue>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "kernels.h"
#include "learned.h"
#include "mlp.h"

namespace bte {

constexpr double kPi = 3.14159265358979323846;
constexpr uint64_t kIndicatorSeed = 12345;  // SplitMix64 seed of the indicator's pencil sample

// A batch: the instance layout of one (inst, ninst) argument, mapped onto
// slots. Instances are grouped by weight table into segments; a segment's
// slots are padded to a multiple of 32 (one warp lane per cell).
struct Segment {
    int table;
    int s0, nslots, nvalid;
    int64_t eoff;  // complex-element offset of the segment in the scratch buffers
};
struct Batch {
    std::vector<Segment> segs;
    int nslots = 0;
    int64_t n_celem = 0;  // sum over slots of M
    int64_t extent = 0;   // max(offset + M) over instances
    int64_t *d_slot_off = nullptr;
    int64_t *d_slot_out = nullptr;
    ConvItem *d_items = nullptr;
    int nitems = 0;
    // the same work with the costliest items split into two block ranges
    // (convolution variant 4): items, split codes, partial sums, counters
    // ([0] the queue, [1 + sid] the halves of split sid that finished)
    ConvItem *d_items_split = nullptr;
    int nitems_split = 0, nsplit = 0;
    int *d_split = nullptr;
    float *d_part = nullptr;
    unsigned *d_counters = nullptr;
    uint64_t last_use = 0;  // context tick of the latest lookup (least recently used is evicted first)
    unsigned kinds_mask = 0;
    bool uniform = false;
    int uniform_table = 0;
};

bool GraphKey::operator<(const GraphKey &o) const {
    return std::tie(ninst, table, mode, transport, dt, eps, f, stream) <
           std::tie(o.ninst, o.table, o.mode, o.transport, o.dt, o.eps, o.f, o.stream);
}

}  // namespace bte

using namespace bte;

namespace {

enum ScratchId { SC_T1 = 0, SC_T2, SC_F, SC_QH, SC_FS, SC_Q1, SC_Q2, SC_MISC, SC_FB };

// NVTX range over a host-side stage (enqueue of its launches; inside stream
// capture it marks the capture, not the replays). A no-op without a profiler.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

bte_status fail(bte_ctx *c, bte_status s, const std::string &msg) {
    if (c) c->err = msg;
    return s;
}

bte_status cuda_fail(bte_ctx *c, cudaError_t e, const char *what) {
    cudaGetLastError();  // do not leave a non-sticky error behind for the caller's runtime checks
    return fail(c, BTE_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Events recorded inside captured graphs belong to the graphs; replays also
// list them in c->pending, so pending entries return to the free pool only
// when no graph owns their events (an event must be destroyed exactly once).
bool owned_by_graph(const bte_ctx *c, cudaEvent_t ev) {
    for (const auto &kv : c->graphs)
        for (const ProfEntry &pe : kv.second.prof)
            if (pe.a == ev) return true;
    return false;
}

// Record the context's fence on `st` after the work a call enqueued there.
void fence_record(bte_ctx *c, cudaStream_t st) {
    if (c->capturing) return;
    auto it = c->fence.find(st);
    if (it == c->fence.end()) {
        if (c->fence.size() >= 64) {  // many streams: wait for all and start over
            for (auto &kv : c->fence) {
                cudaEventSynchronize(kv.second);
                cudaEventDestroy(kv.second);
            }
            c->fence.clear();
        }
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            cudaStreamSynchronize(st);  // no event: this call's work is finished instead
            cudaGetLastError();
            return;
        }
        it = c->fence.emplace(st, ev).first;
    }
    cudaEventRecord(it->second, st);
}

// Wait until every kernel this context has enqueued has finished (other
// users of the device are not waited for).
cudaError_t quiesce(bte_ctx *c) {
    cudaError_t r = cudaSuccess;
    for (auto &kv : c->fence) {
        cudaError_t e = cudaEventSynchronize(kv.second);
        if (e != cudaSuccess) r = e;
    }
    return r;
}

// Events of a graph that is being destroyed: those no pending profile entry
// names go back to the pool; pending ones return when they are read.
void release_graph_events(bte_ctx *c, const GraphRec &g) {
    for (const ProfEntry &pe : g.prof) {
        bool named = false;
        for (const ProfEntry &q : c->pending)
            if (q.a == pe.a) named = true;
        if (!named) c->ev_free.push_back({pe.a, pe.b});
    }
}

// Forget every captured step graph (they bake in scratch pointers, options and
// profiling events); the next bte_step captures again. Waits for the
// context's own work.
void drop_graphs(bte_ctx *c) {
    quiesce(c);
    for (const ProfEntry &pe : c->pending)
        if (!owned_by_graph(c, pe.a)) c->ev_free.push_back({pe.a, pe.b});
    c->pending.clear();
    for (auto &kv : c->graphs) {
        cudaGraphExecDestroy(kv.second.exec);
        for (auto &pe : kv.second.prof) c->ev_free.push_back({pe.a, pe.b});
    }
    c->graphs.clear();
}

bte_status ensure_scratch(bte_ctx *c, int id, size_t bytes) {
    if (c->scratch_bytes[id] >= bytes) return BTE_OK;
    if (c->scratch[id]) drop_graphs(c);  // graphs captured earlier hold the old buffer
    cudaFree(c->scratch[id]);
    c->scratch[id] = nullptr;
    c->scratch_bytes[id] = 0;
    cudaError_t e = cudaMalloc(&c->scratch[id], bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, BTE_ENOMEM, std::string("scratch allocation: ") + cudaGetErrorString(e));
    }
    c->scratch_bytes[id] = bytes;
    return BTE_OK;
}

void count_launches(bte_ctx *c, int n) {
    if (c->capturing) c->cap_launches += n;
    else c->launches += n;
}

// Reserve event pairs outside stream capture so that profiled captures never create events.
void prof_reserve(bte_ctx *c, size_t n) {
    if (!c->prof) return;
    while (c->ev_free.size() < n) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess) return;
        if (cudaEventCreate(&b) != cudaSuccess) {
            cudaEventDestroy(a);
            return;
        }
        c->ev_free.push_back({a, b});
    }
}

int prof_begin(bte_ctx *c, int kernel, cudaStream_t st, ProfEntry *pe) {
    if (!c->prof || !(c->prof_mask & (1 << kernel))) return 0;
    if (c->ev_free.empty()) {
        if (c->capturing) return 0;
        prof_reserve(c, 1);
        if (c->ev_free.empty()) return 0;
    }
    pe->kernel = kernel;
    pe->a = c->ev_free.back().first;
    pe->b = c->ev_free.back().second;
    c->ev_free.pop_back();
    // inside stream capture only an "external" record becomes an event-record node
    cudaEventRecordWithFlags(pe->a, st, c->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
    return 1;
}

void prof_end(bte_ctx *c, int active, const ProfEntry &pe, cudaStream_t st) {
    if (!active) return;
    cudaEventRecordWithFlags(pe.b, st, c->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
    if (c->capturing) c->cap_prof.push_back(pe);
    else c->pending.push_back(pe);
}

uint64_t fnv1a(const void *p, size_t n, uint64_t h = 1469598103934665603ull) {
    const unsigned char *b = (const unsigned char *)p;
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    return h;
}

int64_t cell_M(const Table *t) { return (int64_t)t->N * t->N * t->N; }

void free_batch(Batch *B) {
    cudaFree(B->d_slot_off);
    cudaFree(B->d_slot_out);
    cudaFree(B->d_items);
    cudaFree(B->d_items_split);
    cudaFree(B->d_split);
    cudaFree(B->d_part);
    cudaFree(B->d_counters);
    delete B;
}

// Makespan of the atomic queue as list scheduling: items in queue order, each
// taken by the first of W equal workers to become free (LPT when the costs
// are sorted in decreasing order).
double lpt_makespan(const std::vector<double> &cost, int W) {
    std::priority_queue<double, std::vector<double>, std::greater<double>> free_at;
    for (int w = 0; w < W; ++w) free_at.push(0.0);
    double end = 0.0;
    for (double x : cost) {
        const double t = free_at.top() + x;
        free_at.pop();
        free_at.push(t);
        end = std::max(end, t);
    }
    return end;
}

// Split plan of the convolution's queue for variant 4 (3 CTAs of 4 warps per
// SM): the costliest items are cut into two block ranges. Item cost in block
// times of one CTA: ceil(blocks / 4) plus one for the item's first copies and
// its reduction. Splits go level by level (all unsplit pieces of the current
// largest cost at once, at least 8 blocks a half) down to the smallest
// splittable cost; the level with the shortest simulated makespan is kept
// (single levels often leave it unchanged, so there is no early stop).
// out: the items in queue order; code[i] = -1 or 2 sid + half.
void plan_splits(const bte_ctx *c, const std::vector<ConvItem> &items, std::vector<ConvItem> &out,
                 std::vector<int> &code) {
    struct Piece {
        ConvItem it;
        int code;
    };
    const int W = 3 * c->num_sms;
    auto cost_of = [](const ConvItem &it) { return (double)((it.nblocks + 3) / 4) + 1.0; };
    auto order = [&](std::vector<Piece> &v) {
        std::stable_sort(v.begin(), v.end(),
                         [&](const Piece &a, const Piece &b) { return cost_of(a.it) > cost_of(b.it); });
    };
    auto makespan = [&](const std::vector<Piece> &v) {
        std::vector<double> cs(v.size());
        for (size_t i = 0; i < v.size(); ++i) cs[i] = cost_of(v[i].it);
        return lpt_makespan(cs, W);
    };
    std::vector<Piece> cur(items.size());
    for (size_t i = 0; i < items.size(); ++i) cur[i] = Piece{items[i], -1};
    out.clear();
    code.clear();
    if (items.empty() || items.size() > 65536) {  // large batches have no tail to cut
        return;
    }
    double best = makespan(cur);
    std::vector<Piece> best_state;  // empty: no split
    int nsplit = 0, best_nsplit = 0;
    for (int level = 0; level < 64; ++level) {
        // the largest cost among unsplit pieces that can be cut
        double top = -1.0;
        for (const Piece &p : cur)
            if (p.code < 0 && p.it.nblocks >= 16) top = std::max(top, cost_of(p.it));
        if (top < 0.0) break;
        std::vector<Piece> trial;
        trial.reserve(cur.size() * 2);
        int ns = nsplit;
        for (const Piece &p : cur) {
            if (p.code < 0 && p.it.nblocks >= 16 && cost_of(p.it) == top) {
                const Table *t = c->tables[p.it.table];
                const int tile = p.it.kind - t->kind0;
                const uint32_t b0 = p.it.nblocks / 2;
                Piece a = p, b = p;
                a.it.nblocks = b0;
                a.code = 2 * ns;
                b.it.desc_off = p.it.desc_off + b0;
                b.it.wofs = p.it.wofs + (uint64_t)b0 * t->cpad[tile];
                b.it.nblocks = p.it.nblocks - b0;
                b.code = 2 * ns + 1;
                ++ns;
                trial.push_back(a);
                trial.push_back(b);
            } else {
                trial.push_back(p);
            }
        }
        order(trial);
        const double m = makespan(trial);
        cur.swap(trial);
        nsplit = ns;
        if (m < best * 0.999) {
            best = m;
            best_state = cur;
            best_nsplit = nsplit;
        }
    }
    if (best_nsplit == 0) return;
    out.resize(best_state.size());
    code.resize(best_state.size());
    for (size_t i = 0; i < best_state.size(); ++i) {
        out[i] = best_state[i].it;
        code[i] = best_state[i].code;
    }
}

// Build (or fetch) the batch for an instance layout.
bte_status get_batch(bte_ctx *c, const bte_instance *inst, int64_t ninst, Batch **out) {
    if (c->tables.empty()) return fail(c, BTE_ESTATE, "no weight tables: call bte_init_weights first");
    if (ninst <= 0) return fail(c, BTE_EINVAL, "ninst must be > 0");
    if (ninst > (1 << 24)) return fail(c, BTE_EINVAL, "ninst too large");
    std::string key;
    if (!inst) {
        key = "u:" + std::to_string(ninst);
    } else {
        key = "i:" + std::to_string(ninst) + ":" +
              std::to_string(fnv1a(inst, sizeof(bte_instance) * (size_t)ninst));
    }
    auto it = c->batches.find(key);
    if (it != c->batches.end()) {
        it->second->last_use = ++c->batch_tick;
        *out = it->second;
        return BTE_OK;
    }
    // bounded cache: a new layout evicts the least recently used one (an
    // earlier batch of the same API call was looked up later, so it stays)
    while ((int)c->batches.size() >= c->batch_cache_max && !c->batches.empty()) {
        auto lru = c->batches.begin();
        for (auto b = c->batches.begin(); b != c->batches.end(); ++b)
            if (b->second->last_use < lru->second->last_use) lru = b;
        cudaError_t e = quiesce(c);  // this context's kernels in flight may still read it
        if (e != cudaSuccess) return cuda_fail(c, e, "batch eviction");
        drop_graphs(c);  // captured steps hold its device arrays
        free_batch(lru->second);
        c->batches.erase(lru);
    }
    // instance -> (table, offset)
    std::vector<int> tab(ninst);
    std::vector<int64_t> off(ninst);
    const int64_t M0 = cell_M(c->tables[0]);
    for (int64_t i = 0; i < ninst; ++i) {
        if (inst) {
            if (inst[i].table < 0 || inst[i].table >= (int)c->tables.size())
                return fail(c, BTE_EINVAL, "instance " + std::to_string(i) + ": unknown table id");
            if (inst[i].offset < 0) return fail(c, BTE_EINVAL, "instance " + std::to_string(i) + ": negative offset");
            tab[i] = inst[i].table;
            off[i] = inst[i].offset;
        } else {
            tab[i] = 0;
            off[i] = i * M0;
        }
    }
    // non-overlap of instance ranges
    {
        std::vector<int64_t> order(ninst);
        std::iota(order.begin(), order.end(), 0);
        std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return off[a] < off[b]; });
        for (int64_t k = 1; k < ninst; ++k) {
            int64_t a = order[k - 1], b = order[k];
            if (off[a] + cell_M(c->tables[tab[a]]) > off[b])
                return fail(c, BTE_EINVAL, "instances " + std::to_string(a) + " and " + std::to_string(b) + " overlap");
        }
    }
    Batch *B = new Batch();
    B->uniform = inst == nullptr;
    std::vector<int64_t> slot_off, slot_out;
    for (int t = 0; t < (int)c->tables.size(); ++t) {
        std::vector<int64_t> members;
        for (int64_t i = 0; i < ninst; ++i)
            if (tab[i] == t) members.push_back(i);
        if (members.empty()) continue;
        Segment s;
        s.table = t;
        s.s0 = B->nslots;
        s.nvalid = (int)members.size();
        s.nslots = (s.nvalid + kLanes - 1) / kLanes * kLanes;
        s.eoff = B->n_celem;
        const int64_t M = cell_M(c->tables[t]);
        for (int k = 0; k < s.nslots; ++k) {
            if (k < s.nvalid) {
                slot_off.push_back(off[members[k]]);
                slot_out.push_back(members[k]);
                B->extent = std::max(B->extent, off[members[k]] + M);
            } else {
                slot_off.push_back(-1);
                slot_out.push_back(-1);
            }
        }
        B->nslots += s.nslots;
        B->n_celem += (int64_t)s.nslots * M;
        B->segs.push_back(s);
    }
    // convolution work items, costliest first
    std::vector<ConvItem> items;
    std::vector<uint64_t> cost;
    for (const Segment &s : B->segs) {
        const Table *t = c->tables[s.table];
        const int N = t->N;
        const int64_t M = cell_M(t);
        for (int g = 0; g < s.nslots / kLanes; ++g)
            for (int tile = 0; tile < t->ntiles; ++tile)
                for (int kk = 0; kk < N * N; ++kk) {
                    ConvItem ci;
                    ci.fofs = (uint64_t)(s.eoff + (int64_t)g * M * kLanes);
                    ci.wofs = t->wofs[(size_t)tile * N * N + kk];
                    ci.desc_off = t->desc_off[kk];
                    ci.nblocks = t->nblocks[kk];
                    ci.k1 = (uint16_t)(kk / N);
                    ci.k2 = (uint16_t)(kk % N);
                    ci.kind = (uint16_t)(t->kind0 + tile);
                    ci.table = (uint16_t)s.table;
                    if (ci.nblocks == 0) continue;
                    items.push_back(ci);
                    cost.push_back((uint64_t)ci.nblocks * t->cpad[tile]);
                    B->kinds_mask |= 1u << ci.kind;
                }
    }
    std::vector<size_t> order(items.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
    std::vector<ConvItem> sorted(items.size());
    for (size_t i = 0; i < items.size(); ++i) sorted[i] = items[order[i]];
    B->nitems = (int)sorted.size();
    std::vector<ConvItem> split_items;
    std::vector<int> split_code;
    plan_splits(c, sorted, split_items, split_code);
    B->nitems_split = (int)split_items.size();
    B->nsplit = 0;
    for (int v : split_code) B->nsplit = std::max(B->nsplit, v / 2 + 1);
    cudaError_t e = cudaMalloc(&B->d_slot_off, sizeof(int64_t) * slot_off.size());
    if (e == cudaSuccess) e = cudaMalloc(&B->d_slot_out, sizeof(int64_t) * slot_out.size());
    if (e == cudaSuccess) e = cudaMalloc(&B->d_items, sizeof(ConvItem) * std::max<size_t>(sorted.size(), 1));
    if (e == cudaSuccess && B->nsplit > 0) {
        e = cudaMalloc(&B->d_items_split, sizeof(ConvItem) * split_items.size());
        if (e == cudaSuccess) e = cudaMalloc(&B->d_split, sizeof(int) * split_code.size());
        if (e == cudaSuccess) e = cudaMalloc(&B->d_part, sizeof(float) * kSplitFloats * 2 * (size_t)B->nsplit);
    }
    if (e == cudaSuccess) e = cudaMalloc(&B->d_counters, sizeof(unsigned) * (1 + (size_t)B->nsplit));
    if (e != cudaSuccess) {
        free_batch(B);
        return fail(c, BTE_ENOMEM, std::string("batch allocation: ") + cudaGetErrorString(e));
    }
    e = cudaMemcpy(B->d_slot_off, slot_off.data(), sizeof(int64_t) * slot_off.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(B->d_slot_out, slot_out.data(), sizeof(int64_t) * slot_out.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !sorted.empty())
        e = cudaMemcpy(B->d_items, sorted.data(), sizeof(ConvItem) * sorted.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && B->nsplit > 0) {
        e = cudaMemcpy(B->d_items_split, split_items.data(), sizeof(ConvItem) * split_items.size(),
                       cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(B->d_split, split_code.data(), sizeof(int) * split_code.size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        free_batch(B);
        return cuda_fail(c, e, "batch upload");
    }
    B->last_use = ++c->batch_tick;
    c->batches[key] = B;
    *out = B;
    return BTE_OK;
}

// Batch shape key of the tuning cache: the convolution kinds and the slots.
std::string tune_key(const Batch *B) {
    return "k" + std::to_string(B->kinds_mask) + ":s" + std::to_string(B->nslots);
}

// The FP32 configuration of a batch: the autotuned one for its shape, else the options.
ConvCfg cfg_of(const bte_ctx *c, const Batch *B) {
    auto it = c->tuned.find(tune_key(B));
    if (it != c->tuned.end()) return it->second;
    ConvCfg g;
    g.impl = c->conv_impl;
    g.warps = c->conv_warps;
    g.stages = c->conv_stages;
    g.merge = c->conv_merge;
    g.csplit = c->conv_split;
    g.split = c->dft_split;
    return g;
}

ProjArgs proj_args(const Table *t) {
    ProjArgs pa;
    pa.N = t->N;
    pa.dv = t->dv;
    std::memcpy(pa.ainv, t->ainv, sizeof(pa.ainv));
    return pa;
}

// Allocate everything a collide/step on this batch needs (never inside capture).
bte_status prepare(bte_ctx *c, Batch *B, int mode, bool step, bool transport) {
    bte_status s;
    const size_t ce = (size_t)B->n_celem;
    const size_t csz = mode == BTE_FP64_PLAIN ? sizeof(double2) : sizeof(float2);
    for (int id : {SC_T1, SC_T2, SC_F, SC_QH})
        if ((s = ensure_scratch(c, id, ce * csz)) != BTE_OK) return s;
    if (step || transport) {
        for (int id : {SC_FS, SC_Q1, SC_Q2})
            if ((s = ensure_scratch(c, id, sizeof(double) * (size_t)B->extent)) != BTE_OK) return s;
    }
    for (const Segment &sg : B->segs)
        if (fused_dft_supported(c->tables[sg.table]->N)) fused_dft_prepare(c->tables[sg.table]->N);
    if (mode == BTE_FP64_PLAIN) {
        for (const Segment &sg : B->segs) {
            if (c->tables[sg.table]->N > 32)
                return fail(c, BTE_EINVAL, "the plain FP64 operator is limited to N <= 32 (its table holds 8 V(N) "
                                           "bytes: 41 GB at N = 48)");
            int r = build_table_fp64(*c->tables[sg.table], c->err);
            if (r != BTE_OK) return (bte_status)r;
        }
    } else if (mode == BTE_FP32) {
        ConvLaunch L;
        const ConvCfg g = cfg_of(c, B);
        for (const Segment &sg : B->segs) {
            Table *t = c->tables[sg.table];
            if (g.impl == 5 && !t->d_I32)
                return fail(c, BTE_EINVAL, "conv_impl 5 (weights on the fly) needs elastic tables (beta = 1)");
            if (g.impl != 5) {  // variants that stream the stored weights (built lazily at N = 48)
                const int r = build_table_fp32(*t, c->err);
                if (r != BTE_OK) return (bte_status)r;
            }
        }
        cudaError_t e = conv32_configure(B->kinds_mask, c->num_sms, g.warps, g.stages, g.impl, &L);
        if (e != cudaSuccess) return cuda_fail(c, e, "convolution kernel configuration");
    }
    return BTE_OK;
}

// What happens after the inverse transform of a collide.
enum Post { POST_RAW = 0, POST_PROJECT = 1, POST_STAGE1 = 2, POST_STAGE2 = 3 };

// Enqueue the operator for the batch: f -> Q, then `post`:
// RAW: Qt;  PROJECT: P Qt;  STAGE1: Q = P Qt and y = x + a Q;  STAGE2: Q = P Qt and
// y += a (qp + Q). Scratch must be ready (prepare). fuse (FP32, Heun stages):
// FUSE_NEXT_FWD with STAGE1: y is not written; the inverse transform forms the
// next stage's fhat of x + a Q in SC_F instead; SKIP_FWD: fhat is already in SC_F.
enum Fuse { FUSE_NONE = 0, FUSE_NEXT_FWD = 1, FUSE_SKIP_FWD = 2 };
bte_status enqueue_collide(bte_ctx *c, Batch *B, const double *f, double *Q, int mode, int post,
                           const double *x, double *y, const double *qp, double a, cudaStream_t st,
                           int fuse = FUSE_NONE) {
    NvtxRange range_collide("bte_collide");
    const bool fp64 = mode == BTE_FP64_PLAIN;
    const ConvCfg cfg = cfg_of(c, B);
    ProfEntry pe_all{}, pe_conv{}, pe_fwd{}, pe_inv{};
    const int on_all = prof_begin(c, PK_COLLIDE, st, &pe_all);
    if (!(fuse & FUSE_SKIP_FWD)) {
        NvtxRange range_fwd("bte_forward");
        const int on_fwd = prof_begin(c, PK_FORWARD, st, &pe_fwd);
        for (const Segment &sg : B->segs) {
            const Table *t = c->tables[sg.table];
            DftSeg ds{t->N, sg.s0, sg.nslots, sg.eoff};
            const double sf = std::pow(2.0 * kPi, -1.5) * t->dv * t->dv * t->dv;
            if (fp64) {
                launch_dft_forward<double2>(f, B->d_slot_off, ds, t->d_root64, sf, (double2 *)c->scratch[SC_T1],
                                            (double2 *)c->scratch[SC_T2], (double2 *)c->scratch[SC_F], c->d_status, st);
                count_launches(c, 3);
            } else if (fused_dft_supported(t->N)) {
                launch_dft_forward_fused(f, B->d_slot_off, ds, t->d_root32, sf, (float2 *)c->scratch[SC_F], c->d_status,
                                         st, cfg.split);
                count_launches(c, 1);
            } else {
                launch_dft_forward<float2>(f, B->d_slot_off, ds, t->d_root32, sf, (float2 *)c->scratch[SC_T1],
                                           (float2 *)c->scratch[SC_T2], (float2 *)c->scratch[SC_F], c->d_status, st);
                count_launches(c, 3);
            }
            cudaError_t e0 = cudaGetLastError();
            if (e0 != cudaSuccess) return cuda_fail(c, e0, "forward transform launch");
        }
        prof_end(c, on_fwd, pe_fwd, st);
    }
    NvtxRange range_conv(fp64 ? "bte_conv64" : "bte_conv32");
    if (fp64) {
        const int on = prof_begin(c, PK_CONV64, st, &pe_conv);
        for (const Segment &sg : B->segs) {
            const Table *t = c->tables[sg.table];
            if (2 * sg.nvalid <= sg.nslots)  // groups less than half full: lanes over the box instead of cells
                launch_conv64_cells((const double2 *)c->scratch[SC_F], (double2 *)c->scratch[SC_QH], t->d_w64,
                                    t->d_w64_off, B->d_slot_off, sg.s0, sg.nslots, t->N, sg.eoff, st);
            else
                launch_conv64((const double2 *)c->scratch[SC_F], (double2 *)c->scratch[SC_QH], t->d_w64,
                              t->d_w64_off, t->N, sg.eoff, sg.nslots / kLanes, st);
            count_launches(c, 1);
        }
        prof_end(c, on, pe_conv, st);
    } else {
        ConvLaunch L;
        cudaError_t e = conv32_configure(B->kinds_mask, c->num_sms, cfg.warps, cfg.stages, cfg.impl, &L);
        if (e != cudaSuccess) return cuda_fail(c, e, "convolution kernel configuration");
        ConvParams p{};
        const bool split = cfg.impl >= 4 && cfg.csplit && B->nsplit > 0;
        p.items = split ? B->d_items_split : B->d_items;
        p.nitems = split ? B->nitems_split : B->nitems;
        p.counter = B->d_counters;
        if (split) {
            p.split = B->d_split;
            p.part = B->d_part;
            p.split_cnt = B->d_counters + 1;
        }
        p.F = (const float2 *)c->scratch[SC_F];
        p.Qh = (float2 *)c->scratch[SC_QH];
        for (size_t i = 0; i < c->tables.size() && i < (size_t)kMaxTables; ++i) {
            const Table *t = c->tables[i];
            p.W[i] = t->d_w32;
            p.D[i] = t->d_desc;
            p.I32[i] = t->d_I32;
            p.J32[i] = t->d_J32;
            p.E[i] = t->d_etab;
            p.nq[i] = t->nq;
            p.estride[i] = t->estride;
        }
        p.status = c->d_status;
        p.merge = cfg.merge;
        p.stall = c->debug_conv_stall;
        e = cudaMemsetAsync(B->d_counters, 0, sizeof(unsigned) * (1 + (split ? (size_t)B->nsplit : 0)), st);
        if (e != cudaSuccess) return cuda_fail(c, e, "queue reset");
        const int on = prof_begin(c, PK_CONV32, st, &pe_conv);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(c, e, "before the convolution launch");
        e = conv32_launch(L, p, st);
        prof_end(c, on, pe_conv, st);
        count_launches(c, 1);
        if (e != cudaSuccess) {
            char msg[256];
            std::snprintf(msg, sizeof msg, "convolution launch (impl %d, grid %d, threads %d, smem %zu, items %d)",
                          L.impl, L.grid, L.threads, L.smem, p.nitems);
            return cuda_fail(c, e, msg);
        }
    }
    NvtxRange range_inv("bte_inverse");
    const int on_inv = prof_begin(c, PK_INVERSE, st, &pe_inv);
    for (const Segment &sg : B->segs) {
        const Table *t = c->tables[sg.table];
        DftSeg ds{t->N, sg.s0, sg.nslots, sg.eoff};
        const double si = std::pow(2.0 * kPi, -1.5) * t->dz * t->dz * t->dz;
        if (fuse & FUSE_NEXT_FWD) {  // post == POST_STAGE1 (checked by the caller)
            const double sf = std::pow(2.0 * kPi, -1.5) * t->dv * t->dv * t->dv;
            launch_dft_inverse_forward_fused((const float2 *)c->scratch[SC_QH], B->d_slot_off, ds, t->d_root32, si,
                                             Q, proj_args(t), x, a, sf, (float2 *)c->scratch[SC_F], c->d_status, st,
                                             cfg.split);
            count_launches(c, 1);
            continue;
        }
        if (!fp64 && fused_dft_supported(t->N)) {
            launch_dft_inverse_fused((const float2 *)c->scratch[SC_QH], B->d_slot_off, ds, t->d_root32, si, Q,
                                     proj_args(t), post, x, y, qp, a, st, cfg.split);
            count_launches(c, 1);
            continue;
        }
        if (fp64)
            launch_dft_inverse<double2>((const double2 *)c->scratch[SC_QH], B->d_slot_off, ds, t->d_root64, si,
                                        (double2 *)c->scratch[SC_T1], (double2 *)c->scratch[SC_T2], Q, st);
        else
            launch_dft_inverse<float2>((const float2 *)c->scratch[SC_QH], B->d_slot_off, ds, t->d_root32, si,
                                       (float2 *)c->scratch[SC_T1], (float2 *)c->scratch[SC_T2], Q, st);
        count_launches(c, 3);
        if (post != POST_RAW) {
            launch_project(Q, B->d_slot_off, sg.s0, sg.nslots, proj_args(t), post - 1, x, y, qp, a, st);
            count_launches(c, 1);
        }
    }
    prof_end(c, on_inv, pe_inv, st);
    prof_end(c, on_all, pe_all, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
    return BTE_OK;
}

// Heun step of the homogeneous problem on f (in place); the stage updates are
// fused into the projection that ends each collide.
bte_status enqueue_learned(bte_ctx *c, Batch *B, const double *f, double *Q, unsigned flags, const ConvCfg &cfg,
                           cudaStream_t st);

bte_status enqueue_rk2(bte_ctx *c, Batch *B, double *f, double dt, double eps, int mode, cudaStream_t st,
                       const ConvCfg *lcfg = nullptr) {
    double *fs = (double *)c->scratch[SC_FS];
    double *q1 = (double *)c->scratch[SC_Q1];
    double *q2 = (double *)c->scratch[SC_Q2];
    if (mode == BTE_LEARNED) {  // Q from the learned path, then the stage updates
        const int64_t n = (int64_t)B->segs[0].nvalid * cell_M(c->tables[0]);
        bte_status s = enqueue_learned(c, B, f, q1, 0u, *lcfg, st);
        if (s != BTE_OK) return s;
        launch_stage_update(q1, f, fs, nullptr, dt / eps, n, 1, st);
        if ((s = enqueue_learned(c, B, fs, q2, 0u, *lcfg, st)) != BTE_OK) return s;
        launch_stage_update(q2, nullptr, f, q1, 0.5 * dt / eps, n, 2, st);
        count_launches(c, 2);
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? BTE_OK : cuda_fail(c, e, "learned step: launch");
    }
    // FP32: the first stage's inverse transform also forms the second stage's
    // forward transform (f* = f + dt/eps Q1 is then never stored)
    bool fz = mode == BTE_FP32 && c->dft_fuse_stages;
    const int split = cfg_of(c, B).split;
    for (const Segment &sg : B->segs)
        fz = fz && inverse_forward_fused_supported(c->tables[sg.table]->N, split);
    bte_status s = enqueue_collide(c, B, f, q1, mode, POST_STAGE1, f, fs, nullptr, dt / eps, st,
                                   fz ? FUSE_NEXT_FWD : FUSE_NONE);
    if (s != BTE_OK) return s;
    return enqueue_collide(c, B, fs, q2, mode, POST_STAGE2, nullptr, f, q1, 0.5 * dt / eps, st,
                           fz ? FUSE_SKIP_FWD : FUSE_NONE);
}

// Wall Maxwellian M_w(v) = (2 pi T_w)^{-3/2} exp(-|v|^2 / (2 T_w)) on the grid of table t
// (FP64, host) and den = sum over the half entering the slab of |v.n| M_w
// (side 0: left wall, n = +e1; side 1: right wall, n = -e1). Cached per (grid, T_w).
bte_status wall_table(bte_ctx *c, const Table *t, double Tw, int side, const double **dptr, double *den) {
    const auto key = std::make_tuple(t->N, t->dv, Tw);
    auto it = c->walls.find(key);
    const int N = t->N, M = N * N * N, h = N / 2;
    if (it == c->walls.end()) {
        std::vector<double> mw(M);
        const double pref = std::pow(2.0 * kPi * Tw, -1.5);
        for (int j = 0; j < M; ++j) {
            const double v1 = t->dv * (j / (N * N) - h), v2 = t->dv * ((j / N) % N - h), v3 = t->dv * (j % N - h);
            mw[j] = pref * std::exp(-(v1 * v1 + v2 * v2 + v3 * v3) / (2.0 * Tw));
        }
        double *d = nullptr;
        cudaError_t e = cudaMalloc(&d, sizeof(double) * M);
        if (e != cudaSuccess) return cuda_fail(c, e, "wall table allocation");
        e = cudaMemcpy(d, mw.data(), sizeof(double) * M, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(d);
            return cuda_fail(c, e, "wall table upload");
        }
        WallTable w;
        w.d = d;
        w.host = std::move(mw);
        it = c->walls.emplace(key, std::move(w)).first;
    }
    double sum = 0.0;
    for (int j = 0; j < M; ++j) {
        const double v1 = t->dv * (j / (N * N) - h);
        const double vn = side == 0 ? v1 : -v1;
        if (vn > 0.0) sum += vn * it->second.host[j];
    }
    *dptr = it->second.d;
    *den = sum;
    return BTE_OK;
}

// Set-up-time configuration of what a uniform batch of table 0 runs with the
// context's options (shared-memory attributes, launch shapes, DFT roots), so
// that later calls -- bte_collide_noalloc in particular -- only look it up.
bte_status prime_configs(bte_ctx *c) {
    if (c->tables.empty()) return BTE_OK;
    for (const Table *t : c->tables)
        if (fused_dft_supported(t->N)) fused_dft_prepare(t->N);
    const Table *t = c->tables[0];
    const unsigned mask = t->kinds_mask();
    ConvLaunch L;
    cudaError_t e = conv32_configure(mask, c->num_sms, c->conv_warps, c->conv_stages, c->conv_impl, &L);
    return e == cudaSuccess ? BTE_OK : cuda_fail(c, e, "convolution kernel configuration");
}

// Transport coefficients of a slab with cells of widths dx[0..nx) (cached per
// width list): alpha_c = dx_c / (2 h_{c-1/2}), gamma_c = dx_c / (2 h_{c+1/2})
// for c = -1 .. nx (h = distance between cell centres; the ghost widths mirror
// the adjacent cells: dx_{-1} = dx_0, dx_{-2} = dx_1, dx_nx = dx_{nx-1},
// dx_{nx+1} = dx_{nx-2}) and 1/dx_c for c = 0 .. nx-1.
bte_status grid_coefficients(bte_ctx *c, const double *dx, int nx, TransportArgs *ta) {
    std::vector<double> key(dx, dx + nx);
    auto it = c->grids.find(key);
    if (it == c->grids.end()) {
        auto w = [&](int k) {  // width of cell k in [-2, nx + 1]
            if (k == -1) return dx[0];
            if (k == -2) return dx[1];
            if (k == nx) return dx[nx - 1];
            if (k == nx + 1) return dx[nx - 2];
            return dx[k];
        };
        std::vector<double> h((size_t)(2 * (nx + 2) + nx));
        for (int k = -1; k <= nx; ++k) {
            h[k + 1] = w(k) / (w(k - 1) + w(k));               // dx_k / (2 h_{k-1/2})
            h[nx + 2 + k + 1] = w(k) / (w(k) + w(k + 1));      // dx_k / (2 h_{k+1/2})
        }
        for (int k = 0; k < nx; ++k) h[2 * (nx + 2) + k] = 1.0 / dx[k];
        double *d = nullptr;
        cudaError_t e = cudaMalloc(&d, sizeof(double) * h.size());
        if (e != cudaSuccess) return cuda_fail(c, e, "transport grid allocation");
        e = cudaMemcpy(d, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(d);
            return cuda_fail(c, e, "transport grid upload");
        }
        it = c->grids.emplace(std::move(key), d).first;
    }
    ta->g_alpha = it->second;
    ta->g_gamma = it->second + (nx + 2);
    ta->g_rdx = it->second + 2 * (nx + 2);
    return BTE_OK;
}

bte_status check_mode(bte_ctx *c, int mode) {
    if (mode == BTE_FP64_PLAIN || mode == BTE_FP32) return BTE_OK;
    if (mode == BTE_LEARNED) {
        if (!c->mlp) return fail(c, BTE_ESTATE, "learned mode: no surrogate (bte_mlp_init)");
        return BTE_OK;
    }
    return fail(c, BTE_EINVAL, "unknown mode");
}

// The indicator's sampled pencils for table 0 (built on first use).
bte_status ensure_indicator(bte_ctx *c) {
    if (c->ind) return BTE_OK;
    const Table *t = c->tables[0];
    if (t->N > 16) return fail(c, BTE_EINVAL, "learned mode: N <= 16");
    IndicatorTable *it = new IndicatorTable();
    if (build_indicator_table(*t, c->learned_samples, kIndicatorSeed, *it) != 0) {
        free_indicator_table(*it);
        delete it;
        return fail(c, BTE_ENOMEM, "learned mode: indicator table");
    }
    c->ind = it;
    return BTE_OK;
}

// Indicator of the uniform batch B (cells of table 0): transform of f at every
// mode, of Q at the sampled pencils, the exact sums there and the per-slot
// ratio. *ind receives the device array (one float per slot, in SC_MISC).
bte_status enqueue_indicator(bte_ctx *c, Batch *B, const double *f, const double *Q, float **ind, cudaStream_t st) {
    const Segment &sg = B->segs[0];
    const Table *t = c->tables[0];
    bte_status s;
    if ((s = ensure_indicator(c)) != BTE_OK) return s;
    if ((s = ensure_scratch(c, SC_MISC, sizeof(float) * indicator_scratch_floats(*c->ind, t->N, B->nslots))) !=
        BTE_OK)
        return s;
    DftSeg ds{t->N, sg.s0, sg.nslots, sg.eoff};
    const double sf = std::pow(2.0 * kPi, -1.5) * t->dv * t->dv * t->dv;
    // sector order; one CTA per cell once the cells fill the SMs (the fastest for
    // this transform alone), else the batch's tuned split
    const int split = B->nslots >= c->num_sms ? 1 : cfg_of(c, B).split;
    launch_dft_forward_fused(f, B->d_slot_off, ds, t->d_root32, sf, (float2 *)c->scratch[SC_F], c->d_status, st,
                             split, true);
    launch_dft_forward_pencils(Q, B->d_slot_off, ds, sf, c->ind->d_kk, c->ind->S, (float2 *)c->scratch[SC_QH],
                               c->d_status, st);  // only the sampled pencils are compared
    float *e2 = (float *)c->scratch[SC_MISC];
    float *d2 = e2 + (size_t)B->nslots * c->ind->S;
    *ind = d2 + (size_t)B->nslots * c->ind->S;
    launch_indicator(*c->ind, *t, (const float2 *)c->scratch[SC_F], (const float2 *)c->scratch[SC_QH], sg.eoff,
                     sg.nslots, sg.nvalid, e2, d2, *ind, st);
    count_launches(c, 4);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BTE_OK : cuda_fail(c, e, "indicator launch");
}

constexpr int64_t kLearnedChunk = 8192;  // cells per surrogate pass

// Device work arrays of the learned mode's fallback for a uniform batch of
// nslots slots (in SC_FB): queue counter, work-list length, slot offsets, work list.
struct FallbackArrays {
    unsigned *counter;
    int *nitems;
    int64_t *off;
    ConvItem *items;
};
size_t fallback_bytes(int nslots, int ntmpl) {
    const size_t off = 256 + (((size_t)nslots * sizeof(int64_t) + 255) & ~(size_t)255);
    return off + sizeof(ConvItem) * (size_t)(nslots / kLanes) * (size_t)std::max(ntmpl, 1);
}
FallbackArrays fallback_arrays(bte_ctx *c, int nslots) {
    unsigned char *b = (unsigned char *)c->scratch[SC_FB];
    FallbackArrays a;
    a.counter = (unsigned *)b;
    a.nitems = (int *)(b + 64);
    a.off = (int64_t *)(b + 256);
    a.items = (ConvItem *)(b + 256 + (((size_t)nslots * sizeof(int64_t) + 255) & ~(size_t)255));
    return a;
}

// Everything the learned mode allocates or configures for the uniform batch B
// (never inside stream capture): surrogate activations, the indicator's
// pencils and scratch, the fallback's arrays and statistics, the FP32
// convolution (variant 4, or 5 when chosen; both read the work-list length
// from the device). *cfg receives the fallback's configuration.
bte_status prepare_learned(bte_ctx *c, Batch *B, ConvCfg *cfg) {
    Mlp *m = c->mlp;
    if (!B->uniform || B->segs.size() != 1 || B->uniform_table != 0 || m->table != 0)
        return fail(c, BTE_EINVAL, "learned mode: uniform cells of table 0 only (inst == NULL)");
    Table *t = c->tables[0];
    if (t->N > 16 || !fused_dft_supported(t->N)) return fail(c, BTE_EINVAL, "learned mode: N = 8, 12 or 16");
    bte_status s;
    if (!m->ensure_batch((int)std::min<int64_t>(kLearnedChunk, B->segs[0].nvalid)))
        return fail(c, BTE_ENOMEM, "learned mode: activations");
    if ((s = ensure_indicator(c)) != BTE_OK) return s;
    if ((s = ensure_scratch(c, SC_MISC, sizeof(float) * indicator_scratch_floats(*c->ind, t->N, B->nslots))) !=
        BTE_OK)
        return s;
    if ((s = ensure_scratch(c, SC_FB, fallback_bytes(B->nslots, t->n_tmpl))) != BTE_OK) return s;
    if (!c->d_lstats) {
        cudaError_t e = cudaMalloc(&c->d_lstats, 4 * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMemset(c->d_lstats, 0, 4 * sizeof(unsigned long long));
        if (e != cudaSuccess) return cuda_fail(c, e, "learned mode: statistics");
    }
    ConvCfg g = cfg_of(c, B);
    if (g.impl < 4 || (g.impl == 5 && !t->d_I32)) g.impl = 4;
    g.csplit = 0;
    if (g.impl == 4) {
        const int r = build_table_fp32(*t, c->err);
        if (r != BTE_OK) return (bte_status)r;
    }
    ConvLaunch L;
    cudaError_t e = conv32_configure(t->kinds_mask(), c->num_sms, g.warps, g.stages, g.impl, &L);
    if (e != cudaSuccess) return cuda_fail(c, e, "learned mode: convolution configuration");
    *cfg = g;
    return BTE_OK;
}

// Learned path on the uniform batch B (prepared by prepare_learned), all on
// the stream with no host round trip, so that it also runs inside a captured
// step: 1. surrogate in chunks of up to kLearnedChunk cells, 2. its output
// projected (fused), 3. the indicator at the sampled modes, 4. on the device,
// the list of cells whose indicator exceeds the tolerance and the FP32
// operator's batch for them, 5. that operator (forward transform, convolution
// over the listed groups only, inverse transform with the projection), which
// overwrites Q of those cells.
bte_status enqueue_learned(bte_ctx *c, Batch *B, const double *f, double *Q, unsigned flags, const ConvCfg &cfg,
                           cudaStream_t st) {
    NvtxRange range("bte_learned");
    Mlp *m = c->mlp;
    const Table *t = c->tables[0];
    const int64_t ncells = B->segs[0].nvalid;
    const int64_t M = cell_M(t);
    bte_status s;
    for (int64_t c0 = 0; c0 < ncells; c0 += kLearnedChunk) {
        const int n = (int)std::min<int64_t>(kLearnedChunk, ncells - c0);
        const int64_t o = c0 * M;
        if (m->run(f + o, nullptr, n, false, c->d_status, st, m->rowuni))
            return fail(c, BTE_ECUDA, "learned mode: surrogate");
        launch_post_project(m->Y, m->rho, n, t->N, m->s_out, proj_args(t), Q + o, st);
        count_launches(c, 5);
    }
    if (flags & BTE_FLAG_NO_FALLBACK) {
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? BTE_OK : cuda_fail(c, e, "learned mode: launch");
    }
    float *ind = nullptr;
    if ((s = enqueue_indicator(c, B, f, Q, &ind, st)) != BTE_OK) return s;
    const FallbackArrays fa = fallback_arrays(c, B->nslots);
    const double tol = 1e-6 * c->learned_tol_ppm;
    launch_fallback_setup(ind, (int)ncells, tol, M, t->d_tmpl, t->n_tmpl, B->nslots, fa.off, fa.items, fa.nitems,
                          fa.counter, c->d_lstats, st);
    DftSeg ds{t->N, 0, B->nslots, 0};
    const double sf = std::pow(2.0 * kPi, -1.5) * t->dv * t->dv * t->dv;
    const double si = std::pow(2.0 * kPi, -1.5) * t->dz * t->dz * t->dz;
    launch_dft_forward_fused(f, fa.off, ds, t->d_root32, sf, (float2 *)c->scratch[SC_F], c->d_status, st, cfg.split);
    ConvLaunch L;
    cudaError_t e = conv32_configure(t->kinds_mask(), c->num_sms, cfg.warps, cfg.stages, cfg.impl, &L);
    if (e != cudaSuccess) return cuda_fail(c, e, "learned mode: convolution configuration");
    ConvParams p{};
    p.items = fa.items;
    p.nitems = (B->nslots / kLanes) * t->n_tmpl;  // capacity (sizes the grid); the kernel reads the length
    p.nitems_dev = fa.nitems;
    p.counter = fa.counter;
    p.F = (const float2 *)c->scratch[SC_F];
    p.Qh = (float2 *)c->scratch[SC_QH];
    p.W[0] = t->d_w32;
    p.D[0] = t->d_desc;
    p.I32[0] = t->d_I32;
    p.J32[0] = t->d_J32;
    p.E[0] = t->d_etab;
    p.nq[0] = t->nq;
    p.estride[0] = t->estride;
    p.status = c->d_status;
    p.merge = cfg.merge;
    p.stall = c->debug_conv_stall;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "learned mode: launch");
    if ((e = conv32_launch(L, p, st)) != cudaSuccess) return cuda_fail(c, e, "learned mode: convolution launch");
    launch_dft_inverse_fused((const float2 *)c->scratch[SC_QH], fa.off, ds, t->d_root32, si, Q, proj_args(t),
                             POST_PROJECT, nullptr, nullptr, nullptr, 0.0, st, cfg.split);
    count_launches(c, 4);
    e = cudaGetLastError();
    return e == cudaSuccess ? BTE_OK : cuda_fail(c, e, "learned mode: launch");
}

}  // namespace

extern "C" {

const char *bte_version(void) { return "libbte 0.1 (sm_103a)"; }

bte_status bte_batch_count(const bte_ctx *c, int64_t *count) {
    if (!c || !count) return BTE_EINVAL;
    *count = (int64_t)c->batches.size();
    return BTE_OK;
}

bte_status bte_create(bte_ctx **ctx, int device) {
    if (!ctx) return BTE_EINVAL;
    *ctx = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) return BTE_ECUDA;
    if (device < 0 || device >= n) return BTE_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return BTE_ECUDA;
    bte_ctx *c = new bte_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    {
        cudaDeviceProp prop{};
        if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) c->gpu_name = prop.name;
    }
    if (cudaMalloc(&c->d_status, sizeof(int)) != cudaSuccess || cudaMalloc(&c->d_counter, 64) != cudaSuccess ||
        cudaMalloc(&c->d_wall, 2 * sizeof(double)) != cudaSuccess) {
        bte_destroy(c);
        return BTE_ENOMEM;
    }
    cudaMemset(c->d_status, 0, sizeof(int));
    cudaMemset(c->d_counter, 0, 64);
    *ctx = c;
    return BTE_OK;
}

void bte_destroy(bte_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    drop_graphs(c);  // graph-owned events move to the free pool once, pending entries too
    for (auto &kv : c->fence) cudaEventDestroy(kv.second);
    for (auto &ab : c->ev_free) {
        cudaEventDestroy(ab.first);
        cudaEventDestroy(ab.second);
    }
    for (auto &kv : c->batches) {
        free_batch(kv.second);
    }
    for (Table *t : c->tables) {
        free_table(*t);
        delete t;
    }
    delete c->mlp;
    if (c->ind) {
        free_indicator_table(*c->ind);
        delete c->ind;
    }
    for (int i = 0; i < bte_ctx::kScratch; ++i) cudaFree(c->scratch[i]);
    cudaFree(c->d_status);
    cudaFree(c->d_counter);
    cudaFree(c->d_wall);
    cudaFree(c->d_lstats);
    for (auto &kv : c->walls) cudaFree(kv.second.d);
    for (auto &kv : c->grids) cudaFree(kv.second);
    delete c;
}

const char *bte_last_error(const bte_ctx *c) { return c ? c->err.c_str() : "null context"; }

bte_status bte_init_weights(bte_ctx *c, const bte_grid *grids, int ngrids, int *table_ids) {
    if (!c || !grids || !table_ids || ngrids <= 0) return fail(c, BTE_EINVAL, "bte_init_weights: bad arguments");
    std::vector<bte_grid_ex> ex(ngrids);
    for (int i = 0; i < ngrids; ++i) ex[i] = bte_grid_ex{grids[i].N, grids[i].L, grids[i].lambda, 1.0};
    return bte_init_weights_ex(c, ex.data(), ngrids, table_ids);
}

bte_status bte_init_weights_ex(bte_ctx *c, const bte_grid_ex *grids, int ngrids, int *table_ids) {
    if (!c || !grids || !table_ids || ngrids <= 0) return fail(c, BTE_EINVAL, "bte_init_weights: bad arguments");
    if ((int)c->tables.size() + ngrids > kMaxTables)
        return fail(c, BTE_EINVAL, "too many weight tables (max " + std::to_string(kMaxTables) + ")");
    cudaSetDevice(c->device);
    for (int i = 0; i < ngrids; ++i) {
        Table *t = new Table();
        t->N = grids[i].N;
        t->L = grids[i].L;
        t->lam = grids[i].lambda;
        t->beta = grids[i].beta;
        int r = build_table(*t, c->err);
        if (r != BTE_OK) {
            delete t;
            return (bte_status)r;
        }
        table_ids[i] = (int)c->tables.size();
        c->tables.push_back(t);
        // batches built before this call stay valid (they name tables by id)
    }
    return prime_configs(c);
}

bte_status bte_collide_ex(bte_ctx *c, const double *f, double *Q, const bte_instance *inst, int64_t ninst,
                          int mode, unsigned flags, void *stream) {
    if (!c) return BTE_EINVAL;
    if (!f || !Q) return fail(c, BTE_EINVAL, "bte_collide: null f or Q");
    if (f == Q) return fail(c, BTE_EINVAL, "bte_collide: f and Q must not overlap");
    bte_status s = check_mode(c, mode);
    if (s != BTE_OK) return s;
    cudaSetDevice(c->device);
    Batch *B = nullptr;
    if ((s = get_batch(c, inst, ninst, &B)) != BTE_OK) return s;
    if ((s = prepare(c, B, mode == BTE_LEARNED ? BTE_FP32 : mode, false, false)) != BTE_OK) return s;
    if (mode == BTE_LEARNED) {
        ConvCfg lc;
        if ((s = prepare_learned(c, B, &lc)) == BTE_OK) s = enqueue_learned(c, B, f, Q, flags, lc, (cudaStream_t)stream);
    } else
        s = enqueue_collide(c, B, f, Q, mode, (flags & BTE_FLAG_RAW) ? POST_RAW : POST_PROJECT, nullptr, nullptr,
                            nullptr, 0.0, (cudaStream_t)stream);
    fence_record(c, (cudaStream_t)stream);
    return s;
}

bte_status bte_collide(bte_ctx *c, const double *f, double *Q, const bte_instance *inst, int64_t ninst, int mode,
                       void *stream) {
    return bte_collide_ex(c, f, Q, inst, ninst, mode, 0u, stream);
}

bte_status bte_project(bte_ctx *c, double *Q, const bte_instance *inst, int64_t ninst, void *stream) {
    if (!c) return BTE_EINVAL;
    if (!Q) return fail(c, BTE_EINVAL, "bte_project: null Q");
    cudaSetDevice(c->device);
    Batch *B = nullptr;
    bte_status s = get_batch(c, inst, ninst, &B);
    if (s != BTE_OK) return s;
    for (const Segment &sg : B->segs)
        launch_project(Q, B->d_slot_off, sg.s0, sg.nslots, proj_args(c->tables[sg.table]), 0, nullptr, nullptr,
                       nullptr, 0.0, (cudaStream_t)stream);
    fence_record(c, (cudaStream_t)stream);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BTE_OK : cuda_fail(c, e, "projection launch");
}

bte_status bte_moments(bte_ctx *c, const double *f, double *out, const bte_instance *inst, int64_t ninst,
                       void *stream) {
    if (!c) return BTE_EINVAL;
    if (!f || !out) return fail(c, BTE_EINVAL, "bte_moments: null pointer");
    cudaSetDevice(c->device);
    Batch *B = nullptr;
    bte_status s = get_batch(c, inst, ninst, &B);
    if (s != BTE_OK) return s;
    for (const Segment &sg : B->segs) {
        const Table *t = c->tables[sg.table];
        launch_moments(f, B->d_slot_off, sg.s0, sg.nslots, t->N, t->dv, B->d_slot_out, out, (cudaStream_t)stream);
    }
    fence_record(c, (cudaStream_t)stream);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BTE_OK : cuda_fail(c, e, "moments launch");
}

bte_status bte_step(bte_ctx *c, double *f, const bte_instance *inst, int64_t ninst, double dt, double eps,
                    const bte_transport *tr, int mode, void *stream) {
    if (!tr) return bte_step_ex(c, f, inst, ninst, dt, eps, nullptr, mode, stream);
    const bte_transport_ex ex{tr->nx, nullptr, tr->x0, tr->x1, tr->bc_left, tr->bc_right, tr->Tw_left, tr->Tw_right};
    return bte_step_ex(c, f, inst, ninst, dt, eps, &ex, mode, stream);
}

bte_status bte_step_ex(bte_ctx *c, double *f, const bte_instance *inst, int64_t ninst, double dt, double eps,
                       const bte_transport_ex *tr, int mode, void *stream) {
    if (!c) return BTE_EINVAL;
    if (!f) return fail(c, BTE_EINVAL, "bte_step: null f");
    if (!(dt > 0.0) || !(eps > 0.0) || !std::isfinite(dt) || !std::isfinite(eps))
        return fail(c, BTE_EINVAL, "bte_step: dt and eps must be finite and > 0");
    bte_status s = check_mode(c, mode);
    if (s != BTE_OK) return s;
    cudaSetDevice(c->device);
    TransportArgs ta{};
    if (tr) {
        if (inst) return fail(c, BTE_EINVAL, "bte_step: transport needs uniform cells (inst == NULL)");
        if (tr->nx != ninst || tr->nx < 2) return fail(c, BTE_EINVAL, "bte_step: tr->nx must equal ninst (>= 2)");
        if (!tr->dx && !(tr->x1 > tr->x0)) return fail(c, BTE_EINVAL, "bte_step: x1 must exceed x0");
        for (int bc : {tr->bc_left, tr->bc_right})
            if (bc != BTE_BC_DIFFUSE && bc != BTE_BC_SPECULAR && bc != BTE_BC_NOFLUX)
                return fail(c, BTE_EINVAL, "bte_step: unknown boundary type");
        if (tr->dx)
            for (int k = 0; k < tr->nx; ++k)
                if (!(tr->dx[k] > 0.0) || !std::isfinite(tr->dx[k]))
                    return fail(c, BTE_EINVAL, "bte_step: cell widths must be finite and > 0");
        if ((tr->bc_left == BTE_BC_DIFFUSE && !(tr->Tw_left > 0.0)) ||
            (tr->bc_right == BTE_BC_DIFFUSE && !(tr->Tw_right > 0.0)))
            return fail(c, BTE_EINVAL, "bte_step: wall temperatures must be > 0");
        const Table *t0 = c->tables.empty() ? nullptr : c->tables[0];
        if (!t0) return fail(c, BTE_ESTATE, "no weight tables: call bte_init_weights first");
        if (t0->N > kTransportMaxN) return fail(c, BTE_EINVAL, "bte_step: transport needs N <= 32");
        ta.N = t0->N;
        ta.nx = tr->nx;
        ta.dv = t0->dv;
        ta.dx = tr->dx ? 0.0 : (tr->x1 - tr->x0) / tr->nx;
        ta.bc_left = tr->bc_left;
        ta.bc_right = tr->bc_right;
        if (tr->dx && (s = grid_coefficients(c, tr->dx, tr->nx, &ta)) != BTE_OK) return s;
        if (ta.bc_left == BTE_BC_DIFFUSE &&
            (s = wall_table(c, t0, tr->Tw_left, 0, &ta.mw_left, &ta.den_left)) != BTE_OK)
            return s;
        if (ta.bc_right == BTE_BC_DIFFUSE &&
            (s = wall_table(c, t0, tr->Tw_right, 1, &ta.mw_right, &ta.den_right)) != BTE_OK)
            return s;
    }
    Batch *B = nullptr;
    if ((s = get_batch(c, inst, ninst, &B)) != BTE_OK) return s;
    if ((s = prepare(c, B, mode, true, tr != nullptr)) != BTE_OK) return s;
    ConvCfg lcfg;
    if (mode == BTE_LEARNED && (s = prepare_learned(c, B, &lcfg)) != BTE_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    auto body = [&]() -> bte_status {
        if (tr) {
            NvtxRange range_tr("bte_transport");
            ProfEntry pe{};
            const int on = prof_begin(c, PK_TRANSPORT, st, &pe);
            launch_transport_half(f, (double *)c->scratch[SC_FS], (double *)c->scratch[SC_Q1], ta, 0.5 * dt, st);
            prof_end(c, on, pe, st);
            count_launches(c, 2);
        }
        bte_status r = enqueue_rk2(c, B, f, dt, eps, mode, st, &lcfg);
        if (r != BTE_OK) return r;
        if (tr) {
            NvtxRange range_tr("bte_transport");
            ProfEntry pe{};
            const int on = prof_begin(c, PK_TRANSPORT, st, &pe);
            launch_transport_half(f, (double *)c->scratch[SC_FS], (double *)c->scratch[SC_Q1], ta, 0.5 * dt, st);
            prof_end(c, on, pe, st);
            count_launches(c, 2);
        }
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? BTE_OK : cuda_fail(c, e, "kernel launch");
    };
    if (st == nullptr) {  // the legacy stream cannot be captured
        bte_status r = body();
        fence_record(c, st);
        return r;
    }
    // the slab (walls, temperatures, cell widths) is baked into the graph too,
    // and so are the surrogate's buffers and scales in the learned mode
    std::vector<double> trdesc;
    if (tr) {
        trdesc = {(double)tr->nx, tr->x0, tr->x1, (double)tr->bc_left, (double)tr->bc_right, tr->Tw_left,
                  tr->Tw_right, tr->dx ? 1.0 : 0.0};
        if (tr->dx) trdesc.insert(trdesc.end(), tr->dx, tr->dx + tr->nx);
    }
    if (mode == BTE_LEARNED)
        trdesc.insert(trdesc.end(), {-1.0, (double)c->mlp->gen, (double)c->mlp->s_in, (double)c->mlp->s_out});
    const int trkey = trdesc.empty() ? 0 : (int)(fnv1a(trdesc.data(), sizeof(double) * trdesc.size()) & 0x7fffffff) | 1;
    GraphKey key{ninst, inst ? (int)(fnv1a(inst, sizeof(bte_instance) * ninst) & 0x7fffffff) : -1, mode,
                 trkey, dt, eps, f, stream};
    auto it = c->graphs.find(key);
    if (it != c->graphs.end() &&
        ((inst && (it->second.inst.size() != (size_t)ninst ||
                   std::memcmp(it->second.inst.data(), inst, sizeof(bte_instance) * ninst) != 0)) ||
         it->second.trdesc != trdesc)) {
        // another instance list or slab with the same hashes: capture anew. A
        // replay of the old graph may still be in flight, which the driver lets
        // finish before it frees the executable.
        cudaGraphExecDestroy(it->second.exec);
        release_graph_events(c, it->second);
        c->graphs.erase(it);
        it = c->graphs.end();
    }
    if (it == c->graphs.end()) {
        // bounded cache (its key holds f and dt, which a caller may vary):
        // the least recently replayed graph goes first
        while ((int)c->graphs.size() >= c->graph_cache_max && !c->graphs.empty()) {
            auto lru = c->graphs.begin();
            for (auto g = c->graphs.begin(); g != c->graphs.end(); ++g)
                if (g->second.last_use < lru->second.last_use) lru = g;
            cudaGraphExecDestroy(lru->second.exec);  // an in-flight replay completes first
            release_graph_events(c, lru->second);
            c->graphs.erase(lru);
        }
        prof_reserve(c, 16);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(c, e, "stream capture");
        c->capturing = true;
        c->cap_launches = 0;
        c->cap_prof.clear();
        bte_status r = body();
        c->capturing = false;
        e = cudaStreamEndCapture(st, &g);
        GraphRec rec;
        rec.prof = c->cap_prof;
        rec.launches = c->cap_launches;
        if (inst) rec.inst.assign(inst, inst + ninst);
        rec.trdesc = trdesc;
        c->cap_prof.clear();
        if (r != BTE_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            for (auto &pe : rec.prof) c->ev_free.push_back({pe.a, pe.b});
            return r != BTE_OK ? r : cuda_fail(c, e, "stream capture end");
        }
        e = cudaGraphInstantiate(&rec.exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            for (auto &pe : rec.prof) c->ev_free.push_back({pe.a, pe.b});
            return cuda_fail(c, e, "graph instantiate");
        }
        it = c->graphs.emplace(key, rec).first;
    }
    cudaError_t e = cudaGraphLaunch(it->second.exec, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph launch");
    it->second.last_use = ++c->graph_tick;
    c->launches += it->second.launches;
    for (const ProfEntry &pe : it->second.prof) c->pending.push_back(pe);
    fence_record(c, st);
    return BTE_OK;
}

bte_status bte_graph_count(const bte_ctx *c, int64_t *count) {
    if (!c || !count) return BTE_EINVAL;
    *count = (int64_t)c->graphs.size();
    return BTE_OK;
}

bte_status bte_profile_enable(bte_ctx *c, int enable) {
    if (!c) return BTE_EINVAL;
    if (c->prof != (enable != 0)) drop_graphs(c);  // step graphs are captured again, with or without events
    c->prof = enable != 0;
    return BTE_OK;
}

bte_status bte_profile_read(bte_ctx *c, const char *kernel, int64_t *launches, double *total_ms, void *stream) {
    if (!c || !kernel || !launches || !total_ms) return fail(c, BTE_EINVAL, "bte_profile_read: bad arguments");
    int want = -1;
    if (!std::strcmp(kernel, "conv32")) want = PK_CONV32;
    else if (!std::strcmp(kernel, "conv64")) want = PK_CONV64;
    else if (!std::strcmp(kernel, "collide")) want = PK_COLLIDE;
    else if (!std::strcmp(kernel, "forward")) want = PK_FORWARD;
    else if (!std::strcmp(kernel, "inverse")) want = PK_INVERSE;
    else if (!std::strcmp(kernel, "transport")) want = PK_TRANSPORT;
    else if (std::strcmp(kernel, "*") != 0) return fail(c, BTE_EINVAL, "bte_profile_read: unknown kernel name");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
    int64_t n = 0;
    double ms = 0.0;
    // entries owned by graphs stay with the graphs; the others return to the pool
    std::vector<cudaEvent_t> owned;
    for (auto &kv : c->graphs)
        for (auto &pe : kv.second.prof) owned.push_back(pe.a);
    std::vector<ProfEntry> keep;
    for (const ProfEntry &pe : c->pending) {
        if (want >= 0 && pe.kernel != want) {  // another kernel's entry stays pending
            keep.push_back(pe);
            continue;
        }
        float t = 0.f;
        if (cudaEventElapsedTime(&t, pe.a, pe.b) == cudaSuccess) {
            ms += t;
            ++n;
        } else {
            cudaGetLastError();
        }
        if (std::find(owned.begin(), owned.end(), pe.a) == owned.end()) c->ev_free.push_back({pe.a, pe.b});
    }
    c->pending.swap(keep);
    *launches = n;
    *total_ms = ms;
    return BTE_OK;
}

bte_status bte_launch_count(const bte_ctx *c, int64_t *count) {
    if (!c || !count) return BTE_EINVAL;
    *count = c->launches;
    return BTE_OK;
}

static int *option_slot(bte_ctx *c, const char *name, int *lo, int *hi) {
    if (!std::strcmp(name, "conv_impl")) { *lo = 0; *hi = 5; return &c->conv_impl; }
    if (!std::strcmp(name, "dft_split")) { *lo = 1; *hi = 4; return &c->dft_split; }
    if (!std::strcmp(name, "debug_conv_stall")) { *lo = 0; *hi = 1; return &c->debug_conv_stall; }
    if (!std::strcmp(name, "profile_mask")) { *lo = 0; *hi = 63; return &c->prof_mask; }
    if (!std::strcmp(name, "conv_warps")) { *lo = 1; *hi = 8; return &c->conv_warps; }
    if (!std::strcmp(name, "conv_stages")) { *lo = 0; *hi = 4; return &c->conv_stages; }
    if (!std::strcmp(name, "conv_merge")) { *lo = 1; *hi = 1 << 20; return &c->conv_merge; }
    if (!std::strcmp(name, "conv_split")) { *lo = 0; *hi = 1; return &c->conv_split; }
    if (!std::strcmp(name, "batch_cache")) { *lo = 2; *hi = 1 << 20; return &c->batch_cache_max; }
    if (!std::strcmp(name, "graph_cache")) { *lo = 1; *hi = 1 << 20; return &c->graph_cache_max; }
    if (!std::strcmp(name, "learned_tol_ppm")) { *lo = 0; *hi = 1 << 30; return &c->learned_tol_ppm; }
    if (!std::strcmp(name, "dft_fuse_stages")) { *lo = 0; *hi = 1; return &c->dft_fuse_stages; }
    return nullptr;
}

bte_status bte_set_option(bte_ctx *c, const char *name, int value) {
    if (!c || !name) return BTE_EINVAL;
    int lo, hi;
    int *slot = option_slot(c, name, &lo, &hi);
    if (!slot) return fail(c, BTE_EINVAL, std::string("unknown option ") + name);
    if (value < lo || value > hi) return fail(c, BTE_EINVAL, std::string("option out of range: ") + name);
    if (*slot != value) {
        drop_graphs(c);
        *slot = value;
    }
    // an explicit choice of the FP32 path's configuration replaces the tuned ones
    if (!std::strncmp(name, "conv_", 5) || !std::strcmp(name, "dft_split")) {
        c->tuned.clear();
        cudaSetDevice(c->device);
        return prime_configs(c);
    }
    return BTE_OK;
}

bte_status bte_get_option(const bte_ctx *c, const char *name, int *value) {
    if (!c || !name || !value) return BTE_EINVAL;
    int lo, hi;
    int *slot = option_slot(const_cast<bte_ctx *>(c), name, &lo, &hi);
    if (!slot) return BTE_EINVAL;
    *value = *slot;
    return BTE_OK;
}

bte_status bte_learned_stats(bte_ctx *c, int64_t *cells, int64_t *fallbacks, double *max_indicator, int reset) {
    if (!c) return BTE_EINVAL;
    unsigned long long h[4] = {0, 0, 0, 0};
    if (c->d_lstats) {
        cudaSetDevice(c->device);
        cudaError_t e = quiesce(c);  // the context's learned calls and steps have finished
        if (e == cudaSuccess) e = cudaMemcpy(h, c->d_lstats, sizeof h, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && reset) e = cudaMemsetAsync(c->d_lstats, 0, sizeof h, 0);
        if (e == cudaSuccess) e = cudaStreamSynchronize(0);
        if (e != cudaSuccess) return cuda_fail(c, e, "bte_learned_stats");
    }
    if (cells) *cells = (int64_t)h[0];
    if (fallbacks) *fallbacks = (int64_t)h[1];
    if (max_indicator) {
        const unsigned bits = (unsigned)h[2];
        float v;
        std::memcpy(&v, &bits, sizeof v);
        *max_indicator = (double)v;
    }
    return BTE_OK;
}

bte_status bte_learned_sample(bte_ctx *c, int *kk, int cap, int *S) {
    if (!c || !S) return BTE_EINVAL;
    if (c->tables.empty()) return fail(c, BTE_ESTATE, "bte_learned_sample: no weight tables");
    cudaSetDevice(c->device);
    bte_status s = ensure_indicator(c);
    if (s != BTE_OK) return s;
    *S = c->ind->S;
    if (kk)
        for (int i = 0; i < c->ind->S && i < cap; ++i) kk[i] = c->ind->kks[i];
    return BTE_OK;
}

bte_status bte_learned_indicator(bte_ctx *c, const double *f, const double *Q, int64_t ncells, double *ind,
                                 void *stream) {
    if (!c) return BTE_EINVAL;
    if (!f || !Q || !ind) return fail(c, BTE_EINVAL, "bte_learned_indicator: null pointer");
    if (c->tables.empty()) return fail(c, BTE_ESTATE, "bte_learned_indicator: no weight tables");
    if (c->tables[0]->N > 16) return fail(c, BTE_EINVAL, "bte_learned_indicator: table 0 must have N <= 16");
    cudaSetDevice(c->device);
    Batch *B = nullptr;
    bte_status s;
    if ((s = get_batch(c, nullptr, ncells, &B)) != BTE_OK) return s;
    if ((s = prepare(c, B, BTE_FP32, false, false)) != BTE_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    float *d_ind = nullptr;
    if ((s = enqueue_indicator(c, B, f, Q, &d_ind, st)) != BTE_OK) return s;
    launch_widen(d_ind, ind, (int)ncells, st);
    count_launches(c, 1);
    fence_record(c, st);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BTE_OK : cuda_fail(c, e, "bte_learned_indicator: launch");
}

bte_status bte_sync_status(bte_ctx *c, void *stream) {
    if (!c) return BTE_EINVAL;
    cudaSetDevice(c->device);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
    int st = 0;
    e = cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "status read");
    if (st) cudaMemset(c->d_status, 0, sizeof(int));
    if (st & ST_TIMEOUT) return fail(c, BTE_ETIMEOUT, "a bounded wait in a kernel ran out");
    if (st & ST_BADDESC) return fail(c, BTE_ECUDA, "a convolution block descriptor was out of range");
    if (st & ST_NONFINITE) return fail(c, BTE_ENONFINITE, "non-finite value in the input f");
    return BTE_OK;
}

bte_status bte_autotune(bte_ctx *c, const double *f, const bte_instance *inst, int64_t ninst, int reps,
                        int *out_cfg, double *out_ms, void *stream) {
    if (!c || !f || ninst <= 0) return fail(c, BTE_EINVAL, "bte_autotune: bad arguments");
    if (c->tables.empty()) return fail(c, BTE_ESTATE, "bte_autotune: no weight tables");
    cudaSetDevice(c->device);
    reps = reps < 1 ? 1 : (reps > 100 ? 100 : reps);
    cudaStream_t st = (cudaStream_t)stream;
    Batch *B = nullptr;
    bte_status s = get_batch(c, inst, ninst, &B);
    if (s != BTE_OK) return s;
    if ((s = ensure_scratch(c, SC_Q2, sizeof(double) * (size_t)B->extent)) != BTE_OK) return s;
    double *Qtmp = (double *)c->scratch[SC_Q2];
    bool small_n = true;
    for (const Segment &sg : B->segs) small_n = small_n && c->tables[sg.table]->N <= 16;
    const std::string key = tune_key(B);
    const bool had = c->tuned.count(key) != 0;
    const ConvCfg before = had ? c->tuned[key] : ConvCfg{};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "bte_autotune: events");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(c, cudaGetLastError(), "bte_autotune: events");
    }
    ConvCfg best;
    best.ms = -1.0;
    bte_status err = BTE_OK;
    for (int impl : {4, 2, 1, 3})
        for (int warps : {4, 3})
            for (int stages : {1, 2})
                for (int merge : {16, 32})
                    for (int split : {4, 2, 1})
                        for (int csplit : {1, 0}) {
                        if (!small_n && split != 4) continue;
                        if (csplit && (impl != 4 || B->nsplit == 0)) continue;
                        // kinds of N = 48: variant 4, and 3 when they are the only kinds
                        if ((B->kinds_mask >> 7) && impl != 4 && !(impl == 3 && B->kinds_mask == (128u | 256u | 512u)))
                            continue;
                        ConvCfg g;
                        g.impl = impl;
                        g.warps = warps;
                        g.stages = stages;
                        g.merge = merge;
                        g.split = split;
                        g.csplit = csplit;
                        c->tuned[key] = g;
                        if ((err = prepare(c, B, BTE_FP32, false, false)) != BTE_OK) break;
                        if ((err = enqueue_collide(c, B, f, Qtmp, BTE_FP32, POST_PROJECT, nullptr, nullptr, nullptr,
                                                   0.0, st)) != BTE_OK)
                            break;  // warm-up (kernel attributes, caches)
                        cudaEventRecord(e0, st);
                        for (int r = 0; r < reps && err == BTE_OK; ++r)
                            err = enqueue_collide(c, B, f, Qtmp, BTE_FP32, POST_PROJECT, nullptr, nullptr, nullptr,
                                                  0.0, st);
                        cudaEventRecord(e1, st);
                        cudaError_t ce = cudaEventSynchronize(e1);
                        float ms = 0.f;
                        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
                        if (ce != cudaSuccess) err = cuda_fail(c, ce, "bte_autotune: timing");
                        if (err != BTE_OK) break;
                        g.ms = ms / reps;
                        if (best.ms < 0.0 || g.ms < best.ms) best = g;
                    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (const ProfEntry &pe : c->pending)  // profile entries of the trial runs are not the caller's
        if (!owned_by_graph(c, pe.a)) c->ev_free.push_back({pe.a, pe.b});
    c->pending.clear();
    if (err == BTE_OK) err = bte_sync_status(c, stream);
    if (err != BTE_OK || best.ms < 0.0) {
        if (had) c->tuned[key] = before;
        else c->tuned.erase(key);
        return err != BTE_OK ? err : fail(c, BTE_ECUDA, "bte_autotune: no configuration ran");
    }
    c->tuned[key] = best;
    drop_graphs(c);  // captured steps used the previous configuration
    if ((s = prepare(c, B, BTE_FP32, false, false)) != BTE_OK) return s;
    if (out_cfg) {
        out_cfg[0] = best.impl;
        out_cfg[1] = best.warps;
        out_cfg[2] = best.stages;
        out_cfg[3] = best.merge;
        out_cfg[4] = best.split;
        out_cfg[5] = best.csplit;
    }
    if (out_ms) *out_ms = best.ms;
    return BTE_OK;
}

namespace {
struct StateHeader {
    char magic[8];     // "BTESTATE"
    uint32_t version;  // 1
    uint32_t pad;
    int64_t n;
    double t;
    int64_t step;
    uint64_t grids;    // FNV-1a of the context's (N, L, lambda) list
};
static_assert(sizeof(StateHeader) == 48, "state header layout");

uint64_t grids_hash(const bte_ctx *c) {
    uint64_t h = 1469598103934665603ull;
    for (const Table *t : c->tables) {
        const double v[3] = {(double)t->N, t->L, t->lam};
        h = fnv1a(v, sizeof v, h);
        if (t->beta != 1.0) h = fnv1a(&t->beta, sizeof t->beta, h);  // elastic grids hash as before
    }
    return h;
}
}  // namespace

bte_status bte_state_save(bte_ctx *c, const char *path, const double *f, int64_t n, double t, int64_t step,
                          void *stream) {
    if (!c || !path || !f || n <= 0) return fail(c, BTE_EINVAL, "bte_state_save: bad arguments");
    cudaSetDevice(c->device);
    std::vector<double> h((size_t)n);
    cudaError_t e = cudaMemcpyAsync(h.data(), f, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost,
                                    (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "bte_state_save: copy");
    StateHeader hd{};
    std::memcpy(hd.magic, "BTESTATE", 8);
    hd.version = 1;
    hd.n = n;
    hd.t = t;
    hd.step = step;
    hd.grids = grids_hash(c);
    uint64_t sum = fnv1a(&hd, sizeof hd);
    sum = fnv1a(h.data(), sizeof(double) * h.size(), sum);
    FILE *fp = std::fopen(path, "wb");
    if (!fp) return fail(c, BTE_EINVAL, std::string("bte_state_save: cannot write ") + path);
    bool ok = std::fwrite(&hd, sizeof hd, 1, fp) == 1 && std::fwrite(h.data(), sizeof(double), h.size(), fp) == h.size() &&
              std::fwrite(&sum, sizeof sum, 1, fp) == 1;
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? BTE_OK : fail(c, BTE_EINVAL, "bte_state_save: write failed");
}

bte_status bte_state_load(bte_ctx *c, const char *path, double *f, int64_t n, double *t, int64_t *step,
                          void *stream) {
    if (!c || !path || !f || n <= 0) return fail(c, BTE_EINVAL, "bte_state_load: bad arguments");
    FILE *fp = std::fopen(path, "rb");
    if (!fp) return fail(c, BTE_EINVAL, std::string("bte_state_load: cannot read ") + path);
    StateHeader hd{};
    bool ok = std::fread(&hd, sizeof hd, 1, fp) == 1 && std::memcmp(hd.magic, "BTESTATE", 8) == 0 && hd.version == 1;
    if (!ok) {
        std::fclose(fp);
        return fail(c, BTE_EINVAL, "bte_state_load: not a state file (magic or version)");
    }
    if (hd.n != n) {
        std::fclose(fp);
        return fail(c, BTE_EINVAL, "bte_state_load: the file holds " + std::to_string(hd.n) + " values, not " +
                                       std::to_string(n));
    }
    std::vector<double> h((size_t)n);
    uint64_t stored = 0;
    ok = std::fread(h.data(), sizeof(double), h.size(), fp) == h.size() && std::fread(&stored, sizeof stored, 1, fp) == 1;
    std::fclose(fp);
    if (!ok) return fail(c, BTE_EINVAL, "bte_state_load: truncated file");
    uint64_t sum = fnv1a(&hd, sizeof hd);
    sum = fnv1a(h.data(), sizeof(double) * h.size(), sum);
    if (sum != stored) return fail(c, BTE_EINVAL, "bte_state_load: checksum mismatch (corrupt file)");
    if (hd.grids != grids_hash(c))
        return fail(c, BTE_ESTATE, "bte_state_load: written under other weight grids (N, L, lambda)");
    cudaSetDevice(c->device);
    cudaError_t e = cudaMemcpyAsync(f, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice,
                                    (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "bte_state_load: copy");
    if (t) *t = hd.t;
    if (step) *step = hd.step;
    return BTE_OK;
}

bte_status bte_tune_save(const bte_ctx *c, const char *path) {
    if (!c || !path) return BTE_EINVAL;
    FILE *fp = std::fopen(path, "w");
    if (!fp) return fail(const_cast<bte_ctx *>(c), BTE_EINVAL, std::string("bte_tune_save: cannot write ") + path);
    std::fprintf(fp, "{\n\"gpu\": \"%s\",\n\"entries\": [\n", c->gpu_name.c_str());
    size_t i = 0;
    for (const auto &kv : c->tuned) {
        const ConvCfg &g = kv.second;
        std::fprintf(fp, "{\"key\": \"%s\", \"impl\": %d, \"warps\": %d, \"stages\": %d, \"merge\": %d, "
                         "\"split\": %d, \"csplit\": %d, \"ms\": %.6f}%s\n",
                     kv.first.c_str(), g.impl, g.warps, g.stages, g.merge, g.split, g.csplit, g.ms,
                     ++i < c->tuned.size() ? "," : "");
    }
    std::fprintf(fp, "]\n}\n");
    const bool ok = std::fclose(fp) == 0;
    return ok ? BTE_OK : fail(const_cast<bte_ctx *>(c), BTE_EINVAL, "bte_tune_save: write failed");
}

bte_status bte_tune_load(bte_ctx *c, const char *path, int *loaded) {
    if (!c || !path) return BTE_EINVAL;
    if (loaded) *loaded = 0;
    FILE *fp = std::fopen(path, "r");
    if (!fp) return fail(c, BTE_EINVAL, std::string("bte_tune_load: cannot read ") + path);
    std::string text;
    char buf[4096];
    size_t n;
    while ((n = std::fread(buf, 1, sizeof buf, fp)) > 0) text.append(buf, n);
    std::fclose(fp);
    // the format bte_tune_save writes: one entry per line
    const size_t g0 = text.find("\"gpu\": \"");
    if (g0 == std::string::npos) return fail(c, BTE_EINVAL, "bte_tune_load: not a tuning cache");
    const size_t g1 = text.find('"', g0 + 8);
    if (g1 == std::string::npos) return fail(c, BTE_EINVAL, "bte_tune_load: not a tuning cache");
    const std::string gpu = text.substr(g0 + 8, g1 - (g0 + 8));
    if (gpu != c->gpu_name) return BTE_OK;  // tuned on another GPU: nothing applies
    std::map<std::string, ConvCfg> got;
    size_t pos = 0;
    while ((pos = text.find("{\"key\": \"", pos)) != std::string::npos) {
        const size_t eol = text.find('\n', pos);
        const std::string line = text.substr(pos, eol == std::string::npos ? std::string::npos : eol - pos);
        char key[128] = {0};
        ConvCfg g;
        if (std::sscanf(line.c_str(),
                        "{\"key\": \"%127[^\"]\", \"impl\": %d, \"warps\": %d, \"stages\": %d, \"merge\": %d, "
                        "\"split\": %d, \"csplit\": %d, \"ms\": %lf}",
                        key, &g.impl, &g.warps, &g.stages, &g.merge, &g.split, &g.csplit, &g.ms) != 8)
            return fail(c, BTE_EINVAL, "bte_tune_load: malformed entry: " + line);
        if (g.impl < 0 || g.impl > 5 || g.warps < 1 || g.warps > 8 || g.stages < 0 || g.stages > 4 || g.merge < 1 ||
            g.csplit < 0 || g.csplit > 1 ||
            (g.split != 1 && g.split != 2 && g.split != 4))
            return fail(c, BTE_EINVAL, "bte_tune_load: out-of-range entry: " + line);
        got[key] = g;
        pos += 10;
    }
    drop_graphs(c);
    for (auto &kv : got) c->tuned[kv.first] = kv.second;
    if (loaded) *loaded = (int)got.size();
    return BTE_OK;
}

}  // extern "C"
