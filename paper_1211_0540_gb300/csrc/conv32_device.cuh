// FP32 weighted convolution of Sec. 3.2 (the O(N^6) hot loop):
//   Qhat(zeta_k) = dz^3 sum_m Ghat(xi_m, zeta_k) fhat(xi_m) fhat(zeta_k - xi_m),
// zero extension: only m with n = k - m + N/2 on the grid.
//
// Design (GB300, sm_103a):
// - One warp lane per spatial cell: a warp evaluates the same (zeta, xi) pairs
//   for 32 cells, so each weight is loaded once per warp and shared by 32
//   cells (the paper's weights Ghat are the same for every cell, Sec. 4).
// - Pair symmetry: fhat_m fhat_n serves both m and its partner n, so every
//   unordered pair is evaluated once with the weight Ghat(k,m) + Ghat(k,n)
//   (host-packed, see tables.cpp). Half the products, half the weight bytes.
// - Work item = (32-cell group, pencil (k1, k2), k3 tile of T outputs). The
//   item loops over the kept (m1, m2) blocks of the pencil. For each block the
//   row fhat[m1][m2][:] ("a"), the partner row fhat[n1][n2][:] ("b") and the
//   block's weights are brought into a per-warp shared-memory ring by TMA bulk
//   copies (cp.async.bulk, mbarrier transaction counts). The block is then a
//   fully unrolled (m3, k3) loop: each a-value is reused for all T outputs of
//   the tile, each b-value by T pairs along the diagonal k3 - m3, weights are
//   read as warp-uniform 16-byte shared loads.
// - Accumulation: plain FP32 FMAs inside `merge` blocks, then Knuth's TwoSum
//   folds the partial into a (hi, lo) pair per output (compensated sum).
// - Persistent grid (one resident wave), items taken from an atomic queue in
//   LPT order (costliest first). Every wait is bounded by the global timer; on
//   expiry the warp records BTE_ETIMEOUT in the status word, waits (bounded)
//   for its own copies in flight and leaves.
//
// This header holds the device code; conv32.cu instantiates the kernels for
// the common kind sets and holds the host-side configuration, conv32_wide.cu
// the kernels over the N = 48 kinds (compiled in parallel).
#pragma once

#include "kernels.h"

namespace bte {

namespace {

constexpr int kMaxStages = 4;
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // 1 s

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait on one phase of a stage barrier; false after kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > kWaitLimitNs) return false;
    }
    return true;
}

// Compile-time shape of one kernel variant.
template <int N_, int T_, int K0_>
struct Kind {
    static constexpr int N = N_, T = T_, K0 = K0_, H = N_ / 2;
    static constexpr int lo(int k) { return k - H + 1 > 0 ? k - H + 1 : 0; }
    static constexpr int hi(int k) { return k + H < N - 1 ? k + H : N - 1; }
    static constexpr int count() {
        int c = 0;
        for (int j = 0; j < T; ++j) c += hi(K0 + j) - lo(K0 + j) + 1;
        return c;
    }
    static constexpr int cpad = (count() + 3) & ~3;
    static constexpr int row_bytes = N * kLanes * 8;
    static constexpr int stage_bytes = 2 * row_bytes + cpad * 4;
};

using K8 = Kind<8, 8, 0>;
using K12 = Kind<12, 12, 0>;
using K16 = Kind<16, 16, 0>;
using K24a = Kind<24, 12, 0>;
using K24b = Kind<24, 12, 12>;
using K32a = Kind<32, 16, 0>;
using K32b = Kind<32, 16, 16>;
using K48a = Kind<48, 16, 0>;
using K48b = Kind<48, 16, 16>;
using K48c = Kind<48, 16, 32>;

// One block: a-row, b-row and weights of stage `st` into the part accumulators.
template <class K>
__device__ __forceinline__ void conv_block(const char *st, int lane, float (&part)[2 * K::T]) {
    const float2 *A = reinterpret_cast<const float2 *>(st);
    const float2 *B = A + K::N * kLanes;
    const float4 *W4 = reinterpret_cast<const float4 *>(B + K::N * kLanes);
    float4 w4 = make_float4(0.f, 0.f, 0.f, 0.f);
    int wi = 0;
#pragma unroll
    for (int m3 = 0; m3 < K::N; ++m3) {
        const float2 a = A[m3 * kLanes + lane];
#pragma unroll
        for (int j = 0; j < K::T; ++j) {
            const int n3 = K::K0 + j - m3 + K::H;
            if (n3 >= 0 && n3 < K::N) {
                if ((wi & 3) == 0) w4 = W4[wi >> 2];
                const float w = (wi & 3) == 0 ? w4.x : (wi & 3) == 1 ? w4.y : (wi & 3) == 2 ? w4.z : w4.w;
                ++wi;
                const float2 b = B[n3 * kLanes + lane];
                const float tr = w * a.x, ti = w * a.y;
                part[2 * j] = fmaf(tr, b.x, part[2 * j]);
                part[2 * j] = fmaf(-ti, b.y, part[2 * j]);
                part[2 * j + 1] = fmaf(tr, b.y, part[2 * j + 1]);
                part[2 * j + 1] = fmaf(ti, b.x, part[2 * j + 1]);
            }
        }
    }
}

struct WarpRing {
    char *base;        // stages * stage_bytes (this warp's ring)
    uint32_t bars;     // shared address of the first stage barrier (8 bytes each)
    uint32_t phase;    // bit s: parity of the next completion of stage s
    int stage_bytes;
};

// Issue the three bulk copies of block j of the item into stage s (lane 0 only);
// with OTF only the two rows (the warp builds the weights, gen_weights).
template <class K, bool OTF = false>
__device__ __forceinline__ void issue_block(const WarpRing &r, int s, const ConvItem &it,
                                            const ConvParams &p, int j) {
    const uint32_t d = p.D[it.table][it.desc_off + j];
    int m1 = (int)(d & 0xffffu), m2 = (int)(d >> 16);
    int n1 = (int)it.k1 - m1 + K::H, n2 = (int)it.k2 - m2 + K::H;
    if (m1 >= K::N || m2 >= K::N || n1 < 0 || n1 >= K::N || n2 < 0 || n2 >= K::N) {
        atomicOr(p.status, ST_BADDESC);
        m1 = m2 = n1 = n2 = 0;  // stay in bounds; the result is flagged as invalid
    }
    const float2 *Fg = p.F + it.fofs;
    const float2 *arow = Fg + (size_t)((m1 * K::N + m2) * K::N) * kLanes;
    const float2 *brow = Fg + (size_t)((n1 * K::N + n2) * K::N) * kLanes;
    const float *w = p.W[it.table] + it.wofs + (size_t)j * K::cpad;
    char *dst = r.base + s * r.stage_bytes;
    const uint32_t bar = r.bars + 8u * s;
    mbar_expect_tx(bar, (uint32_t)(OTF ? 2 * K::row_bytes : K::stage_bytes));
    bulk_g2s(smem_u32(dst), arow, K::row_bytes, bar);
    bulk_g2s(smem_u32(dst + K::row_bytes), brow, K::row_bytes, bar);
    if (!OTF) bulk_g2s(smem_u32(dst + 2 * K::row_bytes), w, K::cpad * 4, bar);
}

// The weights of block j of the item, built by the whole warp into the weight
// slot of stage s from the radial integrals (conv_impl 5, the weights computed
// on the fly instead of streamed, Sec. 5's remark on storing Ghat). With
// k' = k - N/2 (likewise m', n' = k' - m') the block's pair weight is
//   Ghat(k, m) + Ghat(k, n) = [I(|k'|^2, |2m' - k'|^2) - J(|m'|^2)] + [I(..) - J(|n'|^2)],
// the gain arguments of m and n being equal (|2n' - k'| = |k' - 2m'|); a block
// that pairs with itself keeps Ghat(k, m). I and J carry sqrt(2/pi) dz^3.
// Entry e of the tile has the third-component parts of the four invariants
// precomputed, C[e] = (k3'^2 | (2m3' - k3')^2 << 16, m3'^2 | n3'^2 << 16); the
// padding up to cpad is 0. Lane l builds entries l, l + 32, ...: all its
// table reads are issued before the first weight is formed (one memory
// latency per block instead of one per entry).
template <class K>
__device__ __forceinline__ void gen_weights(const WarpRing &r, int s, const ConvItem &it, const ConvParams &p, int jb,
                                            int lane) {
    constexpr int NE = (K::cpad + kLanes - 1) / kLanes;
    const uint32_t d = p.D[it.table][it.desc_off + jb];
    const int m1 = (int)(d & 0xffffu), m2 = (int)(d >> 16);
    const int n1 = (int)it.k1 - m1 + K::H, n2 = (int)it.k2 - m2 + K::H;
    const bool valid = m1 < K::N && m2 < K::N && n1 >= 0 && n1 < K::N && n2 >= 0 && n2 < K::N;
    const int k1 = (int)it.k1 - K::H, k2 = (int)it.k2 - K::H, a1 = m1 - K::H, a2 = m2 - K::H;
    const int p12 = k1 * k1 + k2 * k2;
    const int q12 = (2 * a1 - k1) * (2 * a1 - k1) + (2 * a2 - k2) * (2 * a2 - k2);
    const int sm12 = a1 * a1 + a2 * a2, sn12 = (k1 - a1) * (k1 - a1) + (k2 - a2) * (k2 - a2);
    const bool pair = !(m1 == n1 && m2 == n2);
    const float *__restrict__ I = p.I32[it.table];
    const float *__restrict__ J = p.J32[it.table];
    const int nq = p.nq[it.table];
    const uint2 *__restrict__ C =
        reinterpret_cast<const uint2 *>(p.E[it.table]) + (K::K0 / K::T) * p.estride[it.table];
    float g[NE], gm[NE], gn[NE];
#pragma unroll
    for (int t = 0; t < NE; ++t) {
        const int e = lane + t * kLanes;
        g[t] = gm[t] = gn[t] = 0.f;
        if (valid && e < K::count()) {
            const uint2 c = __ldg(C + e);
            const int pp = p12 + (int)(c.x & 0xffffu), q = q12 + (int)(c.x >> 16);
            g[t] = __ldg(I + (size_t)pp * nq + q);
            gm[t] = __ldg(J + sm12 + (int)(c.y & 0xffffu));
            gn[t] = __ldg(J + sn12 + (int)(c.y >> 16));
        }
    }
    float *w = reinterpret_cast<float *>(r.base + s * r.stage_bytes + 2 * K::row_bytes);
#pragma unroll
    for (int t = 0; t < NE; ++t) {
        const int e = lane + t * kLanes;
        const float a = g[t] - gm[t];
        if (e < K::cpad) w[e] = pair ? a + (g[t] - gn[t]) : a;
    }
}

// Process one item; returns false if a wait timed out (the ring is drained).
template <class K>
__device__ bool conv_item(WarpRing &r, const ConvItem &it, const ConvParams &p, int lane) {
    const int nb = (int)it.nblocks;
    const int S = p.stages;
    if (lane == 0)
        for (int s = 0; s < S && s < nb; ++s) issue_block<K>(r, s, it, p, s);
    __syncwarp();

    float part[2 * K::T], hi[2 * K::T], lo[2 * K::T];
#pragma unroll
    for (int i = 0; i < 2 * K::T; ++i) part[i] = hi[i] = lo[i] = 0.f;

    int since = 0;
    bool ok = true;
    int j = 0;
    for (; j < nb; ++j) {
        const int s = j % S;
        const uint32_t par = (r.phase >> s) & 1u;
        bool got = mbar_wait_bounded(r.bars + 8u * s, par);
        got = __all_sync(0xffffffffu, got);
        if (!got) {
            ok = false;
            break;
        }
        r.phase ^= (1u << s);
        conv_block<K>(r.base + s * r.stage_bytes, lane, part);
        if (++since == p.merge || j == nb - 1) {
            since = 0;
#pragma unroll
            for (int i = 0; i < 2 * K::T; ++i) {  // TwoSum(hi, part)
                const float sum = hi[i] + part[i];
                const float bp = sum - hi[i];
                const float err = (hi[i] - (sum - bp)) + (part[i] - bp);
                hi[i] = sum;
                lo[i] += err;
                part[i] = 0.f;
            }
        }
        __syncwarp();
        if (lane == 0 && j + S < nb) issue_block<K>(r, s, it, p, j + S);
    }
    if (!ok) {
        if (lane == 0) atomicOr(p.status, ST_TIMEOUT);
        // drain: wait (bounded) for every copy this warp still has in flight
        const int last = nb < j + S ? nb : j + S;
        for (int jj = j; jj < last; ++jj) {
            const int s = jj % S;
            if (mbar_wait_bounded(r.bars + 8u * s, (r.phase >> s) & 1u)) r.phase ^= (1u << s);
        }
        __syncwarp();
        return false;
    }
    float2 *Q = p.Qh + it.fofs + ((size_t)(it.k1 * K::N + it.k2) * K::N + K::K0) * kLanes + lane;
#pragma unroll
    for (int t = 0; t < K::T; ++t) Q[t * kLanes] = make_float2(hi[2 * t] + lo[2 * t], hi[2 * t + 1] + lo[2 * t + 1]);
    return true;
}

template <class K>
__device__ __forceinline__ bool run_kind(WarpRing &r, const ConvItem &it, const ConvParams &p,
                                         int lane) {
    return conv_item<K>(r, it, p, lane);
}

// MASK: set of kinds compiled into this kernel instance.
template <unsigned MASK>
__global__ void __launch_bounds__(256) conv32_kernel(ConvParams p) {
    extern __shared__ __align__(128) char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    WarpRing r;
    r.base = smem + (size_t)warp * p.warp_smem;
    r.stage_bytes = p.warp_smem / p.stages;
    r.bars = smem_u32(smem + (size_t)nwarps * p.warp_smem) + 8u * kMaxStages * warp;
    r.phase = 0;
    if (lane == 0) {
        for (int s = 0; s < p.stages; ++s) mbar_init(r.bars + 8u * s, 1);
        fence_mbar_init();
    }
    __syncwarp();
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = (int)atomicAdd(p.counter, 1u);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= p.nitems) break;
        const ConvItem it = p.items[idx];
        bool ok = true;
        switch (it.kind) {
            case 0: if (MASK & 1u) ok = run_kind<K8>(r, it, p, lane); break;
            case 1: if (MASK & 2u) ok = run_kind<K12>(r, it, p, lane); break;
            case 2: if (MASK & 4u) ok = run_kind<K16>(r, it, p, lane); break;
            case 3: if (MASK & 8u) ok = run_kind<K24a>(r, it, p, lane); break;
            case 4: if (MASK & 16u) ok = run_kind<K24b>(r, it, p, lane); break;
            case 5: if (MASK & 32u) ok = run_kind<K32a>(r, it, p, lane); break;
            case 6: if (MASK & 64u) ok = run_kind<K32b>(r, it, p, lane); break;
            case 7: if (MASK & 128u) ok = run_kind<K48a>(r, it, p, lane); break;
            case 8: if (MASK & 256u) ok = run_kind<K48b>(r, it, p, lane); break;
            case 9: if (MASK & 512u) ok = run_kind<K48c>(r, it, p, lane); break;
            default: ok = false; break;
        }
        if (!ok) break;
    }
}

// ---------------------------------------------------------------------------
// v2: CTA-cooperative items and packed (f32x2) arithmetic.
// All warps of a CTA work on the same item: warp w takes blocks w, w + W, ...
// of the pencil through its own ring; the W partial (hi, lo) sums are then
// reduced through shared memory in a fixed warp order (deterministic). This
// keeps every warp of a resident CTA busy and turns the heavy-tailed pencil
// costs into many balanced units. With PACKED, a pair costs three packed
// instructions: p = (a.re, a.re) * (b.re, b.im) + (a.im, a.im) * (-b.im, b.re),
// acc += (w, w) * p, which occupy the FP32 pipe as six scalar operations but
// leave issue slots free for the shared loads and bookkeeping.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t pk2(float x, float y) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
    return r;
}
__device__ __forceinline__ float2 up2(uint64_t v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ uint64_t fmul2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

template <class K>
__device__ __forceinline__ void conv_block_packed(const char *st, int lane, uint64_t (&part)[K::T]) {
    const float2 *A = reinterpret_cast<const float2 *>(st);
    const float2 *B = A + K::N * kLanes;
    const float4 *W4 = reinterpret_cast<const float4 *>(B + K::N * kLanes);
    float4 w4 = make_float4(0.f, 0.f, 0.f, 0.f);
    int wi = 0;
#pragma unroll
    for (int m3 = 0; m3 < K::N; ++m3) {
        const float2 a = A[m3 * kLanes + lane];
        const uint64_t aR = pk2(a.x, a.x), aI = pk2(a.y, a.y);
#pragma unroll
        for (int j = 0; j < K::T; ++j) {
            const int n3 = K::K0 + j - m3 + K::H;
            if (n3 >= 0 && n3 < K::N) {
                if ((wi & 3) == 0) w4 = W4[wi >> 2];
                const float w = (wi & 3) == 0 ? w4.x : (wi & 3) == 1 ? w4.y : (wi & 3) == 2 ? w4.z : w4.w;
                ++wi;
                const float2 b = B[n3 * kLanes + lane];
                uint64_t pr = fmul2(aR, pk2(b.x, b.y));
                pr = ffma2(aI, pk2(-b.y, b.x), pr);
                part[j] = ffma2(pk2(w, w), pr, part[j]);
            }
        }
    }
}

__device__ __forceinline__ void two_sum(float &hi, float &lo, float p) {
    const float s = hi + p;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (p - bp);
    hi = s;
}

// One item by all warps of the CTA. Returns false if this warp timed out.
template <class K, bool PACKED>
__device__ bool coop_item(WarpRing &r, const ConvItem &it, const ConvParams &p, int lane, int warp,
                          int nwarps, char *ring0) {
    constexpr int T = K::T;
    const int nb = (int)it.nblocks;
    const int S = p.stages;
    const int mine = nb > warp ? (nb - warp + nwarps - 1) / nwarps : 0;
    if (lane == 0)
        for (int s = 0; s < S && s < mine; ++s)
            if (!(p.stall && s == 0)) issue_block<K>(r, s, it, p, warp + s * nwarps);
    __syncwarp();

    float hi[2 * T], lo[2 * T];
    float part[2 * T];
    uint64_t pp[T];
#pragma unroll
    for (int i = 0; i < 2 * T; ++i) hi[i] = lo[i] = part[i] = 0.f;
#pragma unroll
    for (int i = 0; i < T; ++i) pp[i] = 0ull;

    bool ok = true;
    int since = 0, i = 0;
    for (; i < mine; ++i) {
        const int s = i % S;
        bool got = mbar_wait_bounded(r.bars + 8u * s, (r.phase >> s) & 1u);
        got = __all_sync(0xffffffffu, got);
        if (!got) {
            ok = false;
            break;
        }
        r.phase ^= (1u << s);
        if (PACKED) conv_block_packed<K>(r.base + s * r.stage_bytes, lane, pp);
        else conv_block<K>(r.base + s * r.stage_bytes, lane, part);
        if (++since == p.merge || i == mine - 1) {
            since = 0;
            if (PACKED) {
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    const float2 v = up2(pp[t]);
                    two_sum(hi[2 * t], lo[2 * t], v.x);
                    two_sum(hi[2 * t + 1], lo[2 * t + 1], v.y);
                    pp[t] = 0ull;
                }
            } else {
#pragma unroll
                for (int q = 0; q < 2 * T; ++q) {
                    two_sum(hi[q], lo[q], part[q]);
                    part[q] = 0.f;
                }
            }
        }
        __syncwarp();
        if (lane == 0 && i + S < mine) issue_block<K>(r, s, it, p, warp + (i + S) * nwarps);
    }
    if (!ok) {
        const int last = mine < i + S ? mine : i + S;
        for (int jj = i; jj < last; ++jj) {
            const int s = jj % S;
            if (mbar_wait_bounded(r.bars + 8u * s, (r.phase >> s) & 1u)) r.phase ^= (1u << s);
        }
        __syncwarp();
    }
    // partial sums of this warp into its own (drained) ring: [4T][32] floats
    float *red = reinterpret_cast<float *>(r.base);
#pragma unroll
    for (int q = 0; q < 2 * T; ++q) {
        red[q * kLanes + lane] = hi[q];
        red[(2 * T + q) * kLanes + lane] = lo[q];
    }
    return ok;
}

// Cross-warp reduction of the partials (fixed warp order) and the store.
template <class K>
__device__ __forceinline__ void coop_reduce(const ConvItem &it, const ConvParams &p, int lane, int warp,
                                            int nwarps, const char *ring0, int warp_smem, int sums_off = 0) {
    constexpr int T = K::T;
    float2 *Q = p.Qh + it.fofs + ((size_t)(it.k1 * K::N + it.k2) * K::N + K::K0) * kLanes + lane;
    for (int t = warp; t < T; t += nwarps) {
        float sr = 0.f, lr = 0.f, si = 0.f, li = 0.f;
        for (int w = 0; w < nwarps; ++w) {
            const float *red = reinterpret_cast<const float *>(ring0 + (size_t)w * warp_smem + sums_off);
            two_sum(sr, lr, red[(2 * t) * kLanes + lane]);
            lr += red[(2 * T + 2 * t) * kLanes + lane];
            two_sum(si, li, red[(2 * t + 1) * kLanes + lane]);
            li += red[(2 * T + 2 * t + 1) * kLanes + lane];
        }
        Q[t * kLanes] = make_float2(sr + lr, si + li);
    }
}

template <class K, bool PACKED>
__device__ __forceinline__ bool coop_run(WarpRing &r, const ConvItem &it, const ConvParams &p, int lane,
                                         int warp, int nwarps, char *ring0, int *abort_flag) {
    const bool ok = coop_item<K, PACKED>(r, it, p, lane, warp, nwarps, ring0);
    if (!ok && lane == 0) {
        atomicOr(p.status, ST_TIMEOUT);
        *abort_flag = 1;
    }
    __syncthreads();
    if (!*abort_flag) coop_reduce<K>(it, p, lane, warp, nwarps, ring0, p.warp_smem);
    __syncthreads();
    // the rings are next written by TMA (async proxy) after these generic accesses
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    return !*abort_flag;
}

// ---------------------------------------------------------------------------
// v4: as v2, with the compensated (hi, lo) sums of each warp in shared memory
// (4T x 32 floats after the warp's ring) instead of registers: they are
// touched only at a merge (every `merge` blocks). The registers freed let the
// block loop keep the b-row as packed (re, im) and (-im, re) operands for the
// whole block (N <= 16), so a pair costs its three packed FMA-pipe
// instructions and the (w, w) operand only. One-block rings keep 3 CTAs per
// SM (4 warps x (one 8.75 KB stage + 8 KB of sums) at N = 16).
// ---------------------------------------------------------------------------
template <class K>
__device__ __forceinline__ void conv_block_packed_h(const char *st, int lane, uint64_t (&part)[K::T]) {
    const float2 *A = reinterpret_cast<const float2 *>(st);
    const float2 *B = A + K::N * kLanes;
    const float4 *W4 = reinterpret_cast<const float4 *>(B + K::N * kLanes);
    uint64_t bb[K::N], bs[K::N];
#pragma unroll
    for (int n = 0; n < K::N; ++n) {
        const float2 b = B[n * kLanes + lane];
        bb[n] = pk2(b.x, b.y);
        bs[n] = pk2(-b.y, b.x);
    }
    float4 w4 = make_float4(0.f, 0.f, 0.f, 0.f);
    int wi = 0;
#pragma unroll
    for (int m3 = 0; m3 < K::N; ++m3) {
        const float2 a = A[m3 * kLanes + lane];
        const uint64_t aR = pk2(a.x, a.x), aI = pk2(a.y, a.y);
#pragma unroll
        for (int j = 0; j < K::T; ++j) {
            const int n3 = K::K0 + j - m3 + K::H;
            if (n3 >= 0 && n3 < K::N) {
                if ((wi & 3) == 0) w4 = W4[wi >> 2];
                const float w = (wi & 3) == 0 ? w4.x : (wi & 3) == 1 ? w4.y : (wi & 3) == 2 ? w4.z : w4.w;
                ++wi;
                uint64_t pr = fmul2(aR, bb[n3]);
                pr = ffma2(aI, bs[n3], pr);
                part[j] = ffma2(pk2(w, w), pr, part[j]);
            }
        }
    }
}

// Bytes of a warp's shared (hi, lo) sums: 4T x 32 floats with T <= 16.
constexpr int kSumsBytes = 4 * 16 * kLanes * 4;

// One item by all warps of the CTA, sums in shared memory at r.base + ring
// bytes. Returns false if this warp timed out.
// pre: the copies of this warp's first block were issued before (during the
// previous item's reduction).
template <class K, bool OTF>
__device__ bool coop_item_sm(WarpRing &r, const ConvItem &it, const ConvParams &p, int lane, int warp,
                             int nwarps, float *sums, bool pre) {
    constexpr int T = K::T;
    const int nb = (int)it.nblocks;
    const int S = p.stages;
    const int mine = nb > warp ? (nb - warp + nwarps - 1) / nwarps : 0;
    if (lane == 0)
        for (int s = pre ? 1 : 0; s < S && s < mine; ++s)
            if (!(p.stall && s == 0)) issue_block<K, OTF>(r, s, it, p, warp + s * nwarps);
    if (OTF)
        for (int s = pre ? 1 : 0; s < S && s < mine; ++s) gen_weights<K>(r, s, it, p, warp + s * nwarps, lane);
#pragma unroll
    for (int q = 0; q < 4 * T; ++q) sums[q * kLanes + lane] = 0.f;
    __syncwarp();
    uint64_t pp[T];
#pragma unroll
    for (int i = 0; i < T; ++i) pp[i] = 0ull;

    bool ok = true;
    int since = 0, i = 0;
    for (; i < mine; ++i) {
        const int s = i % S;
        bool got = mbar_wait_bounded(r.bars + 8u * s, (r.phase >> s) & 1u);
        got = __all_sync(0xffffffffu, got);
        if (!got) {
            ok = false;
            break;
        }
        r.phase ^= (1u << s);
        if (K::N <= 16) conv_block_packed_h<K>(r.base + s * r.stage_bytes, lane, pp);
        else conv_block_packed<K>(r.base + s * r.stage_bytes, lane, pp);
        if (++since == p.merge || i == mine - 1) {
            since = 0;
#pragma unroll
            for (int t = 0; t < T; ++t) {
                const float2 v = up2(pp[t]);
                float *h = sums + (2 * t) * kLanes + lane, *l = sums + (2 * T + 2 * t) * kLanes + lane;
                float hr = h[0], lr = l[0], hi = h[kLanes], li = l[kLanes];
                two_sum(hr, lr, v.x);
                two_sum(hi, li, v.y);
                h[0] = hr;
                l[0] = lr;
                h[kLanes] = hi;
                l[kLanes] = li;
                pp[t] = 0ull;
            }
        }
        __syncwarp();
        if (lane == 0 && i + S < mine) issue_block<K, OTF>(r, s, it, p, warp + (i + S) * nwarps);
        if (OTF && i + S < mine) {
            gen_weights<K>(r, s, it, p, warp + (i + S) * nwarps, lane);
            __syncwarp();
        }
    }
    if (!ok) {
        const int last = mine < i + S ? mine : i + S;
        for (int jj = i; jj < last; ++jj) {
            const int s = jj % S;
            if (mbar_wait_bounded(r.bars + 8u * s, (r.phase >> s) & 1u)) r.phase ^= (1u << s);
        }
        __syncwarp();
    }
    return ok;
}

// Half `sp & 1` of split item sp >> 1: the warps' sums reduced in the fixed
// warp order into part[], then the CTA that finishes second (an atomic count,
// no waiting) adds half 0 and half 1 in that order and stores Q.
template <class K>
__device__ __forceinline__ void coop_reduce_split(const ConvItem &it, const ConvParams &p, int lane, int warp,
                                                  int nwarps, const char *ring0, int warp_smem, int sums_off,
                                                  int sp, int *s_last) {
    constexpr int T = K::T;
    const int sid = sp >> 1, half = sp & 1;
    float *mine = p.part + ((size_t)sid * 2 + half) * kSplitFloats;
    for (int t = warp; t < T; t += nwarps) {
        float sr = 0.f, lr = 0.f, si = 0.f, li = 0.f;
        for (int w = 0; w < nwarps; ++w) {
            const float *red = reinterpret_cast<const float *>(ring0 + (size_t)w * warp_smem + sums_off);
            two_sum(sr, lr, red[(2 * t) * kLanes + lane]);
            lr += red[(2 * T + 2 * t) * kLanes + lane];
            two_sum(si, li, red[(2 * t + 1) * kLanes + lane]);
            li += red[(2 * T + 2 * t + 1) * kLanes + lane];
        }
        float *o = mine + (size_t)t * 4 * kLanes + lane;
        o[0] = sr;
        o[kLanes] = lr;
        o[2 * kLanes] = si;
        o[3 * kLanes] = li;
    }
    __threadfence();  // this half's sums before the count
    __syncthreads();
    if (threadIdx.x == 0) *s_last = atomicAdd(p.split_cnt + sid, 1u) == 1u;
    __syncthreads();
    if (!*s_last) return;
    __threadfence();  // the other half's sums after the count
    const float *h0 = p.part + (size_t)sid * 2 * kSplitFloats, *h1 = h0 + kSplitFloats;
    float2 *Q = p.Qh + it.fofs + ((size_t)(it.k1 * K::N + it.k2) * K::N + K::K0) * kLanes + lane;
    for (int t = warp; t < T; t += nwarps) {
        const float *a = h0 + (size_t)t * 4 * kLanes + lane, *b = h1 + (size_t)t * 4 * kLanes + lane;
        float sr = __ldcg(a), lr = __ldcg(a + kLanes), si = __ldcg(a + 2 * kLanes), li = __ldcg(a + 3 * kLanes);
        two_sum(sr, lr, __ldcg(b));
        lr += __ldcg(b + kLanes);
        two_sum(si, li, __ldcg(b + 2 * kLanes));
        li += __ldcg(b + 3 * kLanes);
        Q[t * kLanes] = make_float2(sr + lr, si + li);
    }
}

// Copies of this warp's first block of item it into stage 0 (lane 0 only),
// for any kind compiled into the kernel.
template <unsigned MASK, bool OTF>
__device__ __forceinline__ void issue_first_any(const WarpRing &r, const ConvItem &it, const ConvParams &p,
                                                int warp) {
    if ((int)it.nblocks <= warp || p.stall) return;
    switch (it.kind) {
        case 0: if (MASK & 1u) issue_block<K8, OTF>(r, 0, it, p, warp); break;
        case 1: if (MASK & 2u) issue_block<K12, OTF>(r, 0, it, p, warp); break;
        case 2: if (MASK & 4u) issue_block<K16, OTF>(r, 0, it, p, warp); break;
        case 3: if (MASK & 8u) issue_block<K24a, OTF>(r, 0, it, p, warp); break;
        case 4: if (MASK & 16u) issue_block<K24b, OTF>(r, 0, it, p, warp); break;
        case 5: if (MASK & 32u) issue_block<K32a, OTF>(r, 0, it, p, warp); break;
        case 6: if (MASK & 64u) issue_block<K32b, OTF>(r, 0, it, p, warp); break;
        case 7: if (MASK & 128u) issue_block<K48a, OTF>(r, 0, it, p, warp); break;
        case 8: if (MASK & 256u) issue_block<K48b, OTF>(r, 0, it, p, warp); break;
        case 9: if (MASK & 512u) issue_block<K48c, OTF>(r, 0, it, p, warp); break;
        default: break;
    }
}

// The weights of that first block (all lanes of the warp; conv_impl 5).
template <unsigned MASK>
__device__ __forceinline__ void gen_first_any(const WarpRing &r, const ConvItem &it, const ConvParams &p, int warp,
                                              int lane) {
    if ((int)it.nblocks <= warp || p.stall) return;
    switch (it.kind) {
        case 0: if (MASK & 1u) gen_weights<K8>(r, 0, it, p, warp, lane); break;
        case 1: if (MASK & 2u) gen_weights<K12>(r, 0, it, p, warp, lane); break;
        case 2: if (MASK & 4u) gen_weights<K16>(r, 0, it, p, warp, lane); break;
        case 3: if (MASK & 8u) gen_weights<K24a>(r, 0, it, p, warp, lane); break;
        case 4: if (MASK & 16u) gen_weights<K24b>(r, 0, it, p, warp, lane); break;
        case 5: if (MASK & 32u) gen_weights<K32a>(r, 0, it, p, warp, lane); break;
        case 6: if (MASK & 64u) gen_weights<K32b>(r, 0, it, p, warp, lane); break;
        case 7: if (MASK & 128u) gen_weights<K48a>(r, 0, it, p, warp, lane); break;
        case 8: if (MASK & 256u) gen_weights<K48b>(r, 0, it, p, warp, lane); break;
        case 9: if (MASK & 512u) gen_weights<K48c>(r, 0, it, p, warp, lane); break;
        default: break;
    }
}

// One item, then the next: once every warp has consumed its blocks, the next
// item is taken from the queue (into *s_next) and each warp issues the copies
// of its first block into its now idle ring before the CTA reduces this item's
// sums, which live outside the rings.
template <class K, unsigned MASK, bool OTF>
__device__ __forceinline__ bool coop_run_sm(WarpRing &r, const ConvItem &it, const ConvParams &p, int lane,
                                            int warp, int nwarps, char *ring0, int *abort_flag, float *sums,
                                            int sums_off, int sp, int *s_last, bool pre, int *s_next, int nitems) {
    const bool ok = coop_item_sm<K, OTF>(r, it, p, lane, warp, nwarps, sums, pre);
    if (!ok && lane == 0) {
        atomicOr(p.status, ST_TIMEOUT);
        *abort_flag = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) *s_next = *abort_flag ? nitems : (int)atomicAdd(p.counter, 1u);
    __syncthreads();
    const int nx = *s_next;
    if (nx < nitems && lane == 0) {
        // the ring was last read by generic loads; order them before the copies
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue_first_any<MASK, OTF>(r, p.items[nx], p, warp);
    }
    if (OTF && nx < nitems) {
        gen_first_any<MASK>(r, p.items[nx], p, warp, lane);
        __syncwarp();
    }
    if (!*abort_flag) {
        if (sp < 0) coop_reduce<K>(it, p, lane, warp, nwarps, ring0, p.warp_smem, sums_off);
        else coop_reduce_split<K>(it, p, lane, warp, nwarps, ring0, p.warp_smem, sums_off, sp, s_last);
    }
    __syncthreads();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    return !*abort_flag;
}

template <unsigned MASK, bool OTF = false>
__global__ void __launch_bounds__(128, 3) conv32_sums_kernel(ConvParams p) {
    extern __shared__ __align__(128) char smem[];
    __shared__ int s_item, s_abort, s_last, s_nitems;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const int ring = p.warp_smem - kSumsBytes;
    WarpRing r;
    r.base = smem + (size_t)warp * p.warp_smem;
    r.stage_bytes = ring / p.stages;
    r.bars = smem_u32(smem + (size_t)nwarps * p.warp_smem) + 8u * kMaxStages * warp;
    r.phase = 0;
    float *sums = reinterpret_cast<float *>(r.base + ring);
    if (lane == 0) {
        for (int s = 0; s < p.stages; ++s) mbar_init(r.bars + 8u * s, 1);
        fence_mbar_init();
    }
    if (threadIdx.x == 0) {
        s_abort = 0;
        // a work list built on the device (the learned path's fallback) carries its length there
        s_nitems = p.nitems_dev ? *p.nitems_dev : p.nitems;
        s_item = (int)atomicAdd(p.counter, 1u);
    }
    __syncthreads();
    const int nitems = s_nitems;
    bool pre = false;  // the first block of item s_item is already in flight
    for (;;) {
        const int idx = s_item;
        if (idx >= nitems || s_abort) break;
        const ConvItem it = p.items[idx];
        const int sp = p.split ? p.split[idx] : -1;
        bool ok = true, ran = true;
        switch (it.kind) {
            case 0: if (MASK & 1u) ok = coop_run_sm<K8, MASK, OTF>(r, it, p, lane, warp, nwarps, smem, &s_abort, sums, ring, sp, &s_last, pre, &s_item, nitems); else ran = false; break;
            case 1: if (MASK & 2u) ok = coop_run_sm<K12, MASK, OTF>(r, it, p, lane, warp, nwarps, smem, &s_abort, sums, ring, sp, &s_last, pre, &s_item, nitems); else ran = false; break;
            case 2: if (MASK & 4u) ok = coop_run_sm<K16, MASK, OTF>(r, it, p, lane, warp, nwarps, smem, &s_abort, sums, ring, sp, &s_last, pre, &s_item, nitems); else ran = false; break;
            case 3: if (MASK & 8u) ok = coop_run_sm<K24a, MASK, OTF>(r, it, p, lane, warp, nwarps, smem, &s_abort, sums, ring, sp, &s_last, pre, &s_item, nitems); else ran = false; break;
            case 4: if (MASK & 16u) ok = coop_run_sm<K24b, MASK, OTF>(r, it, p, lane, warp, nwarps, smem, &s_abort, sums, ring, sp, &s_last, pre, &s_item, nitems); else ran = false; break;
            case 5: if (MASK & 32u) ok = coop_run_sm<K32a, MASK, OTF>(r, it, p, lane, warp, nwarps, smem, &s_abort, sums, ring, sp, &s_last, pre, &s_item, nitems); else ran = false; break;
            case 6: if (MASK & 64u) ok = coop_run_sm<K32b, MASK, OTF>(r, it, p, lane, warp, nwarps, smem, &s_abort, sums, ring, sp, &s_last, pre, &s_item, nitems); else ran = false; break;
            case 7: if (MASK & 128u) ok = coop_run_sm<K48a, MASK, OTF>(r, it, p, lane, warp, nwarps, smem, &s_abort, sums, ring, sp, &s_last, pre, &s_item, nitems); else ran = false; break;
            case 8: if (MASK & 256u) ok = coop_run_sm<K48b, MASK, OTF>(r, it, p, lane, warp, nwarps, smem, &s_abort, sums, ring, sp, &s_last, pre, &s_item, nitems); else ran = false; break;
            case 9: if (MASK & 512u) ok = coop_run_sm<K48c, MASK, OTF>(r, it, p, lane, warp, nwarps, smem, &s_abort, sums, ring, sp, &s_last, pre, &s_item, nitems); else ran = false; break;
            default: ran = false; break;
        }
        if (!ok) break;
        if (!ran) {  // a kind this kernel was not built for: flag it, take the next item
            __syncthreads();
            if (threadIdx.x == 0) {
                atomicOr(p.status, ST_BADDESC);
                s_item = (int)atomicAdd(p.counter, 1u);
            }
            __syncthreads();
            pre = false;
            continue;
        }
        pre = true;  // coop_run_sm took the next item and issued its first copies
    }
}

template <unsigned MASK, bool PACKED, int MINB = 3>
__global__ void __launch_bounds__(128, MINB) conv32_coop_kernel(ConvParams p) {
    extern __shared__ __align__(128) char smem[];
    __shared__ int s_item, s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    WarpRing r;
    r.base = smem + (size_t)warp * p.warp_smem;
    r.stage_bytes = p.warp_smem / p.stages;
    r.bars = smem_u32(smem + (size_t)nwarps * p.warp_smem) + 8u * kMaxStages * warp;
    r.phase = 0;
    if (lane == 0) {
        for (int s = 0; s < p.stages; ++s) mbar_init(r.bars + 8u * s, 1);
        fence_mbar_init();
    }
    if (threadIdx.x == 0) s_abort = 0;
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(p.counter, 1u);
        __syncthreads();
        const int idx = s_item;
        if (idx >= p.nitems || s_abort) break;
        const ConvItem it = p.items[idx];
        bool ok = true;
        switch (it.kind) {
            case 0: if (MASK & 1u) ok = coop_run<K8, PACKED>(r, it, p, lane, warp, nwarps, smem, &s_abort); break;
            case 1: if (MASK & 2u) ok = coop_run<K12, PACKED>(r, it, p, lane, warp, nwarps, smem, &s_abort); break;
            case 2: if (MASK & 4u) ok = coop_run<K16, PACKED>(r, it, p, lane, warp, nwarps, smem, &s_abort); break;
            case 3: if (MASK & 8u) ok = coop_run<K24a, PACKED>(r, it, p, lane, warp, nwarps, smem, &s_abort); break;
            case 4: if (MASK & 16u) ok = coop_run<K24b, PACKED>(r, it, p, lane, warp, nwarps, smem, &s_abort); break;
            case 5: if (MASK & 32u) ok = coop_run<K32a, PACKED>(r, it, p, lane, warp, nwarps, smem, &s_abort); break;
            case 6: if (MASK & 64u) ok = coop_run<K32b, PACKED>(r, it, p, lane, warp, nwarps, smem, &s_abort); break;
            case 7: if (MASK & 128u) ok = coop_run<K48a, PACKED>(r, it, p, lane, warp, nwarps, smem, &s_abort); break;
            case 8: if (MASK & 256u) ok = coop_run<K48b, PACKED>(r, it, p, lane, warp, nwarps, smem, &s_abort); break;
            case 9: if (MASK & 512u) ok = coop_run<K48c, PACKED>(r, it, p, lane, warp, nwarps, smem, &s_abort); break;
            default: break;
        }
        if (!ok) break;
    }
}

template <class K>
constexpr int sb() { return K::stage_bytes; }

}  // namespace

}  // namespace bte
