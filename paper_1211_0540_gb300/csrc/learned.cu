// Learned collision path (mode BTE_LEARNED): surrogate -> conservation
// projection -> residual indicator -> exact fallback.
//
// Indicator (per cell). The exact operator is evaluated on S sampled zeta
// pencils (k1, k2) (fixed, seeded, |k1'|, |k2'| <= N/4), all N modes k3 of each:
//   Qhat(k)  = sum_m Ghat(xi_m, zeta_k) dz^3 fhat_m fhat_{k-m+N/2}     (Sec. 3.2)
//   Qhat-(k) = the same sum with the loss term of Ghat only,
// and compared with the forward transform of the projected surrogate output:
//   ind = ||Fhat[P Q_nn](k) - Qhat(k)||_S / ||Qhat-(k)||_S,
// i.e. the parity metric of the fast path restricted to S N modes. Cells with
// ind > tol are recomputed with the FP32 operator. Cost of the check: S of the
// N^2 pencils of the convolution (4 / 256 = 1.6 % at N = 16).
#include <algorithm>
#include <cmath>
#include <vector>

#include "learned.h"
#include "fpconv.cuh"
#include "project.cuh"
#include "rng.h"

namespace bte {

namespace {

// One CTA of kIndWarps warps per (sampled pencil, group), lane = cell: the
// warps work in pairs, each pair takes the pencil's kept (m1, m2) blocks in
// turn (the block layout of the FP32 table: unordered pairs, weights
// Ghat(k,m) + Ghat(k,n)) and each warp of a pair half of the N outputs k3,
// with the full and the loss weights side by side: the a and b rows of a block
// are loaded into registers by both warps of its pair. Half the outputs per
// warp keep the kernel at two CTAs per SM. Partial sums are added across the
// pairs in a fixed order, then compared with the transform of the projected
// surrogate output.
constexpr int kIndWarps = 8;
constexpr int kIndPairs = kIndWarps / 2;

// The pair sums of one block for the outputs k3 in [JH N/2, (JH + 1) N/2):
// acc = full (re, im) per output, then loss (re, im). The weight of the pair
// (m3, k3) sits at its rank among the block's valid pairs (m3 major, k3 minor),
// a compile-time index after unrolling.
template <int N, int JH>
__device__ __forceinline__ void indicator_block(const float2 (&av)[N], const float2 (&bv)[N], const float4 *wf,
                                                const float4 *wl, float (&acc)[2 * N]) {
    constexpr int H = N / 2, J0 = JH * H;
    int wi = 0;
#pragma unroll
    for (int m3 = 0; m3 < N; ++m3)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const int n3 = j - m3 + H;
            if (n3 < 0 || n3 >= N) continue;
            if (j >= J0 && j < J0 + H) {
                const float4 f4 = wf[wi >> 2], l4 = wl[wi >> 2];
                const int q = wi & 3;
                const float wF = q == 0 ? f4.x : q == 1 ? f4.y : q == 2 ? f4.z : f4.w;
                const float wL = q == 0 ? l4.x : q == 1 ? l4.y : q == 2 ? l4.z : l4.w;
                const float pr = av[m3].x * bv[n3].x - av[m3].y * bv[n3].y;
                const float pi = av[m3].x * bv[n3].y + av[m3].y * bv[n3].x;
                const int o = j - J0;
                acc[2 * o] = fmaf(wF, pr, acc[2 * o]);
                acc[2 * o + 1] = fmaf(wF, pi, acc[2 * o + 1]);
                acc[N + 2 * o] = fmaf(wL, pr, acc[N + 2 * o]);
                acc[N + 2 * o + 1] = fmaf(wL, pi, acc[N + 2 * o + 1]);
            }
            ++wi;
        }
}

// The pencil's blocks are split between two CTAs (blockIdx.z = half) so that
// the S x groups items fill the GPU; each half reduces its pairs in a fixed
// order into part[], and the half that finishes second (an atomic count, no
// waiting) adds half 0 and half 1 in that order and forms the errors.
template <int N>
__global__ void __launch_bounds__(32 * kIndWarps, 2)
indicator_kernel(const float2 *__restrict__ F, const float2 *__restrict__ QN, const float *__restrict__ Wfull,
                 const float *__restrict__ Wloss, const uint32_t *__restrict__ desc, const IndPencil *__restrict__ pens,
                 int cpad, int64_t eoff, int nslots, float *err2, float *den2, float *part, unsigned *cnt) {
    constexpr int M = N * N * N, H = N / 2;
    extern __shared__ __align__(16) float red[];  // [kIndPairs][4 N][32]
    const int p = blockIdx.x, g = blockIdx.y, half = blockIdx.z, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pair = warp >> 1, jh = warp & 1;
    const IndPencil pen = pens[p];
    const int k1 = pen.kk / N, k2 = pen.kk % N;
    const float2 *Fg = F + eoff + (int64_t)g * M * kLanes;  // fhat in the sector order of the group
    float acc[2 * N];  // this warp's outputs: full (re, im) per k3, then loss (re, im)
#pragma unroll
    for (int i = 0; i < 2 * N; ++i) acc[i] = 0.f;
    const int bmid = pen.nblocks / 2, bend = half ? pen.nblocks : bmid;
    for (int b = (half ? bmid : 0) + pair; b < bend; b += kIndPairs) {
        const uint32_t d = desc[pen.desc_off + b];
        const int m1 = (int)(d & 0xffffu), m2 = (int)(d >> 16), n1 = k1 - m1 + H, n2 = k2 - m2 + H;
        float2 av[N], bv[N];
#pragma unroll
        for (int i = 0; i < N; i += 2) {  // two modes of the lane per 16-byte load (rows start on a sector)
            const float4 a2 = *reinterpret_cast<const float4 *>(Fg + sector_index((m1 * N + m2) * N + i, lane));
            const float4 b2 = *reinterpret_cast<const float4 *>(Fg + sector_index((n1 * N + n2) * N + i, lane));
            av[i] = make_float2(a2.x, a2.y);
            av[i + 1] = make_float2(a2.z, a2.w);
            bv[i] = make_float2(b2.x, b2.y);
            bv[i + 1] = make_float2(b2.z, b2.w);
        }
        const float4 *wf = reinterpret_cast<const float4 *>(Wfull + pen.wofs_full + (size_t)b * cpad);
        const float4 *wl = reinterpret_cast<const float4 *>(Wloss + pen.wofs_loss + (size_t)b * cpad);
        if (jh == 0) indicator_block<N, 0>(av, bv, wf, wl, acc);
        else indicator_block<N, 1>(av, bv, wf, wl, acc);
    }
    // the pair's 4 N sums: full (re, im) of output k3 at 2 k3, loss at 2 N + 2 k3
#pragma unroll
    for (int o = 0; o < H; ++o) {
        const int k3 = jh * H + o;
        red[(pair * 4 * N + 2 * k3) * kLanes + lane] = acc[2 * o];
        red[(pair * 4 * N + 2 * k3 + 1) * kLanes + lane] = acc[2 * o + 1];
        red[(pair * 4 * N + 2 * N + 2 * k3) * kLanes + lane] = acc[N + 2 * o];
        red[(pair * 4 * N + 2 * N + 2 * k3 + 1) * kLanes + lane] = acc[N + 2 * o + 1];
    }
    __syncthreads();
    if (warp != 0) return;
    const size_t item = (size_t)p * gridDim.y + g;
    float *mine = part + (item * 2 + half) * (4 * N * kLanes) + lane;
    for (int i = 0; i < 4 * N; ++i) {
        float v = 0.f;
        for (int w = 0; w < kIndPairs; ++w) v += red[((size_t)w * 4 * N + i) * kLanes + lane];
        mine[i * kLanes] = v;
    }
    __threadfence();  // this half's sums before the count
    __syncwarp();
    unsigned old = 0;
    if (lane == 0) old = atomicAdd(cnt + item, 1u);
    old = __shfl_sync(0xffffffffu, old, 0);
    if (old != 1u) return;
    __threadfence();  // the other half's sums after the count
    const float *h0 = part + item * 2 * (4 * N * kLanes) + lane, *h1 = h0 + 4 * N * kLanes;
    float e = 0.f, dn = 0.f;
    const float2 *qn = QN + eoff + (int64_t)g * M * kLanes + (int64_t)pen.kk * N * kLanes + lane;
    for (int j = 0; j < N; ++j) {
        const float fr = __ldcg(h0 + (2 * j) * kLanes) + __ldcg(h1 + (2 * j) * kLanes);
        const float fi = __ldcg(h0 + (2 * j + 1) * kLanes) + __ldcg(h1 + (2 * j + 1) * kLanes);
        const float lr = __ldcg(h0 + (2 * N + 2 * j) * kLanes) + __ldcg(h1 + (2 * N + 2 * j) * kLanes);
        const float li = __ldcg(h0 + (2 * N + 2 * j + 1) * kLanes) + __ldcg(h1 + (2 * N + 2 * j + 1) * kLanes);
        const float2 q = qn[(int64_t)j * kLanes];
        const float dr = q.x - fr, di = q.y - fi;
        e += dr * dr + di * di;
        dn += lr * lr + li * li;
    }
    const int slot = g * kLanes + lane;
    err2[(size_t)p * nslots + slot] = e;
    den2[(size_t)p * nslots + slot] = dn;
}

template <int N>
constexpr size_t ind_smem() {
    return sizeof(float) * kIndPairs * 4 * N * kLanes;
}

__global__ void indicator_reduce_kernel(const float *__restrict__ err2, const float *__restrict__ den2, int S,
                                        int nslots, int nvalid, float *ind) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nslots) return;
    float e = 0.f, d = 0.f;
    for (int s = 0; s < S; ++s) {
        e += err2[(size_t)s * nslots + c];
        d += den2[(size_t)s * nslots + c];
    }
    ind[c] = c < nvalid ? sqrtf(e) / fmaxf(sqrtf(d), 1e-30f) : 0.f;
}

// Surrogate output to the caller's cells with the conservation projection of
// Sec. 3.3 fused in: Q = P_N(c Y), c = rho^2 / s_out per cell. One CTA per
// cell, one thread per pencil (j1, j2): the moments of Y are accumulated in
// double-float FP32 (the values are FP32), mu(Q) = c mu(Y) and lambda are
// formed in FP64, and Q_j = c Y_j - C_j^T lambda is written in FP64 on a
// coalesced mapping (one FP64 operation per value).
template <int N>
__global__ void __launch_bounds__((N * N + 31) / 32 * 32)
post_project_kernel(const float *__restrict__ Y, const double *__restrict__ rho, float s_out, ProjArgs pa,
                    double *__restrict__ Q) {
    constexpr int M = N * N * N, NN = N * N, H = N / 2, NT = (NN + 31) / 32 * 32, NW = NT / 32;
    const int r = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const float *y = Y + (size_t)r * M;
    double *q = Q + (size_t)r * M;
    __shared__ float red[NW][10];
    __shared__ float2 base[NN], sg[N];
    __shared__ double lam[5], c_s;
    __shared__ float2 c_hl;
    if (t == 0) {  // the output scale, once per cell (an FP64 division), and its double-float split
        const double c = rho[r] * rho[r] / (double)s_out;
        const float hi = fpc::narrow(c);
        c_s = c;
        c_hl = make_float2(hi, fpc::narrow(c - fpc::widen(hi)));
    }
    Df mom[5];
    if (t < NN) {
        Df s0{0.f, 0.f}, s1{0.f, 0.f}, s2{0.f, 0.f};
        const float *yp = y + t * N;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const float v = yp[j];
            df_add(s0, v);
            df_add_prod(s1, (float)(j - H), v);
            df_add_prod(s2, (float)((j - H) * (j - H)), v);
        }
        const int w1 = t / N - H, w2 = t % N - H;
        mom[0] = s0;
        mom[1] = df_mul_int(s0, (float)w1);
        mom[2] = df_mul_int(s0, (float)w2);
        mom[3] = s1;
        mom[4] = df_add(df_mul_int(s0, (float)(w1 * w1 + w2 * w2)), s2);
    } else {
#pragma unroll
        for (int i = 0; i < 5; ++i) mom[i] = Df{0.f, 0.f};
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) mom[i] = df_warp_sum(mom[i]);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            red[warp][2 * i] = mom[i].hi;
            red[warp][2 * i + 1] = mom[i].lo;
        }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < 5; ++i) mom[i] = lane < NW ? Df{red[lane][2 * i], red[lane][2 * i + 1]} : Df{0.f, 0.f};
#pragma unroll
        for (int i = 0; i < 5; ++i) mom[i] = df_warp_sum(mom[i]);
        double mu = 0.0;
        const double c = c_s;
#pragma unroll
        for (int i = 0; i < 5; ++i)
            if (lane == i) mu = ((double)mom[i].hi + (double)mom[i].lo) * c;
        mu *= lane == 0 ? 1.0 : (lane == 4 ? pa.dv * pa.dv : pa.dv);
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
    __syncthreads();
    // The correction C^T lambda = base(j1, j2) + g(j3) is formed in FP64 per
    // pencil and per j3, then kept as double-float pairs (hi, lo): per value
    // Q = c Y - base - g is then FP32 work (an exact TwoProduct for c Y and
    // two double-float additions, relative error ~2^-48) and one FP64
    // addition hi + lo, instead of three FP64-unit operations.
    const double dv = pa.dv;
    if (t < N) {
        const double v = dv * (double)(t - H);
        const double g = fma(lam[3], v, lam[4] * v * v);
        const float hi = fpc::narrow(g);
        sg[t] = make_float2(hi, fpc::narrow(g - fpc::widen(hi)));
    }
    if (t < NN) {
        const double v1 = dv * (double)(t / N - H), v2 = dv * (double)(t % N - H);
        const double b = lam[0] + fma(lam[1], v1, fma(lam[2], v2, lam[4] * fma(v1, v1, v2 * v2)));
        const float hi = fpc::narrow(b);
        base[t] = make_float2(hi, fpc::narrow(b - fpc::widen(hi)));
    }
    __syncthreads();
    const float c_hi = c_hl.x, c_lo = c_hl.y;
    for (int e = t; e < M; e += NT) {
        const float yv = y[e];
        const float p = c_hi * yv;
        Df prod{p, fmaf(c_lo, yv, fmaf(c_hi, yv, -p))};
        const float2 b = base[e / N], g = sg[e % N];
        const Df corr = df_add(Df{b.x, b.y}, Df{g.x, g.y});
        const Df v = df_add(prod, Df{-corr.hi, -corr.lo});
        q[e] = fpc::widen(v.hi) + fpc::widen(v.lo);
    }
}

// The fallback of the learned mode, laid out on the device (one CTA): cells
// whose indicator is not <= tol are listed in increasing order, and the FP32
// operator's batch for them is written for up to nslots_cap slots: offsets
// (redo[s] M for the listed cells, -1 for the padding lanes of the last
// 32-cell group, -2 for the groups that hold no cell: the transforms skip
// them), the convolution's work list (the one-group template repeated for the
// groups in use, all groups of the costliest pencil first), its length and a
// zeroed queue counter. The statistics (cells seen, cells recomputed, the
// largest indicator as FP32 bits) accumulate in stats. No host round trip.
constexpr int kSetupThreads = 1024;
__global__ void __launch_bounds__(kSetupThreads)
fallback_setup_kernel(const float *__restrict__ ind, int ncells, double tol, int64_t M,
                      const ConvItem *__restrict__ tmpl, int ntmpl, int nslots_cap, int64_t *__restrict__ off,
                      ConvItem *__restrict__ items, int *__restrict__ nitems, unsigned *__restrict__ counter,
                      unsigned long long *__restrict__ stats) {
    __shared__ int warp_tot[kSetupThreads / 32];
    __shared__ int s_base;
    __shared__ unsigned s_max;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) {
        s_base = 0;
        s_max = 0u;
    }
    __syncthreads();
    for (int c0 = 0; c0 < ncells; c0 += kSetupThreads) {
        const int c = c0 + t;
        const float v = c < ncells ? ind[c] : 0.f;
        const int flag = (c < ncells && !((double)v <= tol)) ? 1 : 0;
        // the largest indicator (non-negative floats order as their bit patterns; NaN is left out)
        const unsigned vmax = __reduce_max_sync(0xffffffffu, (c < ncells && v >= 0.f) ? __float_as_uint(v) : 0u);
        if (lane == 0 && vmax) atomicMax(&s_max, vmax);
        // block-wide exclusive prefix sum of the flags (in cell order)
        const unsigned bal = __ballot_sync(0xffffffffu, flag);
        const int before = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) warp_tot[warp] = __popc(bal);
        __syncthreads();
        int wbase = 0;
        for (int w = 0; w < warp; ++w) wbase += warp_tot[w];
        const int base = s_base;
        if (flag) off[base + wbase + before] = (int64_t)c * M;
        __syncthreads();
        if (t == kSetupThreads - 1) s_base = base + wbase + before + flag;
        __syncthreads();
    }
    const int nredo = s_base, ngu = (nredo + kLanes - 1) / kLanes;
    for (int sl = nredo + t; sl < nslots_cap; sl += kSetupThreads) off[sl] = sl < ngu * kLanes ? -1 : -2;
    for (int i = t; i < ngu * ntmpl; i += kSetupThreads) {
        ConvItem it = tmpl[i / ngu];
        it.fofs = (uint64_t)((int64_t)(i % ngu) * M * kLanes);
        items[i] = it;
    }
    if (t == 0) {
        *nitems = ngu * ntmpl;
        *counter = 0u;
        atomicAdd(stats + 0, (unsigned long long)ncells);
        atomicAdd(stats + 1, (unsigned long long)nredo);
        atomicMax(stats + 2, (unsigned long long)s_max);
    }
}

// y = x + a Q (mode 1) or y += a (qp + Q) (mode 2) on n values: the time update
// of a Heun stage when Q comes from the learned mode.
__global__ void stage_update_kernel(const double *__restrict__ Q, const double *__restrict__ x, double *__restrict__ y,
                                    const double *__restrict__ qp, double a, int64_t n, int mode) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = mode == 1 ? fma(a, Q[i], x[i]) : fma(a, qp[i] + Q[i], y[i]);
}

// ind (one float per slot of a uniform batch, slot = cell) to the caller's doubles.
__global__ void widen_kernel(const float *__restrict__ in, double *__restrict__ out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)in[i];
}

}  // namespace

void launch_widen(const float *in, double *out, int n, cudaStream_t st) {
    if (n > 0) widen_kernel<<<(n + 255) / 256, 256, 0, st>>>(in, out, n);
}

void launch_fallback_setup(const float *ind, int ncells, double tol, int64_t M, const ConvItem *tmpl, int ntmpl,
                           int nslots_cap, int64_t *off, ConvItem *items, int *nitems, unsigned *counter,
                           unsigned long long *stats, cudaStream_t st) {
    fallback_setup_kernel<<<1, kSetupThreads, 0, st>>>(ind, ncells, tol, M, tmpl, ntmpl, nslots_cap, off, items,
                                                        nitems, counter, stats);
}

void launch_stage_update(const double *Q, const double *x, double *y, const double *qp, double a, int64_t n,
                         int mode, cudaStream_t st) {
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    stage_update_kernel<<<(unsigned)blocks, 256, 0, st>>>(Q, x, y, qp, a, n, mode);
}

int build_indicator_table(const Table &t, int modes, uint64_t seed, IndicatorTable &out) {
    const int N = t.N, h = N / 2, q = N / 4;
    const int S = std::max(1, modes / N);
    const double dz3 = t.dz * t.dz * t.dz;
    const double c = std::sqrt(2.0 / 3.14159265358979323846);
    // SplitMix64 from `seed`; each pencil offset is (next mod (2q + 1)) - q,
    // k1' first; repeated pencils are skipped. Integer arithmetic only, so
    // every platform draws the same sample.
    SplitMix64 rng(seed);
    const uint64_t span = (uint64_t)(2 * q + 1);
    std::vector<int> kks;
    while ((int)kks.size() < S) {
        const int k1 = (int)(rng.next() % span) - q;
        const int k2 = (int)(rng.next() % span) - q;
        const int kk = (k1 + h) * N + (k2 + h);
        if (std::find(kks.begin(), kks.end(), kk) == kks.end()) kks.push_back(kk);
    }
    // loss weights of the sampled pencils in the FP32 table's block layout (one k3 tile, N <= 16)
    const int cpad = t.cpad[0];
    std::vector<float> wl;
    std::vector<IndPencil> pens;
    std::vector<uint32_t> desc(t.n_desc);
    if (cudaMemcpy(desc.data(), t.d_desc, sizeof(uint32_t) * t.n_desc, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    for (int kk : kks) {
        IndPencil pn{};
        pn.kk = kk;
        pn.desc_off = (int)t.desc_off[kk];
        pn.nblocks = (int)t.nblocks[kk];
        pn.wofs_full = t.wofs[kk];
        pn.wofs_loss = wl.size();
        const int k1 = kk / N, k2 = kk % N;
        for (int b = 0; b < pn.nblocks; ++b) {
            const uint32_t dd = desc[pn.desc_off + b];
            const int m1 = (int)(dd & 0xffffu), m2 = (int)(dd >> 16), n1 = k1 - m1 + h, n2 = k2 - m2 + h;
            const bool pair = !(m1 == n1 && m2 == n2);
            const size_t base = wl.size();
            wl.resize(base + cpad, 0.0f);
            size_t wi = base;
            for (int m3 = 0; m3 < N; ++m3)
                for (int k3 = 0; k3 < N; ++k3) {
                    const int n3 = k3 - m3 + h;
                    if (n3 < 0 || n3 >= N) continue;
                    const int sm = (m1 - h) * (m1 - h) + (m2 - h) * (m2 - h) + (m3 - h) * (m3 - h);
                    double g = -c * t.J[sm];
                    if (pair) {
                        const int sn = (n1 - h) * (n1 - h) + (n2 - h) * (n2 - h) + (n3 - h) * (n3 - h);
                        g += -c * t.J[sn];
                    }
                    wl[wi++] = (float)(g * dz3);
                }
        }
        pens.push_back(pn);
    }
    out.S = S;
    out.kks = kks;
    cudaError_t e = cudaMalloc(&out.d_wloss, sizeof(float) * std::max<size_t>(wl.size(), 4));
    if (e == cudaSuccess) e = cudaMalloc(&out.d_pen, sizeof(IndPencil) * S);
    if (e == cudaSuccess) e = cudaMemcpy(out.d_wloss, wl.data(), sizeof(float) * wl.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(out.d_pen, pens.data(), sizeof(IndPencil) * S, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&out.d_kk, sizeof(int) * S);
    if (e == cudaSuccess) e = cudaMemcpy(out.d_kk, kks.data(), sizeof(int) * S, cudaMemcpyHostToDevice);
    // shared memory of the cross-warp reduction (set outside any stream capture)
    if (e == cudaSuccess) e = cudaFuncSetAttribute(indicator_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ind_smem<8>());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(indicator_kernel<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ind_smem<12>());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(indicator_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ind_smem<16>());
    if (e != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return 0;
}

void free_indicator_table(IndicatorTable &t) {
    cudaFree(t.d_wloss);
    cudaFree(t.d_pen);
    cudaFree(t.d_kk);
    t.d_wloss = nullptr;
    t.d_pen = nullptr;
    t.d_kk = nullptr;
}

void launch_post_project(const float *Y, const double *rho, int B, int N, float s_out, const ProjArgs &pa, double *Q,
                         cudaStream_t st) {
    switch (N) {
        case 8: post_project_kernel<8><<<B, 64, 0, st>>>(Y, rho, s_out, pa, Q); break;
        case 12: post_project_kernel<12><<<B, 160, 0, st>>>(Y, rho, s_out, pa, Q); break;
        case 16: post_project_kernel<16><<<B, 256, 0, st>>>(Y, rho, s_out, pa, Q); break;
        default: break;
    }
}

size_t indicator_scratch_floats(const IndicatorTable &it, int N, int nslots) {
    const size_t items = (size_t)it.S * (nslots / kLanes);
    return 2 * (size_t)it.S * nslots + nslots + items * 2 * 4 * N * kLanes + items;
}

void launch_indicator(const IndicatorTable &it, const Table &t, const float2 *F, const float2 *QN, int64_t eoff,
                      int nslots, int nvalid, float *err2, float *den2, float *ind, cudaStream_t st) {
    dim3 grid(it.S, nslots / kLanes, 2);
    // after err2, den2 and ind: the halves' partial sums, then the per-item counts
    const size_t items = (size_t)it.S * (nslots / kLanes);
    float *part = ind + nslots;
    unsigned *cnt = reinterpret_cast<unsigned *>(part + items * 2 * 4 * t.N * kLanes);
    cudaMemsetAsync(cnt, 0, sizeof(unsigned) * items, st);
    switch (t.N) {
        case 8:
            indicator_kernel<8><<<grid, 32 * kIndWarps, ind_smem<8>(), st>>>(F, QN, t.d_w32, it.d_wloss, t.d_desc,
                                                                           it.d_pen, t.cpad[0], eoff, nslots, err2, den2, part, cnt);
            break;
        case 12:
            indicator_kernel<12><<<grid, 32 * kIndWarps, ind_smem<12>(), st>>>(F, QN, t.d_w32, it.d_wloss, t.d_desc,
                                                                             it.d_pen, t.cpad[0], eoff, nslots, err2,
                                                                             den2, part, cnt);
            break;
        default:
            indicator_kernel<16><<<grid, 32 * kIndWarps, ind_smem<16>(), st>>>(F, QN, t.d_w32, it.d_wloss, t.d_desc,
                                                                             it.d_pen, t.cpad[0], eoff, nslots, err2,
                                                                             den2, part, cnt);
            break;
    }
    indicator_reduce_kernel<<<(nslots + 255) / 256, 256, 0, st>>>(err2, den2, it.S, nslots, nvalid, ind);
}

}  // namespace bte
