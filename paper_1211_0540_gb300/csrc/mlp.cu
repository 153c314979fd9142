// Learned surrogate of the collision operator (an addition to the method: the
// paper has no learned part): a residual MLP trained on (f, Q(f)) pairs that
// the operator itself produces.
//   x  = s_in  * f / rho                (rho = sum f dv^3, the cell's mass)
//   h1 = GELU(W1 x + b1)                (4096 -> H)
//   h2 = h1 + GELU(W2 h1 + b2)          (H -> H, residual)
//   y  = W3 h2 + b3                     (H -> 4096)
//   Q  = rho^2 * y / s_out              (Q(f, f) is bilinear: Q(rho g) = rho^2 Q(g))
// BF16 weights and activations, FP32 accumulation (tensor-core GEMMs of
// gemm_tc.cu), FP32 master weights and AdamW state. The loss is the mean
// square error on t = s_out Q / rho^2. GELU uses the tanh form.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "gemm_tc.h"
#include "mlp.h"
#include "fpconv.cuh"
#include "project.cuh"
#include "rng.h"

namespace bte {

namespace {

constexpr int kT = 256;

__device__ __forceinline__ float gelu_grad(float x) {
    const float k0 = 0.7978845608028654f, k1 = 0.044715f;
    const float u = k0 * (x + k1 * x * x * x);
    const float t = tanhf(u);
    return 0.5f * (1.0f + t) + 0.5f * x * (1.0f - t * t) * k0 * (1.0f + 3.0f * k1 * x * x);
}

// One CTA per batch row: rho, x (bf16, optionally transposed) and the target.
// Each value is converted to FP32 once (kept in shared memory, M <= 4096) and
// rho is summed in double-float FP32: its ~1e-7 relative precision only
// scales the surrogate's input and output, whose conservation the projection
// restores exactly.
__global__ void __launch_bounds__(kT) prep_kernel(const double *__restrict__ f, const int64_t *__restrict__ off,
                                                   int B, int M, double dv3, float s_in, __nv_bfloat16 *X,
                                                   __nv_bfloat16 *Xt, int ldt, double *rho_out,
                                                   const double *__restrict__ Q, float s_out, float *T) {
    const int r = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double *fr = f + off[r];
    __shared__ float xs[4096];
    __shared__ float red[kT / 32][2];
    __shared__ double rho_s;
    Df s{0.f, 0.f};
    int j = threadIdx.x;
    for (; j + 3 * kT < M; j += 4 * kT) {  // four loads in flight per thread, summed in the same order
        double d[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) d[u] = fr[j + u * kT];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float v = fpc::narrow(d[u]);  // integer pipes, not the FP64 unit
            xs[j + u * kT] = v;
            df_add(s, v);
        }
    }
    for (; j < M; j += kT) {
        const float v = fpc::narrow(fr[j]);
        xs[j] = v;
        df_add(s, v);
    }
    s = df_warp_sum(s);
    if (lane == 0) {
        red[warp][0] = s.hi;
        red[warp][1] = s.lo;
    }
    __syncthreads();
    if (warp == 0) {
        s = lane < kT / 32 ? Df{red[lane][0], red[lane][1]} : Df{0.f, 0.f};
        s = df_warp_sum(s);
        if (lane == 0) {
            rho_s = ((double)s.hi + (double)s.lo) * dv3;
            if (rho_out) rho_out[r] = rho_s;
        }
    }
    __syncthreads();
    const double rho = rho_s;
    const float a = rho != 0.0 ? (float)((double)s_in / rho) : 0.f;  // a vacuum cell (rho = 0) gets x = 0
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        const __nv_bfloat16 x = __float2bfloat16_rn(xs[j] * a);
        X[(size_t)r * M + j] = x;
        if (Xt) Xt[(size_t)j * ldt + r] = x;
    }
    if (T) {
        const double c = (double)s_out / (rho * rho);
        const double *qr = Q + off[r];
        for (int j = threadIdx.x; j < M; j += blockDim.x) T[(size_t)r * M + j] = (float)(qr[j] * c);
    }
}

// Per cell of a uniform array: rho = sum f dv^3 and sum_j Q_j^2 / rho^4 (the
// squared norm of the cell's unscaled target Q / rho^2), FP64 in a fixed order.
__global__ void __launch_bounds__(kT) target_norm_kernel(const double *__restrict__ f, const double *__restrict__ Q,
                                                         int64_t M, double dv3, double *out) {
    const int64_t r = blockIdx.x;
    const double *fr = f + r * M, *qr = Q + r * M;
    __shared__ double sf[kT], sq[kT];
    double a = 0.0, b = 0.0;
    for (int64_t j = threadIdx.x; j < M; j += kT) {
        a += fr[j];
        b = fma(qr[j], qr[j], b);
    }
    sf[threadIdx.x] = a;
    sq[threadIdx.x] = b;
    __syncthreads();
    for (int w = kT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sf[threadIdx.x] += sf[threadIdx.x + w];
            sq[threadIdx.x] += sq[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double rho = sf[0] * dv3;
        out[r] = sq[0] / (rho * rho * rho * rho);
    }
}

// d = Y - T; loss partial per row; dY = 2 d / (B M) in bf16 (row-major and transposed) and FP32.
__global__ void __launch_bounds__(kT) loss_kernel(const float *__restrict__ Y, const float *__restrict__ T, int B,
                                                   int M, __nv_bfloat16 *dY, __nv_bfloat16 *dYt, int ldt, float *dYf,
                                                   double *loss_rows) {
    const int r = blockIdx.x;
    __shared__ double red[kT / 32];
    const float g = 2.0f / ((float)B * (float)M);
    double s = 0.0;
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        const float d = Y[(size_t)r * M + j] - T[(size_t)r * M + j];
        s += (double)d * d;
        const float gd = g * d;
        dYf[(size_t)r * M + j] = gd;
        const __nv_bfloat16 b = __float2bfloat16_rn(gd);
        dY[(size_t)r * M + j] = b;
        dYt[(size_t)j * ldt + r] = b;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kT / 32; ++w) t += red[w];
        loss_rows[r] = t;
    }
}

// dZ = (dH + dH2) * gelu'(Z): bf16 row-major (optional), bf16 transposed, FP32.
__global__ void gelu_bwd_kernel(const float *__restrict__ dH, const float *__restrict__ dH2,
                                const float *__restrict__ Z, int B, int n, __nv_bfloat16 *dZ, __nv_bfloat16 *dZt,
                                int ldt, float *dZf) {
    const int64_t total = (int64_t)B * n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / n), c = (int)(i % n);
        float d = dH[i];
        if (dH2) d += dH2[i];
        const float v = d * gelu_grad(Z[i]);
        dZf[i] = v;
        const __nv_bfloat16 b = __float2bfloat16_rn(v);
        if (dZ) dZ[i] = b;
        dZt[(size_t)c * ldt + r] = b;
    }
}

// out[c] = sum over rows of x[r][c] (fixed order).
__global__ void colsum_kernel(const float *__restrict__ x, int B, int n, float *out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    float s = 0.f;
    for (int r = 0; r < B; ++r) s += x[(size_t)r * n + c];
    out[c] = s;
}

__global__ void adamw_kernel(float *p, const float *__restrict__ g, float *m, float *v, int64_t n, float lr, float b1,
                             float b2, float eps, float wd, float bc1, float bc2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / bc1, vh = vi / bc2;
        p[i] -= lr * (mh / (sqrtf(vh) + eps) + wd * p[i]);
    }
}

// bf16 copy of an FP32 [rows][cols] matrix, optionally its transpose [cols][rows].
__global__ void cast_kernel(const float *__restrict__ w, int rows, int cols, __nv_bfloat16 *wb, __nv_bfloat16 *wt) {
    const int64_t total = (int64_t)rows * cols;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / cols), c = (int)(i % cols);
        const __nv_bfloat16 b = __float2bfloat16_rn(w[i]);
        wb[i] = b;
        if (wt) wt[(size_t)c * rows + r] = b;
    }
}

// Q = rho^2 / s_out * Y into the caller's FP64 cells.
__global__ void post_kernel(const float *__restrict__ Y, const double *__restrict__ rho,
                            const int64_t *__restrict__ off, int B, int M, float s_out, double *Q) {
    const int r = blockIdx.x;
    const double c = rho[r] * rho[r] / (double)s_out;
    for (int j = threadIdx.x; j < M; j += blockDim.x) Q[off[r] + j] = c * (double)Y[(size_t)r * M + j];
}

inline int blocks_for(int64_t n, int t) { return (int)std::min<int64_t>((n + t - 1) / t, 152 * 32); }

}  // namespace

// ---------------------------------------------------------------------------

void Mlp::free_all() {
    for (void *p : allocs) cudaFree(p);
    allocs.clear();
}

bool Mlp::alloc(void **p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    allocs.push_back(*p);
    return true;
}

uint64_t mlp_next_gen() {
    static std::atomic<uint64_t> g{0};
    return ++g;
}

bool Mlp::ensure_batch(int B) {
    const int Bp = (B + 127) / 128 * 128;
    if (Bp <= bcap) return true;
    gen = mlp_next_gen();
    for (void *p : act_allocs) cudaFree(p);
    act_allocs.clear();
    bcap = 0;
    auto A = [&](void **p, size_t bytes) {
        if (cudaMalloc(p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        act_allocs.push_back(*p);
        return cudaMemset(*p, 0, bytes) == cudaSuccess;
    };
    const size_t bm = (size_t)Bp * M, bh = (size_t)Bp * H;
    std::vector<int64_t> uni((size_t)Bp);
    for (int i = 0; i < Bp; ++i) uni[i] = (int64_t)i * M;
    bool ok = A((void **)&X, 2 * bm) && A((void **)&Xt, 2 * bm) && A((void **)&H1, 2 * bh) && A((void **)&H1t, 2 * bh) &&
              A((void **)&H2, 2 * bh) && A((void **)&H2t, 2 * bh) && A((void **)&dY, 2 * bm) &&
              A((void **)&dYt, 2 * bm) && A((void **)&dZ2, 2 * bh) && A((void **)&dZ2t, 2 * bh) &&
              A((void **)&dZ1t, 2 * bh) && A((void **)&Z1, 4 * bh) && A((void **)&Z2, 4 * bh) &&
              A((void **)&Y, 4 * bm) && A((void **)&T, 4 * bm) && A((void **)&dYf, 4 * bm) &&
              A((void **)&dH2, 4 * bh) && A((void **)&dH1, 4 * bh) && A((void **)&dZf, 4 * bh) &&
              A((void **)&rho, 8 * (size_t)Bp) && A((void **)&loss_rows, 8 * (size_t)Bp) &&
              A((void **)&rowoff, 8 * (size_t)Bp) && A((void **)&rowuni, 8 * (size_t)Bp) &&
              cudaMemcpy(rowuni, uni.data(), 8 * (size_t)Bp, cudaMemcpyHostToDevice) == cudaSuccess;
    if (ok) bcap = Bp;
    return ok;
}

Mlp::~Mlp() {
    free_all();
    for (void *p : act_allocs) cudaFree(p);
}

// Parameter layout in the flat FP32 buffer.
size_t Mlp::off_W1() const { return 0; }
size_t Mlp::off_b1() const { return (size_t)H * M; }
size_t Mlp::off_W2() const { return off_b1() + H; }
size_t Mlp::off_b2() const { return off_W2() + (size_t)H * H; }
size_t Mlp::off_W3() const { return off_b2() + H; }
size_t Mlp::off_b3() const { return off_W3() + (size_t)M * H; }
size_t Mlp::nparams() const { return off_b3() + M; }

void Mlp::refresh_bf16(cudaStream_t st) {
    cast_kernel<<<blocks_for((int64_t)H * M, kT), kT, 0, st>>>(params + off_W1(), H, M, w1, nullptr);
    cast_kernel<<<blocks_for((int64_t)H * H, kT), kT, 0, st>>>(params + off_W2(), H, H, w2, w2t);
    cast_kernel<<<blocks_for((int64_t)M * H, kT), kT, 0, st>>>(params + off_W3(), M, H, w3, w3t);
}

// Forward pass on B rows whose cells start at rowoff (device). With training
// set, also the transposed activations, the targets and the backward pass
// into grads; returns the loss sum through loss_rows.
int Mlp::run(const double *f, const double *Qt, int B, bool training, int *status, cudaStream_t st,
             const int64_t *rows) {
    if (!rows) rows = rowoff;
    const int Bp = (B + 127) / 128 * 128;
    if (training && B != Bp) {
        // the transposed activations are the K operand of the weight gradients:
        // their padding columns [B, Bp) must be zero in the current layout
        const size_t bm = (size_t)Bp * M * 2, bh = (size_t)Bp * H * 2;
        for (auto pr : {std::make_pair((void *)Xt, bm), std::make_pair((void *)dYt, bm), std::make_pair((void *)H1t, bh),
                        std::make_pair((void *)H2t, bh), std::make_pair((void *)dZ2t, bh),
                        std::make_pair((void *)dZ1t, bh)})
            if (cudaMemsetAsync(pr.first, 0, pr.second, st) != cudaSuccess) return -1;
    }
    prep_kernel<<<B, kT, 0, st>>>(f, rows, B, M, dv3, s_in, X, training ? Xt : nullptr, Bp, rho, Qt, s_out,
                                  training ? T : nullptr);
    GemmEpi g1;
    g1.bias = params + off_b1();
    g1.out_f32 = training ? Z1 : nullptr;
    g1.ld_f32 = H;
    g1.act = GEMM_ACT_GELU;
    g1.out_bf16 = H1;
    g1.ld_bf16 = H;
    g1.out_bf16_t = training ? H1t : nullptr;
    g1.ld_t = Bp;
    if (gemm_bf16(X, w1, B, H, M, g1, status, st)) return -1;
    GemmEpi g2;
    g2.bias = params + off_b2();
    g2.out_f32 = training ? Z2 : nullptr;
    g2.ld_f32 = H;
    g2.act = GEMM_ACT_GELU;
    g2.residual = H1;
    g2.ld_res = H;
    g2.out_bf16 = H2;
    g2.ld_bf16 = H;
    g2.out_bf16_t = training ? H2t : nullptr;
    g2.ld_t = Bp;
    if (gemm_bf16(H1, w2, B, H, H, g2, status, st)) return -1;
    GemmEpi g3;
    g3.bias = params + off_b3();
    g3.out_f32 = Y;
    g3.ld_f32 = M;
    if (gemm_bf16(H2, w3, B, M, H, g3, status, st)) return -1;
    if (!training) return 0;
    // backward
    loss_kernel<<<B, kT, 0, st>>>(Y, T, B, M, dY, dYt, Bp, dYf, loss_rows);
    colsum_kernel<<<(M + kT - 1) / kT, kT, 0, st>>>(dYf, B, M, grads + off_b3());
    GemmEpi gw3;  // dW3 = dY^T H2   [M x H]
    gw3.out_f32 = grads + off_W3();
    gw3.ld_f32 = H;
    if (gemm_bf16(dYt, H2t, M, H, Bp, gw3, status, st)) return -1;
    GemmEpi gh2;  // dH2 = dY W3     [B x H]
    gh2.out_f32 = dH2;
    gh2.ld_f32 = H;
    if (gemm_bf16(dY, w3t, B, H, M, gh2, status, st)) return -1;
    gelu_bwd_kernel<<<blocks_for((int64_t)B * H, kT), kT, 0, st>>>(dH2, nullptr, Z2, B, H, dZ2, dZ2t, Bp, dZf);
    colsum_kernel<<<(H + kT - 1) / kT, kT, 0, st>>>(dZf, B, H, grads + off_b2());
    GemmEpi gw2;  // dW2 = dZ2^T H1  [H x H]
    gw2.out_f32 = grads + off_W2();
    gw2.ld_f32 = H;
    if (gemm_bf16(dZ2t, H1t, H, H, Bp, gw2, status, st)) return -1;
    GemmEpi gh1;  // dH1 = dZ2 W2 (+ dH2 through the residual, added below)
    gh1.out_f32 = dH1;
    gh1.ld_f32 = H;
    if (gemm_bf16(dZ2, w2t, B, H, H, gh1, status, st)) return -1;
    gelu_bwd_kernel<<<blocks_for((int64_t)B * H, kT), kT, 0, st>>>(dH1, dH2, Z1, B, H, nullptr, dZ1t, Bp, dZf);
    colsum_kernel<<<(H + kT - 1) / kT, kT, 0, st>>>(dZf, B, H, grads + off_b1());
    GemmEpi gw1;  // dW1 = dZ1^T X   [H x M]
    gw1.out_f32 = grads + off_W1();
    gw1.ld_f32 = M;
    if (gemm_bf16(dZ1t, Xt, H, M, Bp, gw1, status, st)) return -1;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

void Mlp::adam_step(float lr, float wd, cudaStream_t st) {
    ++step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = 1.f - std::pow(b1, (float)step), bc2 = 1.f - std::pow(b2, (float)step);
    const int64_t n = (int64_t)nparams();
    adamw_kernel<<<blocks_for(n, kT), kT, 0, st>>>(params, grads, adam_m, adam_v, n, lr, b1, b2, 1e-8f, wd, bc1, bc2);
    refresh_bf16(st);
}

void launch_mlp_post(const float *Y, const double *rho, const int64_t *off, int B, int M, float s_out, double *Q,
                     cudaStream_t st) {
    post_kernel<<<B, kT, 0, st>>>(Y, rho, off, B, M, s_out, Q);
}

}  // namespace bte

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
using namespace bte;

namespace {
bte_status mlp_fail(bte_ctx *c, bte_status s, const std::string &m) {
    cudaGetLastError();
    if (c) c->err = m;
    return s;
}

bte_status need_mlp(bte_ctx *c) {
    if (!c) return BTE_EINVAL;
    if (!c->mlp) return mlp_fail(c, BTE_ESTATE, "no surrogate: call bte_mlp_init first");
    return BTE_OK;
}

// upload row offsets (cells c0 .. c0+B-1 of a uniform array, or an index list)
bool upload_rows(Mlp *m, const int64_t *host_rows, int B, cudaStream_t st) {
    return cudaMemcpyAsync(m->rowoff, host_rows, sizeof(int64_t) * B, cudaMemcpyHostToDevice, st) == cudaSuccess &&
           cudaStreamSynchronize(st) == cudaSuccess;
}
}  // namespace

extern "C" {

bte_status bte_mlp_init(bte_ctx *c, int table, int width, uint64_t seed) {
    if (!c) return BTE_EINVAL;
    if (table < 0 || table >= (int)c->tables.size()) return mlp_fail(c, BTE_EINVAL, "bte_mlp_init: unknown table");
    const Table *t = c->tables[table];
    if (t->N > 16) return mlp_fail(c, BTE_EINVAL, "bte_mlp_init: N <= 16 supported");
    if (width < 64 || width % 128 != 0) return mlp_fail(c, BTE_EINVAL, "bte_mlp_init: width must be a multiple of 128");
    cudaSetDevice(c->device);
    if (gemm_bf16_prepare() != cudaSuccess) return mlp_fail(c, BTE_ECUDA, "bte_mlp_init: GEMM set-up");
    if (c->mlp) cudaDeviceSynchronize();  // work in flight may still read the old surrogate
    delete c->mlp;
    c->mlp = nullptr;
    Mlp *m = new Mlp();
    m->gen = mlp_next_gen();
    m->table = table;
    m->N = t->N;
    m->M = t->N * t->N * t->N;
    m->H = width;
    m->dv3 = t->dv * t->dv * t->dv;
    if (m->M % 64 != 0) {
        delete m;
        return mlp_fail(c, BTE_EINVAL, "bte_mlp_init: N^3 must be a multiple of 64");
    }
    const size_t P = m->nparams();
    bool ok = m->alloc((void **)&m->params, 4 * P) && m->alloc((void **)&m->grads, 4 * P) &&
              m->alloc((void **)&m->adam_m, 4 * P) && m->alloc((void **)&m->adam_v, 4 * P) &&
              m->alloc((void **)&m->w1, 2 * (size_t)m->H * m->M) && m->alloc((void **)&m->w2, 2 * (size_t)m->H * m->H) &&
              m->alloc((void **)&m->w3, 2 * (size_t)m->M * m->H) && m->alloc((void **)&m->w2t, 2 * (size_t)m->H * m->H) &&
              m->alloc((void **)&m->w3t, 2 * (size_t)m->M * m->H);
    if (!ok) {
        delete m;
        return mlp_fail(c, BTE_ENOMEM, "bte_mlp_init: allocation");
    }
    // He-style initialisation (host, seeded), zero biases, zero Adam state
    std::vector<float> h(P, 0.0f);
    SplitMix64 rng(seed);
    auto fill = [&](size_t off, int rows, int cols, float sd) {
        for (size_t i = 0; i < (size_t)rows * cols; ++i) h[off + i] = (float)(sd * rng.normal());
    };
    fill(m->off_W1(), m->H, m->M, std::sqrt(2.0f / m->M));
    fill(m->off_W2(), m->H, m->H, std::sqrt(1.0f / m->H));
    fill(m->off_W3(), m->M, m->H, 0.5f * std::sqrt(1.0f / m->H));
    if (cudaMemcpy(m->params, h.data(), 4 * P, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->adam_m, 0, 4 * P) != cudaSuccess || cudaMemset(m->adam_v, 0, 4 * P) != cudaSuccess ||
        cudaMemset(m->grads, 0, 4 * P) != cudaSuccess) {
        delete m;
        return mlp_fail(c, BTE_ECUDA, "bte_mlp_init: upload");
    }
    m->refresh_bf16(0);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        delete m;
        return mlp_fail(c, BTE_ECUDA, "bte_mlp_init: cast");
    }
    c->mlp = m;
    return BTE_OK;
}

bte_status bte_mlp_info(const bte_ctx *c, int64_t *nparams, int *width, int *ndim, double *s_in, double *s_out) {
    if (!c || !c->mlp) return BTE_ESTATE;
    if (nparams) *nparams = (int64_t)c->mlp->nparams();
    if (width) *width = c->mlp->H;
    if (ndim) *ndim = c->mlp->M;
    if (s_in) *s_in = c->mlp->s_in;
    if (s_out) *s_out = c->mlp->s_out;
    return BTE_OK;
}

bte_status bte_mlp_set_scales(bte_ctx *c, double s_in, double s_out) {
    bte_status s = need_mlp(c);
    if (s != BTE_OK) return s;
    if (!(s_in > 0) || !(s_out > 0)) return mlp_fail(c, BTE_EINVAL, "bte_mlp_set_scales: scales must be > 0");
    c->mlp->s_in = (float)s_in;
    c->mlp->s_out = (float)s_out;
    return BTE_OK;
}

bte_status bte_mlp_fit_scales(bte_ctx *c, const double *f, const double *Q, int64_t n, double s_in, double *s_out,
                              void *stream) {
    bte_status s = need_mlp(c);
    if (s != BTE_OK) return s;
    if (!f || !Q || n < 1 || n > (1 << 30) || !(s_in > 0))
        return mlp_fail(c, BTE_EINVAL, "bte_mlp_fit_scales: bad arguments");
    cudaSetDevice(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    double *d = nullptr;
    if (cudaMalloc(&d, sizeof(double) * (size_t)n) != cudaSuccess)
        return mlp_fail(c, BTE_ENOMEM, "bte_mlp_fit_scales: scratch");
    target_norm_kernel<<<(unsigned)n, kT, 0, st>>>(f, Q, c->mlp->M, c->mlp->dv3, d);
    std::vector<double> h((size_t)n);
    cudaError_t e = cudaMemcpyAsync(h.data(), d, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    if (e != cudaSuccess) return mlp_fail(c, BTE_ECUDA, "bte_mlp_fit_scales: reduction");
    double sum = 0.0;
    for (double v : h) sum += v;  // fixed order: the same scale on every run
    const double ms = sum / ((double)n * c->mlp->M);
    if (!(ms > 0.0) || !std::isfinite(ms)) return mlp_fail(c, BTE_EINVAL, "bte_mlp_fit_scales: targets are zero or not finite");
    c->mlp->s_in = (float)s_in;
    c->mlp->s_out = (float)(1.0 / std::sqrt(ms));
    if (s_out) *s_out = c->mlp->s_out;
    return BTE_OK;
}

bte_status bte_mlp_get_params(bte_ctx *c, float *host, int64_t n) {
    bte_status s = need_mlp(c);
    if (s != BTE_OK) return s;
    if (!host || n != (int64_t)c->mlp->nparams()) return mlp_fail(c, BTE_EINVAL, "bte_mlp_get_params: size");
    cudaSetDevice(c->device);
    if (cudaMemcpy(host, c->mlp->params, 4 * (size_t)n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return mlp_fail(c, BTE_ECUDA, "bte_mlp_get_params: copy");
    return BTE_OK;
}

bte_status bte_mlp_set_params(bte_ctx *c, const float *host, int64_t n) {
    bte_status s = need_mlp(c);
    if (s != BTE_OK) return s;
    if (!host || n != (int64_t)c->mlp->nparams()) return mlp_fail(c, BTE_EINVAL, "bte_mlp_set_params: size");
    cudaSetDevice(c->device);
    if (cudaMemcpy(c->mlp->params, host, 4 * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess)
        return mlp_fail(c, BTE_ECUDA, "bte_mlp_set_params: copy");
    c->mlp->refresh_bf16(0);
    if (cudaDeviceSynchronize() != cudaSuccess) return mlp_fail(c, BTE_ECUDA, "bte_mlp_set_params: cast");
    return BTE_OK;
}

bte_status bte_mlp_grads(bte_ctx *c, const double *f, const double *Q, int64_t n, double *loss, float *host_grads,
                         void *stream) {
    bte_status s = need_mlp(c);
    if (s != BTE_OK) return s;
    Mlp *m = c->mlp;
    if (!f || !Q || n <= 0 || n > 65536) return mlp_fail(c, BTE_EINVAL, "bte_mlp_grads: bad arguments");
    cudaSetDevice(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (!m->ensure_batch((int)n)) return mlp_fail(c, BTE_ENOMEM, "bte_mlp_grads: activations");
    std::vector<int64_t> rows(n);
    for (int64_t i = 0; i < n; ++i) rows[i] = i * m->M;
    if (!upload_rows(m, rows.data(), (int)n, st)) return mlp_fail(c, BTE_ECUDA, "bte_mlp_grads: upload");
    if (m->run(f, Q, (int)n, true, c->d_status, st)) return mlp_fail(c, BTE_ECUDA, "bte_mlp_grads: launch");
    std::vector<double> lr(n);
    if (cudaMemcpyAsync(lr.data(), m->loss_rows, 8 * n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return mlp_fail(c, BTE_ECUDA, "bte_mlp_grads: readback");
    double L = 0.0;
    for (double v : lr) L += v;
    if (loss) *loss = L / ((double)n * m->M);
    if (host_grads && cudaMemcpy(host_grads, m->grads, 4 * m->nparams(), cudaMemcpyDeviceToHost) != cudaSuccess)
        return mlp_fail(c, BTE_ECUDA, "bte_mlp_grads: gradient copy");
    return BTE_OK;
}

bte_status bte_mlp_train(bte_ctx *c, const double *f, const double *Q, int64_t nsamples, int epochs, int batch,
                         double lr, double weight_decay, uint64_t seed, double *final_loss, void *stream) {
    bte_status s = need_mlp(c);
    if (s != BTE_OK) return s;
    Mlp *m = c->mlp;
    if (!f || !Q || nsamples < batch || batch < 1 || batch > 65536 || epochs < 1 || !(lr > 0))
        return mlp_fail(c, BTE_EINVAL, "bte_mlp_train: bad arguments");
    cudaSetDevice(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (!m->ensure_batch(batch)) return mlp_fail(c, BTE_ENOMEM, "bte_mlp_train: activations");
    SplitMix64 rng(seed);
    std::vector<int64_t> perm(nsamples), rows(nsamples);
    for (int64_t i = 0; i < nsamples; ++i) perm[i] = i;
    const int64_t steps_per_epoch = nsamples / batch;
    const int64_t total = steps_per_epoch * epochs;
    int64_t k = 0;
    double last = 0.0;
    std::vector<double> lr_rows(batch);
    int64_t *d_rows = nullptr;
    if (cudaMalloc(&d_rows, sizeof(int64_t) * nsamples) != cudaSuccess)
        return mlp_fail(c, BTE_ENOMEM, "bte_mlp_train: row table");
    struct Free {
        int64_t *p;
        ~Free() { cudaFree(p); }
    } free_rows{d_rows};
    for (int e = 0; e < epochs; ++e) {
        rng.shuffle(perm);
        for (int64_t i = 0; i < nsamples; ++i) rows[i] = perm[i] * m->M;
        // one upload per epoch; the stream orders it after the previous epoch's steps
        if (cudaMemcpyAsync(d_rows, rows.data(), sizeof(int64_t) * nsamples, cudaMemcpyHostToDevice, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return mlp_fail(c, BTE_ECUDA, "bte_mlp_train: upload");
        double esum = 0.0;
        for (int64_t b = 0; b < steps_per_epoch; ++b, ++k) {
            if (m->run(f, Q, batch, true, c->d_status, st, d_rows + b * batch))
                return mlp_fail(c, BTE_ECUDA, "bte_mlp_train: launch");
            // cosine decay to lr / 20
            const double frac = (double)k / (double)std::max<int64_t>(total - 1, 1);
            const double lrk = lr * (0.05 + 0.95 * 0.5 * (1.0 + std::cos(3.14159265358979 * frac)));
            m->adam_step((float)lrk, (float)weight_decay, st);
            if (b == steps_per_epoch - 1) {
                if (cudaMemcpyAsync(lr_rows.data(), m->loss_rows, 8 * batch, cudaMemcpyDeviceToHost, st) !=
                        cudaSuccess ||
                    cudaStreamSynchronize(st) != cudaSuccess)
                    return mlp_fail(c, BTE_ECUDA, "bte_mlp_train: readback");
                for (double v : lr_rows) esum += v;
                last = esum / ((double)batch * m->M);
            }
        }
    }
    if (cudaGetLastError() != cudaSuccess) return mlp_fail(c, BTE_ECUDA, "bte_mlp_train: kernel launch");
    if (final_loss) *final_loss = last;
    return BTE_OK;
}

bte_status bte_mlp_infer(bte_ctx *c, const double *f, double *Q, int64_t n, void *stream) {
    bte_status s = need_mlp(c);
    if (s != BTE_OK) return s;
    Mlp *m = c->mlp;
    if (!f || !Q || n <= 0 || n > 65536) return mlp_fail(c, BTE_EINVAL, "bte_mlp_infer: bad arguments");
    cudaSetDevice(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (!m->ensure_batch((int)n)) return mlp_fail(c, BTE_ENOMEM, "bte_mlp_infer: activations");
    std::vector<int64_t> rows(n);
    for (int64_t i = 0; i < n; ++i) rows[i] = i * m->M;
    if (!upload_rows(m, rows.data(), (int)n, st)) return mlp_fail(c, BTE_ECUDA, "bte_mlp_infer: upload");
    if (m->run(f, nullptr, (int)n, false, c->d_status, st)) return mlp_fail(c, BTE_ECUDA, "bte_mlp_infer: launch");
    launch_mlp_post(m->Y, m->rho, m->rowoff, (int)n, m->M, m->s_out, Q, st);
    if (cudaGetLastError() != cudaSuccess) return mlp_fail(c, BTE_ECUDA, "bte_mlp_infer: launch");
    return BTE_OK;
}

bte_status bte_tc_gemm(bte_ctx *c, const void *A, const void *B, float *D, int M, int N, int K, const float *bias,
                       int gelu, void *D_bf16, void *D_bf16_t, int ld_t, void *stream) {
    if (!c || !A || !B) return BTE_EINVAL;
    cudaSetDevice(c->device);
    cudaError_t e = gemm_bf16_prepare();
    if (e != cudaSuccess) return mlp_fail(c, BTE_ECUDA, std::string("gemm prepare: ") + cudaGetErrorString(e));
    GemmEpi g;
    g.bias = bias;
    g.out_f32 = D;
    g.ld_f32 = N;
    g.act = gelu ? GEMM_ACT_GELU : GEMM_ACT_NONE;
    g.out_bf16 = (__nv_bfloat16 *)D_bf16;
    g.ld_bf16 = N;
    g.out_bf16_t = (__nv_bfloat16 *)D_bf16_t;
    g.ld_t = ld_t;
    if (D_bf16_t && ld_t < M) return mlp_fail(c, BTE_EINVAL, "bte_tc_gemm: ld_t < M");
    int r = gemm_bf16(A, B, M, N, K, g, c->d_status, (cudaStream_t)stream);
    if (r == -1) return mlp_fail(c, BTE_EINVAL, "bte_tc_gemm: need K % 64 == 0 and N % 64 == 0");
    if (r == -2) return mlp_fail(c, BTE_ECUDA, "bte_tc_gemm: tensor map encoding failed");
    if (r != 0) return mlp_fail(c, BTE_ECUDA, "bte_tc_gemm: launch failed");
    return BTE_OK;
}

}  // extern "C"
