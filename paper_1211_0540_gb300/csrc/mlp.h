// Learned surrogate state (internal).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace bte {

struct Mlp {
    int table = 0, N = 0, M = 0, H = 0;
    double dv3 = 0.0;
    float s_in = 10.0f, s_out = 1.0f;
    int64_t step = 0;
    // identity of the device buffers a captured step reads (renewed whenever
    // they are allocated anew; unique across surrogates)
    uint64_t gen = 0;
    // parameters (FP32 master + AdamW state), flat: W1 b1 W2 b2 W3 b3
    float *params = nullptr, *grads = nullptr, *adam_m = nullptr, *adam_v = nullptr;
    __nv_bfloat16 *w1 = nullptr, *w2 = nullptr, *w3 = nullptr, *w2t = nullptr, *w3t = nullptr;
    // activations for up to bcap rows (bcap a multiple of 128)
    int bcap = 0;
    __nv_bfloat16 *X = nullptr, *Xt = nullptr, *H1 = nullptr, *H1t = nullptr, *H2 = nullptr, *H2t = nullptr;
    __nv_bfloat16 *dY = nullptr, *dYt = nullptr, *dZ2 = nullptr, *dZ2t = nullptr, *dZ1t = nullptr;
    float *Z1 = nullptr, *Z2 = nullptr, *Y = nullptr, *T = nullptr, *dYf = nullptr, *dH2 = nullptr, *dH1 = nullptr,
          *dZf = nullptr;
    double *rho = nullptr, *loss_rows = nullptr;
    int64_t *rowoff = nullptr;  // row offsets of the current call (uploaded)
    int64_t *rowuni = nullptr;  // i * M for i < bcap: rows of a contiguous block of cells
    std::vector<void *> allocs, act_allocs;

    ~Mlp();
    bool alloc(void **p, size_t bytes);
    void free_all();
    bool ensure_batch(int B);
    size_t off_W1() const;
    size_t off_b1() const;
    size_t off_W2() const;
    size_t off_b2() const;
    size_t off_W3() const;
    size_t off_b3() const;
    size_t nparams() const;
    void refresh_bf16(cudaStream_t st);
    int run(const double *f, const double *Qt, int B, bool training, int *status, cudaStream_t st,
            const int64_t *rows = nullptr);
    void adam_step(float lr, float wd, cudaStream_t st);
};

uint64_t mlp_next_gen();

void launch_mlp_post(const float *Y, const double *rho, const int64_t *off, int B, int M, float s_out, double *Q,
                     cudaStream_t st);

}  // namespace bte
