// BF16 GEMM on the 5th-generation tensor cores (sm_103a):
//   D[M, N] = A[M, K] . B[N, K]^T  (A, B row-major with K contiguous, bf16; FP32 accumulate)
// followed by a fused epilogue (bias, GELU, residual, FP32 / BF16 / transposed BF16 stores).
// Used by the learned surrogate (forward and backward passes of its MLP).
//
// Structure of one CTA (4 warps, one 128 x BN output tile, BN = 64, 128 or 256):
// - thread 0 (producer) streams 128 x 64 tiles of A and BN x 64 tiles of B with
//   TMA (cp.async.bulk.tensor.2d, 128-byte swizzle) into a STAGES-deep ring
//   (4, or 6-8 when the grid fits in one wave),
//   signalling a "full" mbarrier with the transaction byte count;
// - thread 32 (MMA issuer) waits for a full stage, issues four
//   tcgen05.mma.kind::f16 (K = 16 each) into the TMEM accumulator (128 lanes x
//   BN FP32 columns) and commits the stage's "empty" barrier, then the "done"
//   barrier after the last k tile;
// - all four warps read their 32 TMEM lanes (rows) with tcgen05.ld and apply
//   the epilogue.
// Every mbarrier wait is bounded by the global timer (1 s); after a timeout
// the CTA sets the status word, skips the remaining waits and still frees its
// TMEM before leaving.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <mutex>

#include "kernels.h"
#include "gemm_tc.h"

namespace bte {

namespace {

constexpr int BM = 128, BK = 64;
constexpr unsigned long long kWaitNs = 1000000000ull;

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; after the first timeout in the CTA (*abort set) waits are skipped.
__device__ __forceinline__ void wait_bounded(uint32_t bar, uint32_t parity, volatile int *abort, int *status) {
    if (*abort) return;
    if (try_wait(bar, parity)) return;
    const unsigned long long t0 = gtimer();
    while (!try_wait(bar, parity)) {
        if (*abort) return;
        if (gtimer() - t0 > kWaitNs) {
            *abort = 1;
            atomicOr(status, ST_TIMEOUT);
            return;
        }
    }
}

__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    // sm_100 shared-memory matrix descriptor: K-major, 128-byte swizzle,
    // 8-row core-matrix groups 1024 bytes apart (SBO), version 1.
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);           // start address
    d |= (uint64_t)0 << 16;                           // leading byte offset (unused, swizzled K-major)
    d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;    // stride byte offset
    d |= (uint64_t)1 << 46;                           // descriptor version
    d |= (uint64_t)2 << 61;                           // SWIZZLE_128B
    return d;
}

// Instruction descriptor: D = F32, A = B = BF16, both K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float gelu_f(float x) {
    const float k0 = 0.7978845608028654f, k1 = 0.044715f;  // sqrt(2/pi), cubic coefficient
    return 0.5f * x * (1.0f + tanhf(k0 * (x + k1 * x * x * x)));
}

// STAGES: depth of the TMA ring. With one CTA per SM the ring is what keeps
// the copies in flight against the L2 latency, so a grid that fits in one
// wave takes the deepest ring that fits (192 KB). KB: 64-wide K boxes per
// stage and operand (a k-step of KB * 64).
template <int BN, int STAGES, int KB = 1>
__global__ void __launch_bounds__(128, 1)
gemm_bf16_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, GemmEpi g,
                    int M, int N, int K, int *status) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[STAGES], bar_empty[STAGES], bar_done;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag, n_issued, n_consumed;
    // 1024-byte alignment for the 128-byte swizzle atoms
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    // a stage holds KB boxes of 64 K values for each operand (one k-step: KB * 64)
    constexpr int A_BOX = BM * BK * 2, B_BOX = BN * BK * 2, A_BYTES = KB * A_BOX, B_BYTES = KB * B_BOX;
    uint8_t *sA = base;
    uint8_t *sB = base + STAGES * A_BYTES;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile_n = blockIdx.x * BN, tile_m = blockIdx.y * BM;
    const int nk = K / (BK * KB);

    if (threadIdx.x == 0) {
        abort_flag = 0;
        n_issued = 0;
        n_consumed = 0;
        for (int s = 0; s < STAGES; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar_full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar_empty[s])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar_done)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                     "r"((uint32_t)BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    volatile int *abort = &abort_flag;

    if (threadIdx.x == 0) {
        // TMA producer
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % STAGES;
            if (kt >= STAGES) wait_bounded(su32(&bar_empty[s]), ((kt / STAGES) - 1) & 1, abort, status);
            if (*abort) break;
            const uint32_t fb = su32(&bar_full[s]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                         "r"((uint32_t)(A_BYTES + B_BYTES))
                         : "memory");
#pragma unroll
            for (int kb = 0; kb < KB; ++kb) {
                const int kc = (kt * KB + kb) * BK;
                asm volatile(
                    "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
                        "r"(su32(sA + s * A_BYTES + kb * A_BOX)),
                    "l"((uint64_t)&tmA), "r"(kc), "r"(tile_m), "r"(fb)
                    : "memory");
                asm volatile(
                    "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
                        "r"(su32(sB + s * B_BYTES + kb * B_BOX)),
                    "l"((uint64_t)&tmB), "r"(kc), "r"(tile_n), "r"(fb)
                    : "memory");
            }
            n_issued = kt + 1;
        }
    } else if (threadIdx.x == 32) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_bf16(BM, BN);
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % STAGES;
            wait_bounded(su32(&bar_full[s]), (kt / STAGES) & 1, abort, status);
            if (*abort) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = su32(sA + s * A_BYTES), b0 = su32(sB + s * B_BYTES);
#pragma unroll
            for (int kq = 0; kq < KB * (BK / 16); ++kq) {
                const int kb = kq / (BK / 16), kk = kq % (BK / 16);
                const uint64_t ad = smem_desc_sw128(a0 + kb * A_BOX + kk * 32);
                const uint64_t bd = smem_desc_sw128(b0 + kb * B_BOX + kk * 32);
                const uint32_t acc = (kt > 0 || kq > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             su32(&bar_empty[s]))
                         : "memory");
            n_consumed = kt + 1;
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         su32(&bar_done))
                     : "memory");
    }
    __syncwarp();
    // epilogue: warp w owns TMEM lanes (rows) 32w .. 32w + 31
    wait_bounded(su32(&bar_done), 0, abort, status);
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int row = tile_m + warp * 32 + lane;
    const bool rok = row < M && !*abort;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t r[16];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (!rok) continue;
        const int col0 = tile_n + c0;
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]) * g.alpha;
        if (g.bias)
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] += g.bias[col0 + i];
        if (g.out_f32) {
            float4 *o = reinterpret_cast<float4 *>(g.out_f32 + (size_t)row * g.ld_f32 + col0);
#pragma unroll
            for (int i = 0; i < 4; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        }
        if (g.act == GEMM_ACT_GELU)
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = gelu_f(v[i]);
        if (g.residual) {
            const __nv_bfloat16 *rs = g.residual + (size_t)row * g.ld_res + col0;
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] += __bfloat162float(rs[i]);
        }
        if (g.out_bf16) {
            __nv_bfloat162 pk[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) pk[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
            uint4 *o = reinterpret_cast<uint4 *>(g.out_bf16 + (size_t)row * g.ld_bf16 + col0);
            o[0] = *reinterpret_cast<uint4 *>(&pk[0]);
            o[1] = *reinterpret_cast<uint4 *>(&pk[4]);
        }
        if (g.out_bf16_t) {  // transposed copy [N][ld_t]: consecutive lanes write consecutive rows
#pragma unroll
            for (int i = 0; i < 16; ++i) g.out_bf16_t[(size_t)(col0 + i) * g.ld_t + row] = __float2bfloat16_rn(v[i]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && abort_flag) {
        // after a timeout: wait (bounded, once more) for copies still in flight
        for (int kt = n_consumed; kt < n_issued; ++kt) {
            const uint32_t fb = su32(&bar_full[kt % STAGES]);
            const unsigned long long t0 = gtimer();
            while (!try_wait(fb, (kt / STAGES) & 1) && gtimer() - t0 < kWaitNs) {
            }
        }
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN)
                     : "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        else
            cudaGetLastError();
    });
    return fn;
}

// 2-D bf16 tensor [rows][cols] (cols contiguous) with a box of box_rows x 64.
bool make_map(CUtensorMap *m, const void *ptr, int rows, int cols, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t gstride[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), gdim, gstride, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int BN, int STAGES, int KB = 1>
size_t smem_bytes() {
    return (size_t)STAGES * KB * (BM * BK * 2 + BN * BK * 2) + 1024;
}

template <int BN, int STAGES, int KB = 1>
cudaError_t set_smem() {
    return cudaFuncSetAttribute(gemm_bf16_tc_kernel<BN, STAGES, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_bytes<BN, STAGES, KB>());
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            n = 1;
    }
    return n;
}

}  // namespace

cudaError_t gemm_bf16_prepare() {
    cudaError_t e = set_smem<256, 4>();
    if (e == cudaSuccess) e = set_smem<128, 4>();
    if (e == cudaSuccess) e = set_smem<128, 6>();
    if (e == cudaSuccess) e = set_smem<64, 4>();
    if (e == cudaSuccess) e = set_smem<64, 8>();
    if (e == cudaSuccess) e = set_smem<64, 4, 2>();
    sm_count();
    return e;
}

// D[M, N] = alpha * A[M, K] B[N, K]^T (+ epilogue). Requirements (checked):
// K % 64 == 0, N % 64 == 0, 16-byte aligned rows (K % 8 == 0). M is free (TMA
// fills rows beyond M with zeros; the epilogue skips them).
int gemm_bf16(const void *A, const void *B, int M, int N, int K, const GemmEpi &g, int *status, cudaStream_t st) {
    if (M <= 0 || N <= 0 || K <= 0 || K % BK != 0 || N % 64 != 0) return -1;
    // tile width: 256 when a 256-wide grid still fills about two thirds of the
    // SMs in one wave (fewer re-reads of A), else 128 with at least a wave of
    // tiles, else 64
    const long mt = (M + BM - 1) / BM;
    const int BN = (N % 256 == 0 && mt * (N / 256) >= 2 * sm_count() / 3 && mt * (N / 256) <= sm_count()) ? 256
                   : (N % 128 == 0 && mt * (N / 128) >= 148) ? 128
                                                              : 64;
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, M, K, BM) || !make_map(&mb, B, N, K, BN)) return -2;
    dim3 grid(N / BN, (M + BM - 1) / BM);
    const bool deep = (long)grid.x * grid.y <= sm_count() && K / BK > 4;  // one wave: the deep ring
    if (BN == 256) {
        gemm_bf16_tc_kernel<256, 4><<<grid, 128, smem_bytes<256, 4>(), st>>>(ma, mb, g, M, N, K, status);
    } else if (BN == 128) {
        if (deep) gemm_bf16_tc_kernel<128, 6><<<grid, 128, smem_bytes<128, 6>(), st>>>(ma, mb, g, M, N, K, status);
        else gemm_bf16_tc_kernel<128, 4><<<grid, 128, smem_bytes<128, 4>(), st>>>(ma, mb, g, M, N, K, status);
    } else {
        // long K: stages of two 64-wide K boxes (4 of them), half the k-steps (each
        // step's round trip through the ring costs more than its bytes there)
        if (deep && K % (2 * BK) == 0 && K / BK >= 32)
            gemm_bf16_tc_kernel<64, 4, 2><<<grid, 128, smem_bytes<64, 4, 2>(), st>>>(ma, mb, g, M, N, K, status);
        else if (deep) gemm_bf16_tc_kernel<64, 8><<<grid, 128, smem_bytes<64, 8>(), st>>>(ma, mb, g, M, N, K, status);
        else gemm_bf16_tc_kernel<64, 4><<<grid, 128, smem_bytes<64, 4>(), st>>>(ma, mb, g, M, N, K, status);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace bte
