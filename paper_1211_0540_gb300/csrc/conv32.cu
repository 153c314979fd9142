// Host-side configuration and launch of the FP32 weighted convolution
// (Sec. 3.2; the kernels and their design are in conv32_device.cuh).
#include <map>
#include <mutex>
#include <tuple>

#include "conv32_device.cuh"

namespace bte {

// conv32_wide.cu: the variant-4/5 kernels whose kind sets include N = 48
void (*conv32_sums_wide(unsigned mask, bool otf))(ConvParams);
void (*conv32_coop_wide())(ConvParams);  // variant 3, N = 48 alone

int conv_stage_bytes(int kind) {
    switch (kind) {
        case 0: return sb<K8>();
        case 1: return sb<K12>();
        case 2: return sb<K16>();
        case 3: return sb<K24a>();
        case 4: return sb<K24b>();
        case 5: return sb<K32a>();
        case 6: return sb<K32b>();
        case 7: return sb<K48a>();
        case 8: return sb<K48b>();
        case 9: return sb<K48c>();
        default: return 0;
    }
}

namespace {
std::recursive_mutex g_conv_cfg_mu;  // guards the caches below (contexts on several host threads)
}  // namespace

cudaError_t conv32_configure(unsigned kinds_mask, int num_sms, int warps_per_cta, int stages, int impl,
                             ConvLaunch *out) {
    std::lock_guard<std::recursive_mutex> lock(g_conv_cfg_mu);
    // keyed by device too: the shared-memory attribute is set per device
    static std::map<std::tuple<int, unsigned, int, int, int, int>, ConvLaunch> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    auto key = std::make_tuple(dev, kinds_mask, num_sms, warps_per_cta, stages, impl);
    auto itc = cache.find(key);
    if (itc != cache.end()) {
        *out = itc->second;
        return cudaSuccess;
    }
    if (stages < 1) {
        // automatic depth: the deepest ring (up to 2 blocks in flight per warp)
        // that keeps the CTAs per SM of a single-stage ring. At N = 32 a second
        // stage of 8 KB rows would cost a resident CTA, which the block-level
        // latency hiding does not buy back.
        ConvLaunch a{}, b{};
        cudaError_t e1 = conv32_configure(kinds_mask, num_sms, warps_per_cta, 1, impl, &a);
        if (e1 != cudaSuccess) return e1;
        e1 = conv32_configure(kinds_mask, num_sms, warps_per_cta, 2, impl, &b);
        if (e1 != cudaSuccess) return e1;
        *out = b.grid >= a.grid ? b : a;
        cache[key] = *out;
        return cudaSuccess;
    }
    ConvLaunch L{};
    int stage = 0;
    for (int k = 0; k < kNumKinds; ++k)
        if (kinds_mask & (1u << k)) stage = stage > conv_stage_bytes(k) ? stage : conv_stage_bytes(k);
    L.stages = stages > kMaxStages ? kMaxStages : stages;
    L.warp_smem = stage * L.stages + (impl >= 4 ? kSumsBytes : 0);
    const int max_smem = 227 * 1024;
    const int max_warps = impl == 0 ? 8 : 4;
    int warps = warps_per_cta < 1 ? 1 : (warps_per_cta > max_warps ? max_warps : warps_per_cta);
    while (warps > 1 && warps * (L.warp_smem + 8 * kMaxStages) > max_smem) --warps;
    L.threads = warps * 32;
    L.smem = (size_t)warps * (L.warp_smem + 8 * kMaxStages);
    if (impl == 0) {
        switch (kinds_mask) {
            case 1u: L.fn = conv32_kernel<1u>; break;
            case 2u: L.fn = conv32_kernel<2u>; break;
            case 4u: L.fn = conv32_kernel<4u>; break;
            case 8u | 16u: L.fn = conv32_kernel<24u>; break;
            case 32u | 64u: L.fn = conv32_kernel<96u>; break;
            default: L.fn = conv32_kernel<127u>; break;  // N = 48 runs on variants 4 and 5 only
        }
    } else {
        const bool packed = impl >= 2;
#define BTE_PICK(M)                                                                             \
    L.fn = impl == 5   ? conv32_sums_kernel<M, true>                                           \
           : impl == 4 ? conv32_sums_kernel<M>                                                 \
           : impl == 3 ? conv32_coop_kernel<M, true, 2>                                        \
                       : (packed ? conv32_coop_kernel<M, true> : conv32_coop_kernel<M, false>)
#define BTE_PICK4(M) L.fn = conv32_sums_wide(M, impl == 5)
        // N = 48: variants 4 and 5, and 3 for the N = 48 kinds alone
        if (impl < 4 && (kinds_mask >> 7) && !(impl == 3 && kinds_mask == (128u | 256u | 512u)))
            return cudaErrorInvalidValue;
        switch (kinds_mask) {
            case 1u: BTE_PICK(1u); break;
            case 2u: BTE_PICK(2u); break;
            case 4u: BTE_PICK(4u); break;
            case 8u | 16u: BTE_PICK(24u); break;
            case 32u | 64u: BTE_PICK(96u); break;
            case 128u | 256u | 512u:
                if (impl == 3) L.fn = conv32_coop_wide();
                else BTE_PICK4(896u);
                break;
            default:
                if (kinds_mask >> 7) BTE_PICK4(1023u);
                else BTE_PICK(127u);
                break;
        }
#undef BTE_PICK4
#undef BTE_PICK
    }
    // the attribute belongs to the function and is shared by every cached
    // configuration of it: only ever raise it
    static std::map<std::pair<int, void *>, size_t> fn_smem;
    size_t &cur = fn_smem[std::make_pair(dev, (void *)L.fn)];
    if (L.smem > cur) {
        cudaError_t e0 = cudaFuncSetAttribute(L.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
        if (e0 != cudaSuccess) return e0;
        cur = L.smem;
    }
    cudaError_t e = cudaSuccess;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, L.fn, L.threads, L.smem);
    if (e != cudaSuccess) return e;
    L.grid = num_sms * (per_sm < 1 ? 1 : per_sm);
    L.impl = impl;
    cache[key] = L;
    *out = L;
    return cudaSuccess;
}

cudaError_t conv32_launch(const ConvLaunch &L, const ConvParams &p0, cudaStream_t st) {
    ConvParams p = p0;
    p.stages = L.stages;
    p.warp_smem = L.warp_smem;
    if (p.merge < 1) p.merge = 1;
    const int per_cta = L.impl == 0 ? L.threads / 32 : 1;  // items in flight per CTA
    int grid = L.grid;
    if ((int64_t)grid * per_cta > p.nitems) grid = (p.nitems + per_cta - 1) / per_cta;
    if (grid < 1) grid = 1;
    L.fn<<<grid, L.threads, L.smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace bte
