// bte_transfer: a copy between a host buffer and device memory, stream-ordered
// (see include/bte.h). Where the host buffer is reachable from the device
// (page-locked memory, mapped on a system with unified addressing; on GB300
// the device reads and writes it over the chip-to-chip link), a kernel moves
// it with 16-byte accesses from every SM: many more requests in flight than a
// copy engine keeps, so more of the link's bandwidth. Otherwise, and for
// device-to-device copies, cudaMemcpyAsync.
#include <algorithm>
#include <cstdint>

#include "bte_internal.h"

namespace {

// four 16-byte loads in flight per thread before their stores (the link's
// round trip is long: requests in flight set the rate)
__global__ void copy16_kernel(const uint4 *__restrict__ src, uint4 *__restrict__ dst, size_t n) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {
        uint4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = src[i + u * stride];
#pragma unroll
        for (int u = 0; u < 4; ++u) dst[i + u * stride] = v[u];
    }
    for (; i < n; i += stride) dst[i] = src[i];
}

__global__ void copy1_kernel(const unsigned char *__restrict__ src, unsigned char *__restrict__ dst, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// The device address of a host buffer the device can reach, else null.
const void *host_device_view(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

}  // namespace

extern "C" bte_status bte_transfer(bte_ctx *c, void *dst, const void *src, size_t bytes, int kind, void *stream) {
    if (!c) return BTE_EINVAL;
    if ((!dst || !src) && bytes > 0) {
        c->err = "bte_transfer: null buffer";
        return BTE_EINVAL;
    }
    if (kind != BTE_HOST_TO_DEVICE && kind != BTE_DEVICE_TO_HOST) {
        c->err = "bte_transfer: unknown kind";
        return BTE_EINVAL;
    }
    if (bytes == 0) return BTE_OK;
    cudaSetDevice(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const void *hv = host_device_view(kind == BTE_HOST_TO_DEVICE ? src : dst);
    cudaError_t e;
    if (!hv) {
        e = cudaMemcpyAsync(dst, src, bytes,
                            kind == BTE_HOST_TO_DEVICE ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost, st);
    } else {
        const void *s = kind == BTE_HOST_TO_DEVICE ? hv : src;
        void *d = kind == BTE_HOST_TO_DEVICE ? dst : const_cast<void *>(hv);
        const int grid = 4 * (c->num_sms > 0 ? c->num_sms : 1);
        if ((reinterpret_cast<uintptr_t>(s) & 15u) == 0 && (reinterpret_cast<uintptr_t>(d) & 15u) == 0 &&
            bytes % 16 == 0) {
            // at least four vectors per thread, so that each keeps four in flight
            const size_t n = bytes / 16;
            const int g16 = (int)std::min<size_t>((size_t)grid, std::max<size_t>(1, (n + 1023) / 1024));
            copy16_kernel<<<g16, 256, 0, st>>>(static_cast<const uint4 *>(s), static_cast<uint4 *>(d), n);
        } else {
            copy1_kernel<<<grid, 256, 0, st>>>(static_cast<const unsigned char *>(s), static_cast<unsigned char *>(d),
                                               bytes);
        }
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            if (c->capturing) c->cap_launches += 1;
            else c->launches += 1;
        }
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->err = std::string("bte_transfer: ") + cudaGetErrorString(e);
        return BTE_ECUDA;
    }
    return BTE_OK;
}
