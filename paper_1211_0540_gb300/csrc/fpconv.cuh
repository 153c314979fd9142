// Conversions between IEEE-754 binary32 and binary64 on the integer pipes.
//
// On this GPU a float <-> double conversion issues on the FP64 unit, about
// 1/64 of the FP32 rate, and the transforms convert every value of a cell.
// These helpers build the result from the bit fields instead (sign, biased
// exponent, fraction; binary64 bias 1023, binary32 bias 127):
//   widen:  exact for every input (binary32 is a subset of binary64);
//   narrow: round to nearest, ties to even, with gradual underflow to the
//           binary32 subnormals, overflow to infinity, NaN kept a NaN.
// Host and device: the host test compares them bit for bit with the
// compiler's conversions over special values and random bit patterns.
#pragma once

#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

namespace bte {
namespace fpc {

__host__ __device__ __forceinline__ uint32_t bits32(float x) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(x);
#else
    uint32_t u;
    std::memcpy(&u, &x, 4);
    return u;
#endif
}
__host__ __device__ __forceinline__ float from32(uint32_t u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float x;
    std::memcpy(&x, &u, 4);
    return x;
#endif
}
__host__ __device__ __forceinline__ uint64_t bits64(double x) {
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t u;
    std::memcpy(&u, &x, 8);
    return u;
#endif
}
__host__ __device__ __forceinline__ double from64(uint64_t u) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double x;
    std::memcpy(&x, &u, 8);
    return x;
#endif
}
__host__ __device__ __forceinline__ int clz32(uint32_t v) {
#ifdef __CUDA_ARCH__
    return __clz(v);
#else
    int n = 0;
    while (n < 32 && !(v & (0x80000000u >> n))) ++n;
    return n;
#endif
}

// binary32 -> binary64, exact.
__host__ __device__ __forceinline__ double widen(float x) {
    const uint32_t u = bits32(x);
    const uint64_t sign = (uint64_t)(u >> 31) << 63;
    const uint32_t e = (u >> 23) & 0xffu, f = u & 0x7fffffu;
    uint64_t r;
    if (e == 0xffu) {  // infinity, NaN
        r = sign | (0x7ffull << 52) | ((uint64_t)f << 29);
    } else if (e != 0u) {  // normal: rebias 127 -> 1023
        r = sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)f << 29);
    } else if (f == 0u) {  // signed zero
        r = sign;
    } else {  // subnormal f * 2^-149: normalise the fraction
        const int s = clz32(f) - 8;  // shifts that bring the leading 1 to bit 23
        r = sign | ((uint64_t)(897 - s) << 52) | ((uint64_t)((f << s) & 0x7fffffu) << 29);
    }
    return from64(r);
}

// binary64 -> binary32, round to nearest, ties to even.
__host__ __device__ __forceinline__ float narrow(double x) {
    const uint64_t u = bits64(x);
    const uint32_t sign = (uint32_t)(u >> 63) << 31;
    const int e = (int)((u >> 52) & 0x7ffu);
    const uint64_t f = u & 0xfffffffffffffull;
    if (e == 0x7ff) return from32(sign | 0x7f800000u | (f ? 0x400000u | (uint32_t)(f >> 29) : 0u));
    const int e32 = e - 1023 + 127;  // biased binary32 exponent of x
    if (e32 >= 255) return from32(sign | 0x7f800000u);
    // significand with the implicit bit (53 bits); shift right by 29 (normal)
    // or more (subnormal result), then round on the bits shifted out
    const uint64_t m = e ? (f | (1ull << 52)) : f;
    int shift = 29;
    uint32_t ebits = 0;
    if (e32 >= 1) {
        ebits = (uint32_t)e32 << 23;
    } else {
        shift = 29 + 1 - e32;  // subnormal binary32 (exponent field 0)
        if (shift > 54) return from32(sign);  // below half the smallest subnormal
    }
    const uint64_t kept = m >> shift;
    const uint64_t rest = m & ((1ull << shift) - 1);
    const uint64_t half = 1ull << (shift - 1);
    uint32_t r = (uint32_t)kept;
    if (e32 >= 1) r &= 0x7fffffu;  // drop the implicit bit; it lives in the exponent field
    r += ebits;
    if (rest > half || (rest == half && (kept & 1ull))) ++r;  // a carry may step the exponent
    return from32(sign | r);
}

// True when the binary64 value is finite (exponent field not all ones).
__host__ __device__ __forceinline__ bool finite64(double x) { return ((bits64(x) >> 52) & 0x7ffu) != 0x7ffu; }

}  // namespace fpc
}  // namespace bte
