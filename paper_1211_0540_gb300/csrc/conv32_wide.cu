// The FP32 convolution kernels (variants 4 and 5, conv32_device.cuh) for kind
// sets that include N = 48: the grid of N = 48 alone (kinds 7-9) and the
// mixed set of every kind (variant 3 for N = 48 alone: conv32_wide3.cu). A
// translation unit of their own: their fully unrolled N = 48 block loops are
// the slowest code of the library to compile, and here they compile in
// parallel with the rest.
#include "conv32_device.cuh"

namespace bte {

void (*conv32_sums_wide(unsigned mask, bool otf))(ConvParams) {
    if (mask == (128u | 256u | 512u)) return otf ? conv32_sums_kernel<896u, true> : conv32_sums_kernel<896u, false>;
    return otf ? conv32_sums_kernel<1023u, true> : conv32_sums_kernel<1023u, false>;
}

}  // namespace bte
