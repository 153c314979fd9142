// Variant 3 of the FP32 convolution (conv32_device.cuh: packed f32x2
// arithmetic, the compensated sums in registers, up to 255 registers at two
// CTAs per SM) for the N = 48 kinds alone (7-9): without the per-warp sums in
// shared memory four warps per CTA fit beside the 27 KB stages of N = 48. A
// translation unit of its own, compiled in parallel with the other N = 48
// kernels.
#include "conv32_device.cuh"

namespace bte {

void (*conv32_coop_wide())(ConvParams) { return conv32_coop_kernel<896u, true, 2>; }

}  // namespace bte
