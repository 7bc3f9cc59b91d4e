// Instantiations of the fused 16-bit kernels and their lookup.
#include "lowp.cuh"

namespace chw {

using LowpLaunchFn = cudaError_t (*)(const CUtensorMap*, const CUtensorMap*, const LowpArgs&, int64_t, cudaStream_t);

// m in {11, 12}; f16 selects fp16 (else bf16); end selects one 2^{-m/2} multiply (else per
// level).  2^12: one warp per signal (lowp_warp_kernel); 2^11: two warps per signal.
LowpLaunchFn lookup_lowp(int m, bool f16, bool end) {
  if (m == 12) {
    if (f16) return end ? &launch_lowp_warp<true, BfF32Plain, true> : &launch_lowp_warp<true, BfF32PerLevel, false>;
    return end ? &launch_lowp_warp<false, BfF32Plain, true> : &launch_lowp_warp<false, BfF32PerLevel, false>;
  }
  if (m == 11) {
    if (f16) return end ? &launch_lowp<11, true, BfF32Plain, true> : &launch_lowp<11, true, BfF32PerLevel, false>;
    return end ? &launch_lowp<11, false, BfF32Plain, true> : &launch_lowp<11, false, BfF32PerLevel, false>;
  }
  return nullptr;
}

}  // namespace chw
