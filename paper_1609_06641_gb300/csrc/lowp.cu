// Instantiations of the fused 16-bit kernel and their lookup.
#include "lowp.cuh"

namespace chw {

using LowpLaunchFn = cudaError_t (*)(const CUtensorMap*, const LowpArgs&, int64_t, cudaStream_t);

// m in {11, 12}; f16 selects fp16 (else bf16); end selects one 2^{-m/2} multiply (else per level).
LowpLaunchFn lookup_lowp(int m, bool f16, bool end) {
#define CHW_LOWP(M_)                                                                        \
  if (m == M_) {                                                                            \
    if (f16) return end ? &launch_lowp<M_, true, BfF32Plain, true> : &launch_lowp<M_, true, BfF32PerLevel, false>; \
    return end ? &launch_lowp<M_, false, BfF32Plain, true> : &launch_lowp<M_, false, BfF32PerLevel, false>;       \
  }
  CHW_LOWP(11)
  CHW_LOWP(12)
#undef CHW_LOWP
  return nullptr;
}

}  // namespace chw
