// Launchers of the tensor-memory kernel for signals spread over a cluster of SMs (tmem.cuh
// with XP = 1): m = 17 on two SMs, dyadic order, every butterfly variant.
#include "tmem_launch.cuh"

namespace chw {

namespace {

template <int XP>
TmemLaunchFn cross_variant(int var) {
  switch (var) {
    case kVarPerLevel: return &launch_tmem_kernel<16, BfF32PerLevel, false, 0, 0, false, XP>;
    case kVarEnd: return &launch_tmem_kernel<16, BfF32Plain, true, 0, 0, false, XP>;
    case kVarPlain: return &launch_tmem_kernel<16, BfF32Plain, false, 0, 0, false, XP>;
    case kVarI32: return &launch_tmem_kernel<16, BfI32, false, 0, 0, false, XP>;
    default: return nullptr;
  }
}

}  // namespace

TmemLaunchFn lookup_tmem_cross(int m, int var) {
  if (m == 17) return cross_variant<1>(var);
  return nullptr;
}

}  // namespace chw
