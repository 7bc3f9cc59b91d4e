// Launchers of the tensor-memory kernel that also writes the Haar side output z = Psi_m x
// (tmem.cuh with HZ): m = 15, 16, dyadic order, every butterfly variant.
#include "tmem_launch.cuh"

namespace chw {

namespace {

template <int M>
TmemLaunchFn tmem_hz_variant(int var) {
  switch (var) {
    case kVarPerLevel: return &launch_tmem_kernel<M, BfF32PerLevel, false, 0, 0, true>;
    case kVarEnd: return &launch_tmem_kernel<M, BfF32Plain, true, 0, 0, true>;
    case kVarPlain: return &launch_tmem_kernel<M, BfF32Plain, false, 0, 0, true>;
    case kVarI32: return &launch_tmem_kernel<M, BfI32, false, 0, 0, true>;
    default: return nullptr;
  }
}

}  // namespace

TmemLaunchFn lookup_tmem_hz(int m, int var) {
  if (m == 15) return tmem_hz_variant<15>(var);
  if (m == 16) return tmem_hz_variant<16>(var);
  return nullptr;
}

}  // namespace chw
