// Launchers of the tensor-memory whole-signal kernel (tmem.cuh): m = 15, 16, four-byte
// elements, dyadic, natural or sequency order or the column-blocked rows of a two-pass
// split, every butterfly variant.
#include "tmem_launch.cuh"

namespace chw {

namespace {

template <int M, int OM>
TmemLaunchFn tmem_variant(int var) {
  switch (var) {
    case kVarPerLevel: return &launch_tmem_kernel<M, BfF32PerLevel, false, OM>;
    case kVarEnd: return &launch_tmem_kernel<M, BfF32Plain, true, OM>;
    case kVarPlain: return &launch_tmem_kernel<M, BfF32Plain, false, OM>;
    case kVarI32: return &launch_tmem_kernel<M, BfI32, false, OM>;
    default: return nullptr;
  }
}

}  // namespace

template <int M>
TmemLaunchFn tmem_order(int var, int om) {
  switch (om) {
    case 0: return tmem_variant<M, 0>(var);
    case 1: return tmem_variant<M, 1>(var);
    case 2: return tmem_variant<M, 2>(var);
    case 3: return tmem_variant<M, 3>(var);
    default: return nullptr;
  }
}

TmemLaunchFn lookup_tmem(int m, int var, int om) {
  if (m == 15) return tmem_order<15>(var, om);
  if (m == 16) return tmem_order<16>(var, om);
  return nullptr;
}

}  // namespace chw
