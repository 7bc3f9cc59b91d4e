// Launchers of the tensor-memory whole-signal kernel (tmem.cuh): m = 15, 16, four-byte
// elements, dyadic, natural or sequency order or the column-blocked rows of a two-pass
// split, every butterfly variant.
#include "launch.cuh"
#include "tmem.cuh"

namespace chw {

namespace {

template <int M, class BF, bool SC, int OM>
cudaError_t launch_tmem(const CUtensorMap* tin, const CUtensorMap* tout, const FusedArgs& args, int64_t units,
                        cudaStream_t st) {
  constexpr auto kern = tmem_kernel<M, BF, SC, OM>;
  constexpr int smem = tmem_smem_bytes();
  static_assert(2 * smem > 233472, "one CTA per SM: the tensor-memory allocation never waits on a peer");
  static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (attr != cudaSuccess) return attr;
  static const int64_t resident = resident_units(kern, kTmemThreads, smem, 1);
  int64_t grid = units;
  int64_t cap = persistent_cap_override();
  if (cap <= 0) cap = resident;
  if (cap > 0 && grid > cap) grid = cap;
  kern<<<static_cast<unsigned>(grid), kTmemThreads, smem, st>>>(*tin, *tout, args, units);
  return cudaGetLastError();
}

template <int M, int OM>
TmemLaunchFn tmem_variant(int var) {
  switch (var) {
    case kVarPerLevel: return &launch_tmem<M, BfF32PerLevel, false, OM>;
    case kVarEnd: return &launch_tmem<M, BfF32Plain, true, OM>;
    case kVarPlain: return &launch_tmem<M, BfF32Plain, false, OM>;
    case kVarI32: return &launch_tmem<M, BfI32, false, OM>;
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
