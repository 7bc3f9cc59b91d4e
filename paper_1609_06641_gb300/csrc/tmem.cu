// Launchers of the tensor-memory whole-signal kernel (tmem.cuh): m = 15, 16, four-byte
// elements, dyadic order, every butterfly variant.
#include "launch.cuh"
#include "tmem.cuh"

namespace chw {

namespace {

template <int M, class BF, bool SC>
cudaError_t launch_tmem(const CUtensorMap* tin, const CUtensorMap* tout, const FusedArgs& args, int64_t units,
                        cudaStream_t st) {
  constexpr auto kern = tmem_kernel<M, BF, SC>;
  constexpr int smem = tmem_smem_bytes<M>();
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

template <int M>
TmemLaunchFn tmem_variant(int var) {
  switch (var) {
    case kVarPerLevel: return &launch_tmem<M, BfF32PerLevel, false>;
    case kVarEnd: return &launch_tmem<M, BfF32Plain, true>;
    case kVarPlain: return &launch_tmem<M, BfF32Plain, false>;
    case kVarI32: return &launch_tmem<M, BfI32, false>;
    default: return nullptr;
  }
}

}  // namespace

TmemLaunchFn lookup_tmem(int m, int var) {
  if (m == 15) return tmem_variant<15>(var);
  if (m == 16) return tmem_variant<16>(var);
  return nullptr;
}

}  // namespace chw
