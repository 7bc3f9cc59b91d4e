// Host-side launcher of the tensor-memory kernel (tmem.cuh), shared by the translation
// units that instantiate it: one persistent 256-thread CTA per SM, `units` signals (or
// column blocks) of 2^M words.
#pragma once

#include "launch.cuh"
#include "tmem.cuh"

namespace chw {

template <int M, class BF, bool SC, int OM, int CLO = 0, bool HZ = false>
cudaError_t launch_tmem_kernel(const CUtensorMap* tin, const CUtensorMap* tout, const FusedArgs& args, int64_t units,
                               cudaStream_t st) {
  constexpr auto kern = tmem_kernel<M, BF, SC, OM, CLO, HZ>;
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

}  // namespace chw
