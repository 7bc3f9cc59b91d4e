// Host-side launcher of the tensor-memory kernel (tmem.cuh), shared by the translation
// units that instantiate it: one persistent 256-thread CTA per SM, `units` signals (or
// column blocks) of 2^M words, or (XP > 0) one persistent cluster of 2^XP such CTAs per
// signal of 2^(M+XP) words.
#pragma once

#include "launch.cuh"
#include "tmem.cuh"

namespace chw {

template <int M, class BF, bool SC, int OM, int CLO = 0, bool HZ = false, int XP = 0>
cudaError_t launch_tmem_kernel(const CUtensorMap* tin, const CUtensorMap* tout, const FusedArgs& args, int64_t units,
                               cudaStream_t st) {
  constexpr auto kern = tmem_kernel<M, BF, SC, OM, CLO, HZ, XP>;
  constexpr int smem = tmem_smem_bytes<XP>();
  static_assert(2 * smem > 233472, "one CTA per SM: the tensor-memory allocation never waits on a peer");
  static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (attr != cudaSuccess) return attr;
  // signals (XP = 0) or clusters of 2^XP CTAs, one signal each (XP > 0), resident at once
  static const int64_t resident = resident_units(kern, kTmemThreads, smem, 1 << XP);
  int64_t grid = units;
  int64_t cap = persistent_cap_override();
  if (cap <= 0) cap = resident;
  if (cap > 0 && grid > cap) grid = cap;
  if constexpr (XP > 0) {  // one exchange-scratch region per cluster
    if (args.xscratch == nullptr || args.xclusters < 1) return cudaErrorInvalidValue;
    if (grid > args.xclusters) grid = args.xclusters;
  }
  if constexpr (XP == 0) {
    kern<<<static_cast<unsigned>(grid), kTmemThreads, smem, st>>>(*tin, *tout, args, units);
    return cudaGetLastError();
  } else {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(static_cast<unsigned>(grid << XP), 1, 1);
    cfg.blockDim = dim3(kTmemThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 1u << XP;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, *tin, *tout, args, units);
  }
}

}  // namespace chw
