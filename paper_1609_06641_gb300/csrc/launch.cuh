// Host-side launch wrappers for the fused kernels and the lookup of an instantiation.
#pragma once

#include <cuda_runtime.h>

#include "fused.cuh"

namespace chw {

// Butterfly / scaling variant of a fused launch.
enum FusedVariant {
  kVarPerLevel = 0,  // fp32, (a+-b)*c at every level
  kVarEnd = 1,       // fp32, unscaled butterflies then one multiply by FusedArgs::end_scale
  kVarPlain = 2,     // fp32, unscaled butterflies
  kVarI32 = 3        // int32, unscaled, wrapping
};

using FusedLaunchFn = cudaError_t (*)(const CUtensorMap* tin, const FusedArgs& args, int64_t ctas, cudaStream_t st);

template <int TB>
constexpr int fused_smem_bytes() {
  return (4 << TB) + 1024 + 64;
}

template <int TLO, int M, int TB, int CB, class BF, bool SC, int OM>
cudaError_t launch_fused(const CUtensorMap* tin, const FusedArgs& args, int64_t ctas, cudaStream_t st) {
  auto kern = fused_kernel<TLO, M, TB, CB, BF, SC, OM>;
  constexpr int smem = fused_smem_bytes<TB>();
  static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (attr != cudaSuccess) return attr;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(static_cast<unsigned>(ctas), 1, 1);
  cfg.blockDim = dim3(1u << (TB - 6), 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  if constexpr (CB > 0) {
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 1u << CB;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, kern, *tin, args);
}

// Kernel for one fused shape and variant (nullptr if that shape was not compiled).  The
// table is generated by the build from its list of shapes, one translation unit per shape.
FusedLaunchFn lookup_fused(int tlo, int m, int tb, int cb, int var, int om);

}  // namespace chw

