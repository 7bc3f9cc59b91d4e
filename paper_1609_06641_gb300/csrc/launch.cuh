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

// `units`: number of (cluster) tiles; the launcher sizes a persistent grid.
using FusedLaunchFn = cudaError_t (*)(const CUtensorMap* tin, const FusedArgs& args, int64_t units, cudaStream_t st);

template <int TB>
constexpr int fused_smem_bytes() {
  return (8 << TB) + 1024 + 64;  // two tile buffers, alignment slack, two mbarriers
}

// Units the device keeps resident at once for this kernel (0 if the query fails).
template <class K>
int64_t resident_units(K kern, int threads, int smem, int cluster) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cluster <= 1) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess) return 0;
    return static_cast<int64_t>(per_sm) * sms;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(static_cast<unsigned>(cluster), 1, 1);
  cfg.blockDim = dim3(static_cast<unsigned>(threads), 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = static_cast<unsigned>(cluster);
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nc = 0;
  if (cudaOccupancyMaxActiveClusters(&nc, kern, &cfg) != cudaSuccess) return 0;
  return nc;
}

int64_t persistent_cap_override();  // CHW_MAX_RESIDENT_UNITS, 0 = none (tuning)

template <int TLO, int M, int TB, int CB, class BF, bool SC, int OM, bool HZ = false>
cudaError_t launch_fused(const CUtensorMap* tin, const FusedArgs& args, int64_t units, cudaStream_t st) {
  constexpr auto kern = [] {
    if constexpr (CB > 0)
      return cluster_kernel<TLO, M, TB, CB, BF, SC, OM>;
    else
      return fused_kernel<TLO, M, TB, CB, BF, SC, OM, HZ>;
  }();
  constexpr int smem = CB > 0 ? cluster_smem_bytes<TB>() : fused_smem_bytes<TB>();
  constexpr int threads = 1 << (TB - 6);
  static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (attr != cudaSuccess) return attr;
  static const int64_t resident = resident_units(kern, threads, smem, 1 << CB);
  int64_t grid_units = units;
  int64_t cap = persistent_cap_override();
  if (cap <= 0) cap = resident;
  if (cap > 0 && grid_units > cap) grid_units = cap;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(static_cast<unsigned>(grid_units << CB), 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
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
  return cudaLaunchKernelEx(&cfg, kern, *tin, args, units);
}

// Staging key S of a fused shape (see make_plan): a tile-store launch views its output as
// 4-D boxes {32 words, 8 (bits S..S+2), 2^(S-5) (bits 5..S-1), 2^(TB-S-3) (bits S+3..)}.
inline int stage_key(int tlo, int m, int tb, int cb, int om) { return make_plan(tlo, m, tb, cb, om).stage_s; }

// Kernel for one fused shape and variant (nullptr if that shape was not compiled).  The
// table is generated by the build from its list of shapes, one translation unit per shape.
FusedLaunchFn lookup_fused(int tlo, int m, int tb, int cb, int var, int om);

// The single-CTA dyadic row kernel of m = 1..14 (tile bits tb) that also writes the Haar side
// output z = Psi_m x to FusedArgs::haar_z (fused.cuh, HaarZ); nullptr for other shapes.
FusedLaunchFn lookup_fused_hz(int m, int tb, int var);

// The tensor-memory whole-signal kernel (tmem.cuh) for m = 15, 16 in dyadic (om = 0),
// column-blocked two-pass rows (om = 1, FusedArgs::colblock_a), natural (om = 2) or
// sequency (om = 3) order: `tin` maps the input as rows of 32 words
// (boxes of 256 rows), `tout` the output as rows of 2^(m-8) words with boxes of 32 words x
// 256 rows (dyadic; unused by om = 1, 3) or rows of 2^(m-6) words with boxes of
// 32 x 64 (natural), all SWIZZLE_128B; `units` is the number of signals.  nullptr for
// other shapes.
using TmemLaunchFn = cudaError_t (*)(const CUtensorMap* tin, const CUtensorMap* tout, const FusedArgs& args,
                                     int64_t units, cudaStream_t st);
TmemLaunchFn lookup_tmem(int m, int var, int om);

// The dyadic tensor-memory kernel (m = 15, 16) that also writes the Haar side output.
TmemLaunchFn lookup_tmem_hz(int m, int var);

// The same kernel on the column tiles of a two-pass split's second pass: units of 2^m words
// (m = 15, 16) holding 2^clo columns x 2^(m-clo) rows of the first pass's column-blocked
// output, transformed over the rows and written as 2^clo contiguous output rows in dyadic
// order (tin, tout as for the dyadic whole-signal kernel).  clo = 5 for m = 15; 2..5 for
// m = 16.  nullptr for other shapes.
TmemLaunchFn lookup_tmem_col(int m, int clo, int var);

// The tensor-memory kernel for one signal of 2^m words spread over a cluster of 2^(m-16)
// SMs (m = 17: two), dyadic order: `tin` as for the whole-signal kernel, `tout` the output
// as rows of 2^(m-8) words with boxes of 32 words x 256 rows (SWIZZLE_128B); `units` is the
// number of signals.  FusedArgs::diag_mask must be 2^m - 1 when D is given.  nullptr for
// other m.
TmemLaunchFn lookup_tmem_cross(int m, int var);

// Clusters the m = 17 pair kernel's exchange scratch must hold on `device` (one per two
// SMs, the most that can be resident); each takes four 32 KB slots (128 KB).
inline int64_t tmem_cross_clusters(int device) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  return sms >= 2 ? sms / 2 : 1;
}

}  // namespace chw

