// Device code of the ragged batches' short signals (see ragged.cuh).
#pragma once

#include "ragged.cuh"

namespace chw {

// Signals with m <= 12, one after another: the cascade's butterflies level by level in
// shared memory (level t pairs labels differing in bit t), then the dyadic reorder.
template <class BF, bool SCALE>
__device__ void small_group(const RaggedArgs& a, const RaggedTask& task, uint32_t* buf) {
  BF bf{};
  if constexpr (std::is_same_v<BF, BfF32PerLevel>) bf.c = 0.70710678118654752440f;
  for (int s = task.index; s < task.index + task.count; ++s) {
    const int m = a.ms[s];
    const int n = 1 << m;
    const int64_t off = a.off[s];
    if (a.checked && !(off >= 0 && off <= a.total - n)) {  // the same decision in every thread
      if (threadIdx.x == 0) check_fail(a.status, off);
      continue;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) buf[i] = a.x[off + i];
    for (int t = 0; t < m; ++t) {
      __syncthreads();
      const int low = (1 << t) - 1;
      for (int p = threadIdx.x; p < n / 2; p += blockDim.x) {
        const int i0 = ((p & ~low) << 1) | (p & low);
        uint32_t u = buf[i0], w = buf[i0 | (1 << t)];
        bf(u, w);
        buf[i0] = u;
        buf[i0 | (1 << t)] = w;
      }
    }
    __syncthreads();
    const float sc = SCALE ? end_scale_dev(m) : 1.0f;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const int lab = m == 0 ? 0 : static_cast<int>(__brev(static_cast<uint32_t>(k)) >> (32 - m));
      uint32_t v = buf[lab];
      if constexpr (SCALE) v = __float_as_uint(__fmul_rn(__uint_as_float(v), sc));
      a.y[off + k] = v;
    }
  }
}

template <int VAR>
struct RaggedVar;
template <>
struct RaggedVar<kVarPerLevel> {
  using BF = BfF32PerLevel;
  static constexpr bool SC = false;
};
template <>
struct RaggedVar<kVarEnd> {
  using BF = BfF32Plain;
  static constexpr bool SC = true;
};
template <>
struct RaggedVar<kVarPlain> {
  using BF = BfF32Plain;
  static constexpr bool SC = false;
};
template <>
struct RaggedVar<kVarI32> {
  using BF = BfI32;
  static constexpr bool SC = false;
};

constexpr int kRaggedThreads = 256;

// Persistent: every CTA takes runs of short signals from the task list until it is empty.
template <int VAR>
__global__ void __launch_bounds__(kRaggedThreads)
    ragged_small_kernel(const RaggedArgs a) {
  using V = RaggedVar<VAR>;
  __shared__ __align__(16) uint32_t buf[1 << kRaggedSmallMaxM];
  __shared__ int s_task;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_task = atomicAdd(a.queue_head, 1);
    __syncthreads();
    const int t = s_task;
    if (t >= a.ntasks) break;
    small_group<typename V::BF, V::SC>(a, a.tasks[t], buf);
  }
}

template <int VAR>
cudaError_t launch_ragged_small(const RaggedArgs& a, cudaStream_t st) {
  auto kern = ragged_small_kernel<VAR>;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRaggedThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int grid = sms * per_sm;
  if (grid > a.ntasks) grid = a.ntasks;
  if (grid < 1) grid = 1;
  kern<<<grid, kRaggedThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace chw
