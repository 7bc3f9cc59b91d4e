// Device code of the persistent ragged kernel (see ragged.cuh for the schedule).
#pragma once

#include "ragged.cuh"

namespace chw {

__device__ __forceinline__ int ld_acquire_gpu(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_gpu_add(int32_t* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Signals with m <= 13, one after another: the cascade's butterflies level by level in
// shared memory (level t pairs labels differing in bit t), then the dyadic reorder.
template <class BF, bool SCALE>
__device__ void small_group(const RaggedArgs& a, const RaggedTask& task, uint32_t* buf) {
  BF bf{};
  if constexpr (std::is_same_v<BF, BfF32PerLevel>) bf.c = 0.70710678118654752440f;
  for (int s = task.index; s < task.index + task.count; ++s) {
    const int m = a.ms[s];
    const int n = 1 << m;
    const int64_t off = a.off[s];
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
  using BF1 = BfF32PerLevel;
  static constexpr bool SC = false;
};
template <>
struct RaggedVar<kVarEnd> {
  using BF = BfF32Plain;
  using BF1 = BfF32Plain;
  static constexpr bool SC = true;
};
template <>
struct RaggedVar<kVarPlain> {
  using BF = BfF32Plain;
  using BF1 = BfF32Plain;
  static constexpr bool SC = false;
};
template <>
struct RaggedVar<kVarI32> {
  using BF = BfI32;
  using BF1 = BfI32;
  static constexpr bool SC = false;
};

constexpr int kRaggedThreads = 1 << (kRaggedTileBits - 6);

template <int VAR>
__global__ void __launch_bounds__(kRaggedThreads, 2)
    ragged_kernel(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmring,
                  const RaggedArgs a) {
  using V = RaggedVar<VAR>;
  using BF = typename V::BF;
  using BF1 = typename V::BF1;
  constexpr bool SC = V::SC;
  constexpr int TB = kRaggedTileBits;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  uint32_t* buf = reinterpret_cast<uint32_t*>(base);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + (4u << TB));
  __shared__ int s_task;
  const uint32_t tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  uint32_t parity = 0;
  for (;;) {
    __syncthreads();
    if (tid == 0) s_task = atomicAdd(a.queue_head, 1);
    __syncthreads();
    const int t = s_task;
    if (t >= a.ntasks) break;
    const RaggedTask task = a.tasks[t];
    if (task.wait_on >= 0) {
      if (tid == 0) {
        bool ok = false;
        for (uint32_t i = 0; i < (1u << 26); ++i) {
          if (ld_acquire_gpu(a.ctr + task.wait_on) >= task.wait_val) {
            ok = true;
            break;
          }
          __nanosleep(64);
        }
        if (!ok) atomicCAS(a.status, 0, kStatusTimeout);
        // the awaited data was written by generic stores; TMA reads it through the async proxy
        asm volatile("fence.proxy.async.global;" ::: "memory");
      }
      __syncthreads();
    }
    FusedArgs fa{};
    fa.status = a.status;
    fa.diag_in = nullptr;
    fa.diag_out = nullptr;
    fa.diag_mask = 0;
    switch (task.kind) {
      case kTaskSmall:
        small_group<BF, SC>(a, task, buf);
        break;
      case kTaskTile:
        fa.out = a.y;
        fa.out_total = a.total;
        fa.end_scale = end_scale_dev(TB);
        fused_tile<0, TB, TB, 0, BF, SC, 0>(&tmx, static_cast<int>(task.off >> 5), task.off, fa, buf, bar, parity);
        parity ^= 1u;
        break;
      case kTaskRow: {
        fa.out = a.ring;
        fa.out_total = kRingSlots * kRingSlotWords;
        fa.end_scale = 1.0f;
        fa.colblock_a = task.m - TB;
        const int64_t in0 = task.off + (static_cast<int64_t>(task.index) << TB);
        const int64_t ob = static_cast<int64_t>(task.slot) * kRingSlotWords + (static_cast<int64_t>(task.index) << TB);
        fused_tile<0, TB, TB, 0, BF1, false, 1>(&tmx, static_cast<int>(in0 >> 5), ob, fa, buf, bar, parity);
        parity ^= 1u;
        break;
      }
      case kTaskCol: {
        fa.out = a.y;
        fa.out_total = a.total;
        fa.end_scale = end_scale_dev(task.m);
        const int row0 = static_cast<int>(
            (static_cast<int64_t>(task.slot) * kRingSlotWords + (static_cast<int64_t>(task.index) << TB)) >> 5);
        const int64_t ob = task.off + (static_cast<int64_t>(task.index) << TB);
        switch (task.m - TB) {
          case 1: fused_tile<5, 1, TB, 0, BF, SC, 0>(&tmring, row0, ob, fa, buf, bar, parity); break;
          case 2: fused_tile<5, 2, TB, 0, BF, SC, 0>(&tmring, row0, ob, fa, buf, bar, parity); break;
          case 3: fused_tile<5, 3, TB, 0, BF, SC, 0>(&tmring, row0, ob, fa, buf, bar, parity); break;
          case 4: fused_tile<5, 4, TB, 0, BF, SC, 0>(&tmring, row0, ob, fa, buf, bar, parity); break;
          case 5: fused_tile<5, 5, TB, 0, BF, SC, 0>(&tmring, row0, ob, fa, buf, bar, parity); break;
          default: fused_tile<5, 6, TB, 0, BF, SC, 0>(&tmring, row0, ob, fa, buf, bar, parity); break;
        }
        parity ^= 1u;
        break;
      }
      default:
        break;
    }
    if (task.done_ctr >= 0) {
      __threadfence();
      __syncthreads();
      if (tid == 0) red_release_gpu_add(a.ctr + task.done_ctr, 1);
    }
  }
}

template <int VAR>
cudaError_t launch_ragged(const CUtensorMap& tx, const CUtensorMap& tr, const RaggedArgs& a, cudaStream_t st) {
  auto kern = ragged_kernel<VAR>;
  constexpr int smem = (4 << kRaggedTileBits) + 1024 + 64;  // one tile buffer + mbarrier
  static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (attr != cudaSuccess) return attr;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRaggedThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int grid = sms * per_sm;
  if (grid > a.ntasks) grid = a.ntasks;
  if (grid < 1) grid = 1;
  kern<<<grid, kRaggedThreads, smem, st>>>(tx, tr, a);
  return cudaGetLastError();
}


}  // namespace chw
