// Row-stack tier for signals of 2^15..2^17 elements: one persistent CTA per signal, no
// cross-CTA synchronisation.
//
// A signal of 2^M elements is 2^(M-14) rows of 2^14.  The CTA transforms the rows one by
// one (label bits 0..13, the fused tile's three register phases, TMA double-buffered
// across rows and signals) into its private scratch slot, in dyadic order within each row.
// The slot (2^M words per CTA, rewritten for every signal) stays in L2.  A streaming pass
// then finishes label bits 14..M-1: for each in-row position k it reads the 2^(M-14)
// values of that column, runs their butterflies (bit 14 first) and writes the outputs
// (k << (M-14)) | bitrev(q), which are contiguous.  Every value meets bits 0..M-1 in order,
// so the results equal the cascade's bit for bit.
#pragma once

#include "launch.cuh"

namespace chw {

template <int RB>
__device__ __forceinline__ constexpr int bitrev_bits(int q) {
  int r = 0;
  for (int i = 0; i < RB; ++i) r |= ((q >> i) & 1) << (RB - 1 - i);
  return r;
}

template <int M, class BF, bool SCALE>
__global__ void __launch_bounds__(256, 1)
    rowstack_kernel(const __grid_constant__ CUtensorMap tin, const FusedArgs args, uint32_t* scratch,
                    const int64_t batch) {
  constexpr int TB = 14;
  constexpr int RB = M - TB;
  constexpr int R = 1 << RB;
  static_assert(RB >= 1 && RB <= 3, "2 to 8 rows per signal");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  uint32_t* bufs[2] = {reinterpret_cast<uint32_t*>(base), reinterpret_cast<uint32_t*>(base) + (1u << TB)};
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + (8u << TB));
  const uint32_t tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t* slot = scratch + (static_cast<int64_t>(blockIdx.x) << M);
  BF bf{};
  if constexpr (std::is_same_v<BF, BfF32PerLevel>) bf.c = 0.70710678118654752440f;

  // row transforms write the slot; no scaling there (END scales once, in the column pass)
  FusedArgs ra = args;
  ra.out = slot;
  ra.out_total = int64_t{1} << M;
  ra.diag_out = nullptr;

  const int64_t stride = gridDim.x;
  auto tile_row = [&](int64_t s, int q) { return static_cast<int>(((s << RB) + q) << (TB - 5)); };
  if (tid == 0 && blockIdx.x < batch) tile_issue<TB>(&tin, tile_row(blockIdx.x, 0), bufs[0], bar);
  int k = 0;
  for (int64_t s = blockIdx.x; s < batch; s += stride) {
    for (int q = 0; q < R; ++q, ++k) {
      // prefetch the next row (the next signal's first row after the last one)
      if (tid == 0) {
        const int64_t ns = q + 1 < R ? s : s + stride;
        const int nq = q + 1 < R ? q + 1 : 0;
        if (ns < batch) tile_issue<TB>(&tin, tile_row(ns, nq), bufs[(k + 1) & 1], bar + ((k + 1) & 1));
      }
      tile_compute<0, TB, TB, 0, BF, false, 0>(static_cast<int64_t>(tile_row(s, q)) * 32,
                                                 static_cast<int64_t>(q) << TB, ra, bufs[k & 1], bar + (k & 1),
                                                 (k >> 1) & 1);
      __syncthreads();
    }
    // ---- column pass over the rows held in the slot (this CTA's own writes): each thread
    // takes 4 adjacent columns per step (16-byte L2 loads from every row), U steps in flight.
    uint32_t* out = static_cast<uint32_t*>(args.out) + (s << M);
    constexpr int U = 4;
    for (int c0 = tid * 4; c0 < (1 << TB); c0 += 256 * 4 * U) {
      uint4 ld[U][R];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int q = 0; q < R; ++q)
          ld[u][q] = __ldcg(reinterpret_cast<const uint4*>(slot + (q << TB) + c0 + u * 1024));
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int c = c0 + u * 1024;
        uint32_t w[4 * R];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          uint32_t v[R];
#pragma unroll
          for (int q = 0; q < R; ++q) v[q] = j == 0 ? ld[u][q].x : j == 1 ? ld[u][q].y : j == 2 ? ld[u][q].z : ld[u][q].w;
#pragma unroll
          for (int b = 0; b < RB; ++b)
#pragma unroll
            for (int q = 0; q < R; ++q)
              if (((q >> b) & 1) == 0) bf(v[q], v[q | (1 << b)]);
#pragma unroll
          for (int i = 0; i < R; ++i) {
            uint32_t t = v[bitrev_bits<RB>(i)];
            if constexpr (SCALE) t = __float_as_uint(__fmul_rn(__uint_as_float(t), args.end_scale));
            if (args.diag_out != nullptr) {
              const int64_t di = ((static_cast<int64_t>(c + j) << RB) | i) & args.diag_mask;
              if (args.diag_out[di] < 0) t = std::is_same_v<BF, BfI32> ? 0u - t : t ^ 0x80000000u;
            }
            w[j * R + i] = t;
          }
        }
        // columns c..c+3 own the 4R consecutive outputs starting at c << RB
        uint32_t* o = out + (static_cast<int64_t>(c) << RB);
#pragma unroll
        for (int i = 0; i < 4 * R; i += 4) st_global_v4(o + i, w[i], w[i + 1], w[i + 2], w[i + 3]);
      }
    }
    __syncthreads();  // the slot is rewritten by the next signal's rows
  }
}

template <int M, class BF, bool SCALE>
cudaError_t launch_rowstack(const CUtensorMap* tin, const FusedArgs& args, uint32_t* scratch, int64_t grid,
                            int64_t batch, cudaStream_t st) {
  auto kern = rowstack_kernel<M, BF, SCALE>;
  constexpr int smem = fused_smem_bytes<14>();
  static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (attr != cudaSuccess) return attr;
  kern<<<static_cast<unsigned>(grid), 256, smem, st>>>(*tin, args, scratch, batch);
  return cudaGetLastError();
}

}  // namespace chw
