// The Haar wavelet transform Psi_m of eq. (2) and its transpose, for 4-byte elements.
//
// Psi_m x in the layout eq. (2) produces: z = [a, d_m, d_{m-1}, ..., d_1], where the
// level-l details d_l (2^{m-l} values) sit at [2^{m-l}, 2^{m-l+1}) and a at 0.  Level l
// turns the current approximation (2^{m-l+1} values) into pair sums s_i = v_{2i} + v_{2i+1}
// (the next approximation) and differences d_i = v_{2i} - v_{2i+1}.
//
// A pass handles `tc` <= 13 levels on rows of 2^tc consecutive elements: one 256-thread
// CTA per 2^13 elements (a row, or 2^{13-tc} short rows), the approximation ping-ponging
// between two shared arrays while each level's details stream straight to their final
// place in z with 16-byte stores.  Signals longer than 2^13 take several passes: the
// first leaves one approximation per row in a small scratch array (2^{-13} of the data),
// which the next pass transforms as a signal of 2^{m-13} elements, writing the coarse
// levels into the front of z.  The transpose runs the passes in the opposite order: the
// coarse pass rebuilds the row approximations into scratch, and the fine pass
// synthesises each row from its approximation and its details (v_{2i} = u_i + d_i,
// v_{2i+1} = u_i - d_i), coarse to fine.
//
// Normalisation per element, matching the modes of the transform: PER_LEVEL multiplies
// every butterfly output by fp32(1/sqrt2); NONE leaves the butterflies unscaled; END
// leaves them unscaled and multiplies each coefficient once by fp32(2^{-L/2}), L = the
// number of levels behind it (after the analysis, before the synthesis).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "fused.cuh"

namespace chw {

constexpr int kHaarRowBits = 13;
constexpr int kHaarThreads = 256;

struct HaarFwdArgs {
  const uint32_t* in;  // rows of 2^tc words: row r at in + (r << tc)
  uint32_t* out;       // z: signal s's coefficients at out + s * out_stride
  int64_t out_stride;
  uint32_t* approx;    // row approximations for the next pass (approx[r]), or nullptr (last pass)
  int64_t rows;        // batch << (mlen - tc)
  int mlen;            // this pass transforms signals of 2^mlen elements
  int tc;              // levels per row: min(mlen, 13)
  int lev0;            // levels done by earlier passes
  int mtotal;          // m
  int* status;         // device status word (bounded waits)
};

struct HaarInvArgs {
  const uint32_t* z;       // coefficients, signal s at z + s * z_stride
  int64_t z_stride;
  const uint32_t* approx;  // row approximations from the coarser pass, or nullptr (take z[0])
  uint32_t* out;           // row r's 2^tc results at out + (r << tc)
  int64_t rows;
  int mlen, tc, lev0, mtotal;
};

__device__ __forceinline__ uint4 lds4(const uint32_t* p) { return *reinterpret_cast<const uint4*>(p); }
__device__ __forceinline__ void sts4(uint32_t* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  *reinterpret_cast<uint4*>(p) = make_uint4(a, b, c, d);
}
__device__ __forceinline__ uint32_t scale_u32(uint32_t v, float s) {
  return __float_as_uint(__fmul_rn(__uint_as_float(v), s));
}

template <class BF, bool END>
__global__ void __launch_bounds__(kHaarThreads) haar_fwd_kernel(const HaarFwdArgs p) {
  __shared__ __align__(16) uint32_t sa[1 << kHaarRowBits];
  __shared__ __align__(16) uint32_t sb[1 << (kHaarRowBits - 1)];
  BF bf{};
  if constexpr (std::is_same_v<BF, BfF32PerLevel>) bf.c = 0.70710678118654752440f;
  const int tc = p.tc;
  const int64_t row0 = static_cast<int64_t>(blockIdx.x) << (kHaarRowBits - tc);
  const int64_t left = p.rows - row0;
  const int nseg = left < (int64_t{1} << (kHaarRowBits - tc)) ? static_cast<int>(left) : 1 << (kHaarRowBits - tc);
  const int count = nseg << tc;
  const uint32_t* src = p.in + (row0 << tc);  // 2^13-element aligned
  for (int e = threadIdx.x * 4; e < count; e += kHaarThreads * 4) {
    if (e + 4 <= count) {
      *reinterpret_cast<uint4*>(sa + e) = __ldcs(reinterpret_cast<const uint4*>(src + e));
    } else {
      for (int k = e; k < count; ++k) sa[k] = src[k];
    }
  }
  __syncthreads();
  const int cbits = p.mlen - tc;  // rows per signal = 2^cbits
  uint32_t* cur = sa;
  uint32_t* nxt = sb;
  for (int l = 1; l <= tc; ++l) {
    const int half = tc - l;  // 2^half pairs per row at this level
    const int npairs = nseg << half;
    const float sc = END ? end_scale_dev(p.lev0 + l) : 1.0f;
    const int64_t dblock = int64_t{1} << (p.mlen - l);
    if (half >= 2) {
      for (int q = threadIdx.x * 4; q < npairs; q += kHaarThreads * 4) {
        const uint4 u = lds4(cur + 2 * q), w = lds4(cur + 2 * q + 4);
        uint32_t s0 = u.x, d0 = u.y, s1 = u.z, d1 = u.w, s2 = w.x, d2 = w.y, s3 = w.z, d3 = w.w;
        bf(s0, d0);
        bf(s1, d1);
        bf(s2, d2);
        bf(s3, d3);
        sts4(nxt + q, s0, s1, s2, s3);
        if constexpr (END) {
          d0 = scale_u32(d0, sc);
          d1 = scale_u32(d1, sc);
          d2 = scale_u32(d2, sc);
          d3 = scale_u32(d3, sc);
        }
        const int64_t r = row0 + (q >> half);
        const int64_t s = r >> cbits, c = r & ((int64_t{1} << cbits) - 1);
        const int i = q & ((1 << half) - 1);
        st_global_v4(p.out + s * p.out_stride + dblock + (c << half) + i, d0, d1, d2, d3);
      }
    } else {
      for (int q = threadIdx.x; q < npairs; q += kHaarThreads) {
        uint32_t sv = cur[2 * q], dv = cur[2 * q + 1];
        bf(sv, dv);
        nxt[q] = sv;
        if constexpr (END) dv = scale_u32(dv, sc);
        const int64_t r = row0 + (q >> half);
        const int64_t s = r >> cbits, c = r & ((int64_t{1} << cbits) - 1);
        const int i = q & ((1 << half) - 1);
        p.out[s * p.out_stride + dblock + (c << half) + i] = dv;
      }
    }
    __syncthreads();
    uint32_t* t = cur;
    cur = nxt;
    nxt = t;
  }
  for (int g = threadIdx.x; g < nseg; g += kHaarThreads) {
    uint32_t v = cur[g];
    if (p.approx != nullptr) {
      p.approx[row0 + g] = v;  // unscaled: the next pass continues the butterflies
    } else {
      if constexpr (END) v = scale_u32(v, end_scale_dev(p.mtotal));
      p.out[(row0 + g) * p.out_stride] = v;  // last pass: one row per signal
    }
  }
}

template <class BF, bool END>
__global__ void __launch_bounds__(kHaarThreads) haar_inv_kernel(const HaarInvArgs p) {
  __shared__ __align__(16) uint32_t sa[1 << kHaarRowBits];
  __shared__ __align__(16) uint32_t sb[1 << (kHaarRowBits - 1)];
  BF bf{};
  if constexpr (std::is_same_v<BF, BfF32PerLevel>) bf.c = 0.70710678118654752440f;
  const int tc = p.tc;
  const int64_t row0 = static_cast<int64_t>(blockIdx.x) << (kHaarRowBits - tc);
  const int64_t left = p.rows - row0;
  const int nseg = left < (int64_t{1} << (kHaarRowBits - tc)) ? static_cast<int>(left) : 1 << (kHaarRowBits - tc);
  const int cbits = p.mlen - tc;
  for (int g = threadIdx.x; g < nseg; g += kHaarThreads) {
    uint32_t v;
    if (p.approx != nullptr) {
      v = p.approx[row0 + g];
    } else {
      v = p.z[(row0 + g) * p.z_stride];  // the coarsest pass: one row per signal
      if constexpr (END) v = scale_u32(v, end_scale_dev(p.mtotal));
    }
    sa[g] = v;
  }
  __syncthreads();
  if (tc == 0) {
    for (int g = threadIdx.x; g < nseg; g += kHaarThreads) p.out[row0 + g] = sa[g];
    return;
  }
  uint32_t* cur = sa;
  uint32_t* nxt = sb;
  for (int l = tc; l >= 1; --l) {
    const int half = tc - l;  // 2^half approximations per row in, 2^(half+1) out
    const int npairs = nseg << half;
    const float sc = END ? end_scale_dev(p.lev0 + l) : 1.0f;
    const int64_t dblock = int64_t{1} << (p.mlen - l);
    uint32_t* dst = l == 1 ? p.out + (row0 << tc) : nxt;
    if (half >= 2) {
      for (int q = threadIdx.x * 4; q < npairs; q += kHaarThreads * 4) {
        const int64_t r = row0 + (q >> half);
        const int64_t s = r >> cbits, c = r & ((int64_t{1} << cbits) - 1);
        const int i = q & ((1 << half) - 1);
        const uint4 d = __ldcs(reinterpret_cast<const uint4*>(p.z + s * p.z_stride + dblock + (c << half) + i));
        const uint4 u = lds4(cur + q);
        uint32_t e0 = u.x, o0 = d.x, e1 = u.y, o1 = d.y, e2 = u.z, o2 = d.z, e3 = u.w, o3 = d.w;
        if constexpr (END) {
          o0 = scale_u32(o0, sc);
          o1 = scale_u32(o1, sc);
          o2 = scale_u32(o2, sc);
          o3 = scale_u32(o3, sc);
        }
        bf(e0, o0);
        bf(e1, o1);
        bf(e2, o2);
        bf(e3, o3);
        if (l == 1) {
          st_global_v4(dst + 2 * q, e0, o0, e1, o1);
          st_global_v4(dst + 2 * q + 4, e2, o2, e3, o3);
        } else {
          sts4(dst + 2 * q, e0, o0, e1, o1);
          sts4(dst + 2 * q + 4, e2, o2, e3, o3);
        }
      }
    } else {
      for (int q = threadIdx.x; q < npairs; q += kHaarThreads) {
        const int64_t r = row0 + (q >> half);
        const int64_t s = r >> cbits, c = r & ((int64_t{1} << cbits) - 1);
        const int i = q & ((1 << half) - 1);
        uint32_t e = cur[q], o = p.z[s * p.z_stride + dblock + (c << half) + i];
        if constexpr (END) o = scale_u32(o, sc);
        bf(e, o);
        dst[2 * q] = e;
        dst[2 * q + 1] = o;
      }
    }
    __syncthreads();
    uint32_t* t = cur;
    cur = nxt;
    nxt = t;
  }
}

// ------------------------------------------------------------------ whole 2^13 rows
// The common case tc = 13 (signals of 2^13 elements or more): one 256-thread CTA per row,
// the row brought in by one TMA load (SWIZZLE_128B), 32 consecutive elements per thread.
// Levels 1-5 run in each thread's registers and write their details with 16-byte stores;
// the 256 level-5 approximations go through shared memory to warp 0, which does levels
// 6-8 in registers and 9-13 with warp shuffles.  The synthesis runs the same steps
// backwards and writes its row with one TMA store.  Same butterflies, same order, as the
// generic pass kernels above.

// Chunk j (16 bytes) of 128-byte row t of a SWIZZLE_128B tile sits at chunk j ^ (t mod 8).
__device__ __forceinline__ uint32_t* swz_chunk(uint32_t* tile, uint32_t t, uint32_t j) {
  return tile + t * 32u + ((j ^ (t & 7u)) << 2);
}

template <class BF, bool END>
__global__ void __launch_bounds__(kHaarThreads) haar_fwd_row_kernel(const __grid_constant__ CUtensorMap tin,
                                                                   const HaarFwdArgs p) {
  __shared__ __align__(1024) uint32_t tile[1 << kHaarRowBits];
  __shared__ uint32_t apx[kHaarThreads];
  __shared__ uint64_t bar;
  BF bf{};
  if constexpr (std::is_same_v<BF, BfF32PerLevel>) bf.c = 0.70710678118654752440f;
  const uint32_t t = threadIdx.x, lane = t & 31u;
  const int64_t r = blockIdx.x;
  if (t == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&bar, 4u << kHaarRowBits);
    tma_load_2d(tile, &tin, &bar, 0, static_cast<int>(r << (kHaarRowBits - 5)), policy_evict_first());
  }
  __syncthreads();
  if (!mbar_wait_bounded(&bar, 0, kWaitTries) && lane == 0) atomicCAS(p.status, 0, kStatusTimeout);
  const int cbits = p.mlen - kHaarRowBits;
  const int64_t s = r >> cbits, c = r & ((int64_t{1} << cbits) - 1);
  uint32_t* out = p.out + s * p.out_stride;
  auto dpos = [&](int l) { return (int64_t{1} << (p.mlen - l)) + (c << (kHaarRowBits - l)); };
  uint32_t v[32];
#pragma unroll
  for (uint32_t j = 0; j < 8; ++j) {
    const uint4 q = *reinterpret_cast<const uint4*>(swz_chunk(tile, t, j));
    v[4 * j] = q.x;
    v[4 * j + 1] = q.y;
    v[4 * j + 2] = q.z;
    v[4 * j + 3] = q.w;
  }
  // levels 1..5: 16, 8, 4, 2, 1 details per thread
#pragma unroll
  for (int l = 1; l <= 5; ++l) {
    const int h = 32 >> l;
    const float sc = END ? end_scale_dev(p.lev0 + l) : 1.0f;
    uint32_t d[16];
#pragma unroll
    for (int i = 0; i < h; ++i) {
      uint32_t a = v[2 * i], b = v[2 * i + 1];
      bf(a, b);
      v[i] = a;
      d[i] = END ? scale_u32(b, sc) : b;
    }
    uint32_t* o = out + dpos(l) + static_cast<int64_t>(t) * h;
    if (h >= 4) {
#pragma unroll
      for (int i = 0; i < h; i += 4) st_global_v4(o + i, d[i], d[i + 1], d[i + 2], d[i + 3]);
    } else if (h == 2) {
      *reinterpret_cast<uint2*>(o) = make_uint2(d[0], d[1]);
    } else {
      o[0] = d[0];
    }
  }
  apx[t] = v[0];
  __syncthreads();
  if (t >= 32) return;
  // levels 6..8 in registers (8 approximations per lane), then 9..13 by shuffles
  uint32_t w[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) w[i] = apx[8 * lane + i];
#pragma unroll
  for (int l = 6; l <= 8; ++l) {
    const int h = 256 >> l;  // 4, 2, 1 per lane
    const float sc = END ? end_scale_dev(p.lev0 + l) : 1.0f;
    uint32_t d[4];
#pragma unroll
    for (int i = 0; i < h; ++i) {
      uint32_t a = w[2 * i], b = w[2 * i + 1];
      bf(a, b);
      w[i] = a;
      d[i] = END ? scale_u32(b, sc) : b;
    }
    uint32_t* o = out + dpos(l) + static_cast<int64_t>(lane) * h;
    if (h == 4) {
      st_global_v4(o, d[0], d[1], d[2], d[3]);
    } else if (h == 2) {
      *reinterpret_cast<uint2*>(o) = make_uint2(d[0], d[1]);
    } else {
      o[0] = d[0];
    }
  }
  uint32_t x = w[0];
#pragma unroll
  for (int l = 9; l <= 13; ++l) {
    const uint32_t step = 1u << (l - 9);
    const uint32_t y = __shfl_down_sync(0xffffffffu, x, step);
    if ((lane & (2 * step - 1)) == 0) {
      uint32_t a = x, b = y;
      bf(a, b);
      x = a;
      if constexpr (END) b = scale_u32(b, end_scale_dev(p.lev0 + l));
      out[dpos(l) + (lane >> (l - 8))] = b;
    }
  }
  if (lane == 0) {
    if (p.approx != nullptr) {
      p.approx[r] = x;
    } else {
      if constexpr (END) x = scale_u32(x, end_scale_dev(p.mtotal));
      out[0] = x;
    }
  }
  if (t == 0) mbar_wait_bounded(&bar, 0, kWaitTries);  // the row load is not in flight at exit
}

template <class BF, bool END>
__global__ void __launch_bounds__(kHaarThreads) haar_inv_row_kernel(const __grid_constant__ CUtensorMap tout,
                                                                   const HaarInvArgs p) {
  __shared__ __align__(1024) uint32_t tile[1 << kHaarRowBits];
  __shared__ uint32_t apx[kHaarThreads];
  BF bf{};
  if constexpr (std::is_same_v<BF, BfF32PerLevel>) bf.c = 0.70710678118654752440f;
  const uint32_t t = threadIdx.x, lane = t & 31u;
  const int64_t r = blockIdx.x;
  const int cbits = p.mlen - kHaarRowBits;
  const int64_t s = r >> cbits, c = r & ((int64_t{1} << cbits) - 1);
  const uint32_t* zs = p.z + s * p.z_stride;
  auto dpos = [&](int l) { return (int64_t{1} << (p.mlen - l)) + (c << (kHaarRowBits - l)); };
  // Every thread first loads the details of its own levels 5..1 (16+8+4+2+1 values, used
  // after the barrier) so that their latency overlaps warp 0's coarse levels.
  uint32_t dl[31];  // level l's 2^(5-l) details at dl[(32 >> l) - 1 ...]
#pragma unroll
  for (int l = 1; l <= 5; ++l) {
    const int h = 32 >> l;
    const uint32_t* dz = zs + dpos(l) + static_cast<int64_t>(t) * h;
    uint32_t* d = dl + (h - 1);
    if (h >= 4) {
#pragma unroll
      for (int i = 0; i < h; i += 4) {
        const uint4 q = __ldcs(reinterpret_cast<const uint4*>(dz + i));
        d[i] = q.x;
        d[i + 1] = q.y;
        d[i + 2] = q.z;
        d[i + 3] = q.w;
      }
    } else if (h == 2) {
      const uint2 q = *reinterpret_cast<const uint2*>(dz);
      d[0] = q.x;
      d[1] = q.y;
    } else {
      d[0] = dz[0];
    }
  }
  if (t < 32) {
    // all of warp 0's coarse details first: levels 13..9 (one per participating lane),
    // then levels 8..6 (1, 2, 4 per lane)
    uint32_t dc[5];
#pragma unroll
    for (int l = 13; l >= 9; --l) {
      const uint32_t step = 1u << (l - 9);
      dc[l - 9] = (lane & (2 * step - 1)) == 0 ? zs[dpos(l) + (lane >> (l - 8))] : 0u;
    }
    uint32_t dm[7];  // level 8: dm[0]; level 7: dm[1..2]; level 6: dm[3..6]
    dm[0] = zs[dpos(8) + lane];
    {
      const uint2 q = *reinterpret_cast<const uint2*>(zs + dpos(7) + 2 * static_cast<int64_t>(lane));
      dm[1] = q.x;
      dm[2] = q.y;
      const uint4 u = *reinterpret_cast<const uint4*>(zs + dpos(6) + 4 * static_cast<int64_t>(lane));
      dm[3] = u.x;
      dm[4] = u.y;
      dm[5] = u.z;
      dm[6] = u.w;
    }
    uint32_t x = 0;
    if (lane == 0) {
      if (p.approx != nullptr) {
        x = p.approx[r];
      } else {
        x = zs[0];
        if constexpr (END) x = scale_u32(x, end_scale_dev(p.mtotal));
      }
    }
    // levels 13..9 by shuffles: lane L holds the approximation of group L at each level
#pragma unroll
    for (int l = 13; l >= 9; --l) {
      const uint32_t step = 1u << (l - 9);
      uint32_t e = x, o = 0;
      if ((lane & (2 * step - 1)) == 0) {
        o = dc[l - 9];
        if constexpr (END) o = scale_u32(o, end_scale_dev(p.lev0 + l));
        bf(e, o);
      }
      const uint32_t y = __shfl_up_sync(0xffffffffu, o, step);
      x = (lane & (2 * step - 1)) == 0 ? e : ((lane & (2 * step - 1)) == step ? y : x);
    }
    // levels 8..6 in registers
    uint32_t w[8];
    w[0] = x;
#pragma unroll
    for (int l = 8; l >= 6; --l) {
      const int h = 256 >> l;  // 1, 2, 4 details per lane
      const uint32_t* d = dm + (h - 1);
      const float sc = END ? end_scale_dev(p.lev0 + l) : 1.0f;
#pragma unroll
      for (int i = h - 1; i >= 0; --i) {
        uint32_t e = w[i], o = END ? scale_u32(d[i], sc) : d[i];
        bf(e, o);
        w[2 * i] = e;
        w[2 * i + 1] = o;
      }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) apx[8 * lane + i] = w[i];
  }
  __syncthreads();
  // levels 5..1 in each thread's registers
  uint32_t v[32];
  v[0] = apx[t];
#pragma unroll
  for (int l = 5; l >= 1; --l) {
    const int h = 32 >> l;  // 1, 2, 4, 8, 16 details per thread
    const uint32_t* d = dl + (h - 1);
    const float sc = END ? end_scale_dev(p.lev0 + l) : 1.0f;
#pragma unroll
    for (int i = h - 1; i >= 0; --i) {
      uint32_t e = v[i], o = END ? scale_u32(d[i], sc) : d[i];
      bf(e, o);
      v[2 * i] = e;
      v[2 * i + 1] = o;
    }
  }
#pragma unroll
  for (uint32_t j = 0; j < 8; ++j)
    *reinterpret_cast<uint4*>(swz_chunk(tile, t, j)) = make_uint4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
  __syncthreads();
  if (t == 0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the row's generic writes, to TMA
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(&tout), "r"(0),
                 "r"(static_cast<int>(r << (kHaarRowBits - 5))), "r"(smem_u32(tile))
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
  }
}

}  // namespace chw
