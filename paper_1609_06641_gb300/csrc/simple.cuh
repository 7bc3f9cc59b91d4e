// Plain CHW kernel: one CTA per signal, the whole signal in shared memory as fp32 (or
// int32), one __syncthreads per butterfly level.  It covers shapes the fused kernel does
// not take (tiny signals whose batch is not a whole number of 128-byte rows) and the
// bf16/fp16 storage form (per-signal exponent, m <= 13).  Same butterflies, same order:
// level t pairs labels differing in bit t, lowest bit first (Theorem 1; see engine.cuh).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

namespace chw {

enum SimpleDtype { kSimpleI32 = 0, kSimpleF32 = 1, kSimpleBF16 = 2, kSimpleF16 = 3 };
enum SimpleNorm { kNormNone = 0, kNormPerLevel = 1, kNormEnd = 2 };

struct SimpleArgs {
  const void* x;
  void* y;
  int m;
  int64_t batch;
  int norm;
  float end_scale;
  const int32_t* exp_in;
  int32_t* exp_out;
  const int8_t* diag_in;
  const int8_t* diag_out;
  int order;  // output order: 0 dyadic, 1 natural, 2 sequency
};

// floor(log2 v) for a finite v > 0, read from the fp32 encoding (exact, subnormals too).
__device__ __forceinline__ int floor_log2_f32(float v) {
  const uint32_t b = __float_as_uint(v) & 0x7fffffffu;
  const int ex = static_cast<int>(b >> 23);
  if (ex > 0) return ex - 127;
  return (31 - __clz(static_cast<int>(b))) - 149;
}

__device__ __forceinline__ float pow2_f32(int k) {  // 2^k for -126 <= k <= 127
  return __uint_as_float(static_cast<uint32_t>(k + 127) << 23);
}

// u * 2^k in fp32; two multiplies when 2^k is outside fp32's normal range.
__device__ __forceinline__ float scale_pow2(float u, int k) {
  if (k >= -126 && k <= 127) return __fmul_rn(u, pow2_f32(k));
  const int h = k / 2;
  return __fmul_rn(__fmul_rn(u, pow2_f32(h)), pow2_f32(k - h));
}

template <int DT>
__global__ void __launch_bounds__(256) simple_kernel(const SimpleArgs a) {
  extern __shared__ __align__(16) uint32_t s[];
  __shared__ float red[8];
  const int m = a.m;
  const int64_t n = int64_t{1} << m;
  const int64_t sig = blockIdx.x;
  const int tid = threadIdx.x;
  constexpr bool kInt = DT == kSimpleI32;
  constexpr bool kLowp = DT == kSimpleBF16 || DT == kSimpleF16;

  // load (and convert) one signal
  for (int64_t i = tid; i < n; i += blockDim.x) {
    const int64_t g = sig * n + i;
    uint32_t v;
    if constexpr (DT == kSimpleI32 || DT == kSimpleF32) {
      v = static_cast<const uint32_t*>(a.x)[g];
    } else if constexpr (DT == kSimpleBF16) {
      v = __float_as_uint(__bfloat162float(static_cast<const __nv_bfloat16*>(a.x)[g]));
    } else {
      v = __float_as_uint(__half2float(static_cast<const __half*>(a.x)[g]));
    }
    if (a.diag_in != nullptr && a.diag_in[i] < 0) v = kInt ? 0u - v : v ^ 0x80000000u;
    s[i] = v;
  }
  const float c = 0.70710678118654752440f;
  for (int t = 0; t < m; ++t) {
    __syncthreads();
    const int64_t lowmask = (int64_t{1} << t) - 1;
    for (int64_t p = tid; p < n / 2; p += blockDim.x) {
      const int64_t i0 = ((p & ~lowmask) << 1) | (p & lowmask);
      const int64_t i1 = i0 | (int64_t{1} << t);
      const uint32_t x0 = s[i0], x1 = s[i1];
      if constexpr (kInt) {
        s[i0] = x0 + x1;
        s[i1] = x0 - x1;
      } else {
        const float f0 = __uint_as_float(x0), f1 = __uint_as_float(x1);
        float r0 = __fadd_rn(f0, f1), r1 = __fsub_rn(f0, f1);
        if (a.norm == kNormPerLevel) {
          r0 = __fmul_rn(r0, c);
          r1 = __fmul_rn(r1, c);
        }
        s[i0] = __float_as_uint(r0);
        s[i1] = __float_as_uint(r1);
      }
    }
  }
  __syncthreads();
  if constexpr (!kInt) {
    if (a.norm == kNormEnd) {
      for (int64_t i = tid; i < n; i += blockDim.x) s[i] = __float_as_uint(__fmul_rn(__uint_as_float(s[i]), a.end_scale));
      __syncthreads();
    }
  }

  int shift = 0;  // lowp: codes = u * 2^shift
  if constexpr (kLowp) {
    float mx = 0.f;
    for (int64_t i = tid; i < n; i += blockDim.x) mx = fmaxf(mx, fabsf(__uint_as_float(s[i])));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((tid & 31) == 0) red[tid >> 5] = mx;
    __syncthreads();
    if (tid < 32) {
      float r = tid < static_cast<int>(blockDim.x >> 5) ? red[tid] : 0.f;
      for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
      if (tid == 0) red[0] = r;
    }
    __syncthreads();
    const float big = red[0];
    constexpr int K = DT == kSimpleBF16 ? 0 : 14;
    const int e_in = a.exp_in[sig];
    if (big == 0.f) {
      if (tid == 0) a.exp_out[sig] = e_in;
      shift = 0;
    } else {
      const int E = floor_log2_f32(big);
      shift = K - E;
      if (tid == 0) a.exp_out[sig] = e_in + E - K;
    }
  }

  // store: the value of label j is the dyadic output bitrev_m(j), so dyadic output k holds
  // label bitrev_m(k), natural output k label k, and sequency output k (= dyadic output
  // gray(k)) label bitrev_m(k ^ (k >> 1))
  const int rs = m == 0 ? 0 : 32 - m;  // __brev(v) >> rs reverses the low m bits (m >= 1)
  for (int64_t k = tid; k < n; k += blockDim.x) {
    int64_t lab = 0;
    if (m > 0) {
      const uint32_t kk = static_cast<uint32_t>(k);
      const uint32_t d = a.order == 1 ? __brev(kk) >> rs : (a.order == 2 ? kk ^ (kk >> 1) : kk);
      lab = static_cast<int64_t>(__brev(d) >> rs);
    }
    uint32_t v = s[lab];
    if (a.diag_out != nullptr && a.diag_out[k] < 0) v = kInt ? 0u - v : v ^ 0x80000000u;
    const int64_t g = sig * n + k;
    if constexpr (DT == kSimpleI32 || DT == kSimpleF32) {
      static_cast<uint32_t*>(a.y)[g] = v;
    } else if constexpr (DT == kSimpleBF16) {
      static_cast<__nv_bfloat16*>(a.y)[g] = __float2bfloat16_rn(scale_pow2(__uint_as_float(v), shift));
    } else {
      static_cast<__half*>(a.y)[g] = __float2half_rn(scale_pow2(__uint_as_float(v), shift));
    }
  }
}

}  // namespace chw
