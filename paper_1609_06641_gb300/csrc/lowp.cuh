// Fused CHW kernel for bf16/fp16 storage with fp32 accumulation and a per-signal
// power-of-two exponent (one signal of 2^M elements per tile, M = 11 or 12).
//
// Storage form: a signal is (q, e) meaning 2^e q.  The kernel loads q by TMA (rows of 64
// 2-byte codes, SWIZZLE_128B), widens to fp32 (exact), runs the cascade's butterflies in
// two register phases (label bits 0-5, then 6..M-1) through an fp32 exchange buffer,
// reduces max|u| over the signal, and writes
//   e_out = e_in + E - K,   q_out = round(u * 2^(K - E)),   E = floor(log2 max|u|),
// with K = 0 for bf16 and 14 for fp16 (so max|q_out| lies in [2^K, 2^(K+1))).  The codes
// are staged in shared memory and stored with coalesced 16-byte writes.  Persistent CTAs
// walk the signals with two input buffers (the next signal's TMA load is in flight while
// the current one is transformed).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fused.cuh"
#include "simple.cuh"

namespace chw {

struct LowpArgs {
  void* out;              // 2-byte codes, batch * 2^M
  const int32_t* exp_in;  // batch
  int32_t* exp_out;       // batch
  float end_scale;        // used when the kernel's SCALE is set
  const int8_t* diag_in;  // +-1 on the input (adjoint's D) or nullptr
  const int8_t* diag_out; // +-1 on the output (forward's D) or nullptr
  int* status;
};

// Exchange layout (fp32 words): bank bits 0..4 XOR label bits 6..10.
constexpr Lin lin_lowp_exchange() {
  Lin l = lin_identity();
  for (int i = 6; i < 11; ++i) l.img[i] |= 1u << (i - 6);
  return l;
}

template <int M>
struct LowpCfg {
  static_assert(M == 11 || M == 12, "the fused 16-bit kernel takes one signal of 2^11 or 2^12 per tile");
  static constexpr int TB = M;
  static constexpr int NT = 1 << (TB - 6);
  static constexpr uint32_t LMASK = (1u << TB) - 1u;
  static constexpr Phase make1() {
    Phase p{};
    p.nreg = 6;
    for (int i = 0; i < 6; ++i) p.reg[i] = i;
    for (int i = 0; i < 5; ++i) p.lane[i] = 6 + i;
    p.nwarp = TB - 11;
    for (int i = 0; i < p.nwarp; ++i) p.warp[i] = 11 + i;
    return p;
  }
  // registers 0..2 hold output bits 0..2 (labels M-1, M-2, M-3) for 8-code chunks
  static constexpr Phase make2() {
    Phase p{};
    p.nreg = 6;
    for (int i = 0; i < 6; ++i) p.reg[i] = M - 1 - i;
    const int l[5] = {4, 3, 2, 1, 0};
    for (int i = 0; i < 5; ++i) p.lane[i] = l[i];
    p.nwarp = 0;
    for (int b = 5; b < TB; ++b) {
      bool used = false;
      for (int i = 0; i < 6; ++i) used |= p.reg[i] == b;
      if (!used) p.warp[p.nwarp++] = b;
    }
    return p;
  }
  static constexpr Phase P1 = make1();
  static constexpr Phase P2 = make2();
  static constexpr Lin LE = lin_lowp_exchange();
  // input TMA layout on 2-byte codes: 16-byte chunk (code bits 3..5) XOR row (bits 6..8)
  static constexpr int S = M - 5;  // staging key: output bits of lanes 0..2 (labels 4, 3, 2)
  static_assert(phase_covers(P1, TB) && phase_covers(P2, TB), "phases cover the tile");
  static_assert(conflict_degree(P1, LE, LMASK, false) == 1, "phase 1 exchange writes are conflict-free");
  static_assert(conflict_degree(P2, LE, LMASK, false) == 1, "phase 2 exchange reads are conflict-free");
};

__device__ __forceinline__ float code_to_f32(uint32_t c, bool f16) {
  return f16 ? __half2float(__ushort_as_half(static_cast<unsigned short>(c))) : __uint_as_float(c << 16);
}
__device__ __forceinline__ uint32_t f32_to_code(float v, bool f16) {
  return f16 ? __half_as_ushort(__float2half_rn(v)) : __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

template <int M>
constexpr int lowp_smem_bytes() {
  return 2 * (2 << M) + (4 << M) + 1024 + 64;  // two code tiles, fp32 exchange, slack, barriers
}

template <int M, bool F16, class BF, bool SCALE>
__global__ void __launch_bounds__(1 << (M - 6), 6)
    lowp_kernel(const __grid_constant__ CUtensorMap tin, const LowpArgs args, const int64_t batch) {
  using Cfg = LowpCfg<M>;
  constexpr int TB = M;
  constexpr int NT = Cfg::NT;
  constexpr uint32_t LMASK = Cfg::LMASK;
  constexpr Phase P1 = Cfg::P1, P2 = Cfg::P2;
  constexpr Lin LE = Cfg::LE;
  constexpr int K = F16 ? 14 : 0;
  constexpr int S = Cfg::S;
  constexpr int ROWS = 1 << (TB - 6);  // 64-code rows per tile (<= 128)

  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  uint16_t* tiles[2] = {reinterpret_cast<uint16_t*>(base), reinterpret_cast<uint16_t*>(base + (2u << TB))};
  uint32_t* ex = reinterpret_cast<uint32_t*>(base + (4u << TB));
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + (8u << TB));
  __shared__ float red[32];

  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  BF bf{};
  if constexpr (std::is_same_v<BF, BfF32PerLevel>) bf.c = 0.70710678118654752440f;
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto issue = [&](int64_t sig, uint16_t* dst, uint64_t* b) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(b, 2u << TB);
    tma_load_2d(dst, &tin, b, 0, static_cast<int>(sig * ROWS), policy_evict_first());
  };
  const int64_t first = blockIdx.x, stride = gridDim.x;
  if (tid == 0 && first < batch) issue(first, tiles[0], bar);
  int k = 0;
  for (int64_t sig = first; sig < batch; sig += stride, ++k) {
    uint16_t* cur = tiles[k & 1];
    if (tid == 0 && sig + stride < batch) issue(sig + stride, tiles[(k + 1) & 1], bar + ((k + 1) & 1));
    if (!mbar_wait_bounded(bar + (k & 1), (k >> 1) & 1, kWaitTries)) {
      if (lane == 0) atomicCAS(args.status, 0, kStatusTimeout);
    }
    uint32_t v[64];
    // ---- phase 1: 64 consecutive codes per thread (label bits 0..5), 8 chunks of 16 B
    {
      const uint32_t row = thread_label<P1>(lane, warp, 0) >> 6;  // lanes/warps own the rows
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint32_t chunk = static_cast<uint32_t>(j) ^ (row & 7u);
        const uint4 q = *reinterpret_cast<const uint4*>(cur + row * 64 + chunk * 8);
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          v[8 * j + 2 * h] = __float_as_uint(code_to_f32(w[h] & 0xffffu, F16));
          v[8 * j + 2 * h + 1] = __float_as_uint(code_to_f32(w[h] >> 16, F16));
        }
      }
      if (args.diag_in != nullptr) {
#pragma unroll
        for (int i = 0; i < 64; ++i)
          if (args.diag_in[row * 64 + i] < 0) v[i] ^= 0x80000000u;
      }
      butterflies<P1, 0, 6>(v, bf);
      store_phase<P1, P1, LE, LMASK>(v, ex, thread_pos<P1, LE, LMASK>(lane, warp, 0));
    }
    __syncthreads();
    // ---- phase 2: label bits 6..M-1
    load_phase<P2, LE, LMASK>(v, ex, thread_pos<P2, LE, LMASK>(lane, warp, 0));
    butterflies<P2, 6, M>(v, bf);
    float mx = 0.f;
#pragma unroll
    for (int i = 0; i < 64; ++i) {
      if constexpr (SCALE) v[i] = __float_as_uint(__fmul_rn(__uint_as_float(v[i]), args.end_scale));
      mx = fmaxf(mx, fabsf(__uint_as_float(v[i])));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    float big = red[0];
#pragma unroll
    for (int w = 1; w < NT / 32; ++w) big = fmaxf(big, red[w]);
    const int e_in = args.exp_in[sig];
    int shift = 0;
    if (big != 0.f) {
      const int E = floor_log2_f32(big);
      shift = K - E;
      if (tid == 0) args.exp_out[sig] = e_in + E - K;
    } else if (tid == 0) {
      args.exp_out[sig] = e_in;
    }
    // ---- stage codes in output order; output index of label j is bitrev_M(j)
    {
      const uint32_t tl = thread_label<P2>(lane, warp, 0);
      const uint32_t o_thread = (__brev(tl) >> (32 - M)) & ~63u;  // register bits carry output bits 0..5
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const uint32_t lo = f32_to_code(scale_pow2(__uint_as_float(v[8 * j + 2 * h]), shift), F16);
          const uint32_t hi = f32_to_code(scale_pow2(__uint_as_float(v[8 * j + 2 * h + 1]), shift), F16);
          w[h] = lo | (hi << 16);
        }
        const uint32_t o = o_thread | (static_cast<uint32_t>(j) << 3);
        const uint32_t pos = o ^ (((o >> S) & 7u) << 3);
        *reinterpret_cast<uint4*>(cur + pos) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    __syncthreads();
    // ---- copy-out: 16-byte chunks of 8 codes
    uint16_t* out = static_cast<uint16_t*>(args.out) + (sig << M);
#pragma unroll 2
    for (int c = tid; c < (1 << (M - 3)); c += NT) {
      const uint32_t o = static_cast<uint32_t>(c) << 3;
      const uint32_t pos = o ^ (((o >> S) & 7u) << 3);
      uint4 q = *reinterpret_cast<const uint4*>(cur + pos);
      if (args.diag_out != nullptr) {
        uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          if (args.diag_out[o + 2 * h] < 0) w[h] ^= 0x8000u;
          if (args.diag_out[o + 2 * h + 1] < 0) w[h] ^= 0x80000000u;
        }
        q = make_uint4(w[0], w[1], w[2], w[3]);
      }
      st_global_v4(out + o, q.x, q.y, q.z, q.w);
    }
    __syncthreads();
  }
  // no TMA load left in flight into shared memory, even after a wait gave up
  if (tid == 0) {
    for (int b = 0; b < 2 && b < k; ++b) {
      const int kl = b + ((k - 1 - b) / 2) * 2;
      mbar_wait_bounded(bar + b, (kl >> 1) & 1, kWaitTries);
    }
  }
}

template <int M, bool F16, class BF, bool SCALE>
cudaError_t launch_lowp(const CUtensorMap* tin, const LowpArgs& args, int64_t batch, cudaStream_t st) {
  auto kern = lowp_kernel<M, F16, BF, SCALE>;
  constexpr int smem = lowp_smem_bytes<M>();
  static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (attr != cudaSuccess) return attr;
  static const int64_t resident = [&] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 1 << (M - 6), smem);
    return static_cast<int64_t>(per) * sms;
  }();
  const int64_t grid = resident > 0 && batch > resident ? resident : batch;
  kern<<<static_cast<unsigned>(grid), 1 << (M - 6), smem, st>>>(*tin, args, batch);
  return cudaGetLastError();
}

}  // namespace chw
