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

// ------------------------------------------------------------------ one warp per signal
// The 2^12 form as one warp per signal, 128 values per thread, in two register phases:
//   phase 1: registers carry label bits 0..5 and 11, lanes bits 6..10 (thread l owns
//            rows l and l + 32 of the 64 x 64-code input tile), butterflies of bits 0..5;
//   phase 2: registers carry label bits 0, 11, 6..10, lanes bits 5, 4, 3, 2, 1,
//            butterflies of bits 6..11.
// Both phases hold label bits 0 and 11 in registers, so the exchange between them moves
// 16-byte chunks (its layout puts those bits on word bits 0, 1), and its XOR swizzle keeps
// the eight lanes of every quarter warp on distinct 16-byte bank groups on both sides.
// Phase 2 leaves thread l with the outputs of rows l and l + 32 of the 64 x 64-code output
// tile (dyadic output o = bitrev_12(label), row o >> 6), quantised and staged in the TMA
// SWIZZLE_128B layout and written by one tensor store per signal.  No CTA barrier: a CTA is
// one warp, persistent over signals, with 24 KB of shared memory -- two 8 KB code tiles
// (the TMA load of the next signal lands in one while this one is transformed) and 8 KB in
// between, so that a signal's 16 KB fp32 exchange covers its own tile and the middle part
// (even signals [0, 16K), odd ones [8K, 24K)) and never the other tile.
namespace lw {
constexpr int kTile = 8192;  // bytes of one 2^12-code tile

// Exchange position (fp32 words) of a label: bits 0, 1 = labels 0, 11; bits 2..4 = labels
// 3..5 XOR 6..8; bits 5, 6 = labels 1, 2; bits 7..11 = labels 6..10.
constexpr uint32_t xpos(uint32_t L) {
  auto b = [&](int i) { return (L >> i) & 1u; };
  return b(0) | b(11) << 1 | (b(3) ^ b(6)) << 2 | (b(4) ^ b(7)) << 3 | (b(5) ^ b(8)) << 4 | b(1) << 5 | b(2) << 6 |
         b(6) << 7 | b(7) << 8 | b(8) << 9 | b(9) << 10 | b(10) << 11;
}
// Phase-1 register i: label bits 0..5 = i bits 0..5, label bit 11 = i bit 6.
constexpr uint32_t p1_label(int i) { return (static_cast<uint32_t>(i) & 63u) | ((static_cast<uint32_t>(i) >> 6) << 11); }
// Phase-2 register i: label 0 = i bit 0, label 11 = i bit 1, labels 6..10 = i bits 2..6.
constexpr uint32_t p2_label(int i) {
  const uint32_t u = static_cast<uint32_t>(i);
  return (u & 1u) | ((u >> 1) & 1u) << 11 | ((u >> 2) & 31u) << 6;
}
// Phase-2 lane bits: lane bit k carries label 5 - k.
__host__ __device__ constexpr uint32_t p2_lane_label(uint32_t l) {
  return ((l & 1u) << 5) | ((l >> 1) & 1u) << 4 | ((l >> 2) & 1u) << 3 | ((l >> 3) & 1u) << 2 | ((l >> 4) & 1u) << 1;
}
// The exchange is a bijection and both sides are conflict-free (checked below).
constexpr bool xpos_bijective() {
  bool seen[4096] = {};
  for (uint32_t L = 0; L < 4096; ++L) {
    if (seen[xpos(L)]) return false;
    seen[xpos(L)] = true;
  }
  return true;
}
constexpr bool exchange_conflict_free() {
  for (int i = 0; i < 128; i += 4) {
    // phase 1 writes: lanes 8q..8q+7 carry label bits 6..8 (lane bits 0..2)
    for (uint32_t q = 0; q < 4; ++q) {
      int seen = 0;
      for (uint32_t l = 8 * q; l < 8 * q + 8; ++l) seen |= 1 << ((xpos(p1_label(i) | (l << 6)) >> 2) & 7u);
      if (seen != 0xff) return false;
    }
    for (uint32_t q = 0; q < 4; ++q) {
      int seen = 0;
      for (uint32_t l = 8 * q; l < 8 * q + 8; ++l) seen |= 1 << ((xpos(p2_label(i) | p2_lane_label(l)) >> 2) & 7u);
      if (seen != 0xff) return false;
    }
  }
  return true;
}
static_assert(xpos_bijective() && exchange_conflict_free(), "the 2^12 exchange layout");
// 16-byte chunks: phase-1 registers {i, i|1, i|64, i|65} and phase-2 registers {i..i+3}
// are the words 0..3 of one chunk.
static_assert(xpos(p1_label(1)) == 1 && xpos(p1_label(64)) == 2 && xpos(p2_label(1)) == 1 && xpos(p2_label(2)) == 2,
              "labels 0 and 11 on word bits 0, 1");
}  // namespace lw

// Two fp32 values to a packed pair of codes (first value in the low half), each rounded to
// nearest even.
template <bool F16>
__device__ __forceinline__ uint32_t pack_codes(float lo, float hi) {
  uint32_t d;  // cvt packs its first source into the upper half
  if constexpr (F16) {
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  } else {
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  }
  return d;
}

// a *= s, b *= s with one f32x2 multiply (each product rounded to nearest even).
__device__ __forceinline__ void mul2(uint32_t& a, uint32_t& b, float s) {
  const uint32_t sb = __float_as_uint(s);
  asm("{\n\t.reg .b64 x, y, z;\n\t"
      "mov.b64 x, {%0, %1};\n\tmov.b64 y, {%2, %2};\n\t"
      "mul.rn.f32x2 z, x, y;\n\t"
      "mov.b64 {%0, %1}, z;\n\t}"
      : "+r"(a), "+r"(b)
      : "r"(sb));
}

constexpr int lowp_warp_smem_bytes() { return 3 * lw::kTile + 1024 + 64; }

template <bool F16, class BF, bool SCALE>
__global__ void __launch_bounds__(32, 9)
    lowp_warp_kernel(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout,
                     const LowpArgs args, const int64_t batch) {
  constexpr int K = F16 ? 14 : 0;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + 3 * lw::kTile);
  const uint32_t lane = threadIdx.x;
  BF bf{};
  if constexpr (std::is_same_v<BF, BfF32PerLevel>) bf.c = 0.70710678118654752440f;
  if (lane == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
    fence_mbar_init();
  }
  __syncwarp();
  auto tile = [&](int b) { return base + (b ? 2 * lw::kTile : 0); };
  auto issue = [&](int64_t sig, int b) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(bar + b, lw::kTile);
    tma_load_2d(tile(b), &tin, bar + b, 0, static_cast<int>(sig * 64), policy_evict_first());
  };
  const int64_t first = blockIdx.x, stride = gridDim.x;
  if (lane == 0 && first < batch) issue(first, 0);
  bool waiting = true;
  const uint32_t lx = lane & 7u;
  const uint32_t xb1 = lw::xpos(lane << 6);                 // phase 1: lanes carry labels 6..10
  const uint32_t xb2 = lw::xpos(lw::p2_lane_label(lane));  // phase 2: lanes carry labels 5..1
  int k = 0;
  for (int64_t sig = first; sig < batch; sig += stride, ++k) {
    const int b = k & 1;
    uint8_t* cur = tile(b);
    uint32_t* ex = reinterpret_cast<uint32_t*>(base + (b ? lw::kTile : 0));
    if (lane == 0 && sig + stride < batch) {
      bulk_wait_read();  // the previous signal's output store has read the other tile
      issue(sig + stride, b ^ 1);
    }
    if (waiting && !mbar_wait_bounded(bar + b, static_cast<uint32_t>((k >> 1) & 1), kWaitTries)) {
      waiting = false;
      atomicCAS(args.status, 0, kStatusTimeout);
    }
    uint32_t v[128];
    // ---- phase 1: rows lane and lane + 32, 16-byte chunk j of a row at j ^ (row mod 8)
    sfor<16>([&](auto cc) {
      constexpr int r0 = cc >> 3, j = cc & 7;
      const uint4 q = *reinterpret_cast<const uint4*>(cur + ((lane + 32u * r0) << 7) + ((j ^ lx) << 4));
      const uint32_t w[4] = {q.x, q.y, q.z, q.w};
      sfor<4>([&](auto hh) {
        constexpr int h = hh;
        constexpr int i = 64 * r0 + 8 * j + 2 * h;  // register of the even code (column 8j + 2h)
        if constexpr (F16) {
          const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[h]));
          v[i] = __float_as_uint(f.x);
          v[i + 1] = __float_as_uint(f.y);
        } else {
          v[i] = w[h] << 16;
          v[i + 1] = w[h] & 0xffff0000u;
        }
      });
    });
    if (args.diag_in != nullptr) {  // D on the input (natural positions = labels)
      sfor<128>([&](auto ii) {
        constexpr int i = ii;
        if (args.diag_in[lw::p1_label(i) | (lane << 6)] < 0) v[i] ^= 0x80000000u;
      });
    }
    sfor<6>([&](auto bb) {  // label bits 0..5 = register bits 0..5, lowest first
      constexpr int bit = bb;
      sfor<128>([&](auto ii) {
        constexpr int i = ii;
        if constexpr (((i >> bit) & 1) == 0) {
          if constexpr (bit == 0 || !BF::kPacked) {
            bf(v[i], v[i | (1 << bit)]);
          } else if constexpr ((i & 1) == 0) {
            bf.pair(v[i], v[i | 1], v[i | (1 << bit)], v[i | 1 | (1 << bit)]);
          }
        }
      });
    });
    __syncwarp();  // every lane has read its codes: the exchange covers this tile
    sfor<32>([&](auto gg) {
      constexpr int i = 2 * gg;  // register bits 1..5; the chunk's words are i, i|1, i|64, i|65
      constexpr uint32_t kp = lw::xpos(lw::p1_label(i));
      *reinterpret_cast<uint4*>(ex + (xb1 ^ kp)) = make_uint4(v[i], v[i | 1], v[i | 64], v[i | 65]);
    });
    __syncwarp();
    // ---- phase 2: label bits 6..10 on register bits 2..6, then 11 on register bit 1
    sfor<32>([&](auto gg) {
      constexpr int i = 4 * gg;
      constexpr uint32_t kp = lw::xpos(lw::p2_label(i));
      const uint4 q = *reinterpret_cast<const uint4*>(ex + (xb2 ^ kp));
      v[i] = q.x;
      v[i + 1] = q.y;
      v[i + 2] = q.z;
      v[i + 3] = q.w;
    });
    sfor<6>([&](auto tt) {
      constexpr int rb = tt == 5 ? 1 : tt + 2;
      sfor<128>([&](auto ii) {
        constexpr int i = ii;
        if constexpr (((i >> rb) & 1) == 0) {
          if constexpr (!BF::kPacked) {
            bf(v[i], v[i | (1 << rb)]);
          } else if constexpr ((i & 1) == 0) {
            bf.pair(v[i], v[i | 1], v[i | (1 << rb)], v[i | 1 | (1 << rb)]);
          }
        }
      });
    });
    if constexpr (SCALE) {
      sfor<64>([&](auto kk) { mul2(v[2 * kk], v[2 * kk + 1], args.end_scale); });
    }
    float mx = 0.f;
    sfor<128>([&](auto ii) { mx = fmaxf(mx, fabsf(__uint_as_float(v[ii]))); });
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int e_in = args.exp_in[sig];
    int shift = 0;
    if (mx != 0.f) {
      const int E = floor_log2_f32(mx);
      shift = K - E;
      if (lane == 0) args.exp_out[sig] = e_in + E - K;
    } else if (lane == 0) {
      args.exp_out[sig] = e_in;
    }
    // u * 2^shift as scale_pow2 forms it: one multiply inside fp32's normal range, else two
    if (shift >= -126 && shift <= 127) {
      const float f = pow2_f32(shift);
      sfor<64>([&](auto kk) { mul2(v[2 * kk], v[2 * kk + 1], f); });
    } else {
      const int h = shift / 2;
      const float f1 = pow2_f32(h), f2 = pow2_f32(shift - h);
      sfor<64>([&](auto kk) {
        mul2(v[2 * kk], v[2 * kk + 1], f1);
        mul2(v[2 * kk], v[2 * kk + 1], f2);
      });
    }
    // ---- output: dyadic o = bitrev_12(label); this thread holds rows lane and lane + 32
    // (label 0 = row bit 5) of the 64 x 64 output tile; column bits 0..5 are labels 11..6 =
    // register bits 1, 6, 5, 4, 3, 2
    __syncwarp();  // every lane has read the exchange: the staging tile lies inside it
    sfor<16>([&](auto cc) {
      constexpr int r0 = cc >> 3, j = cc & 7;  // row half, 16-byte chunk (column bits 3..5)
      uint32_t w[4];
      sfor<4>([&](auto tt) {
        constexpr int t = tt;  // column bits 1, 2
        constexpr int i = r0 | ((j & 1) << 4) | (((j >> 1) & 1) << 3) | (((j >> 2) & 1) << 2) | ((t & 1) << 6) |
                          (((t >> 1) & 1) << 5);
        w[t] = pack_codes<F16>(__uint_as_float(v[i]), __uint_as_float(v[i | 2]));
      });
      const uint32_t row = lane + 32u * r0;
      if (args.diag_out != nullptr) {  // D on the stored positions
        const int8_t* d = args.diag_out + row * 64 + 8 * j;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          if (d[2 * t] < 0) w[t] ^= 0x8000u;
          if (d[2 * t + 1] < 0) w[t] ^= 0x80000000u;
        }
      }
      *reinterpret_cast<uint4*>(cur + (row << 7) + ((j ^ lx) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
    });
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) {
      tma_store_2d(&tout, cur, 0, static_cast<int>(sig * 64));
      bulk_commit_group();
    }
  }
  // no TMA load or store left in flight on shared memory, even after a wait gave up
  if (lane == 0) {
    bulk_wait_all();
    for (int b = 0; b < 2 && b < k; ++b) {
      const int kl = b + ((k - 1 - b) / 2) * 2;
      mbar_wait_bounded(bar + b, static_cast<uint32_t>((kl >> 1) & 1), kWaitTries);
    }
  }
}

template <bool F16, class BF, bool SCALE>
cudaError_t launch_lowp_warp(const CUtensorMap* tin, const CUtensorMap* tout, const LowpArgs& args, int64_t batch,
                             cudaStream_t st) {
  auto kern = lowp_warp_kernel<F16, BF, SCALE>;
  constexpr int smem = lowp_warp_smem_bytes();
  static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (attr != cudaSuccess) return attr;
  static const int64_t resident = [&] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 32, smem);
    return static_cast<int64_t>(per) * sms;
  }();
  const int64_t grid = resident > 0 && batch > resident ? resident : batch;
  kern<<<static_cast<unsigned>(grid), 32, smem, st>>>(*tin, *tout, args, batch);
  return cudaGetLastError();
}

template <int M, bool F16, class BF, bool SCALE>
cudaError_t launch_lowp(const CUtensorMap* tin, const CUtensorMap* /*tout: the codes leave by 16-byte stores*/,
                        const LowpArgs& args, int64_t batch, cudaStream_t st) {
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
