// Register/shared-memory engine for the CHW butterfly graph.
//
// Indexing.  Inside a CTA (or a thread-block cluster) every element carries a *label*:
// its natural-order index within the tile.  The cascade of Theorem 1 (eq. (3)) performs,
// for t = 0, 1, ..., m-1, one butterfly (a, b) -> (a+b, a-b) (times c = 1/sqrt2 in the
// per-level normalisation) between the two elements whose labels differ in bit t, with
// the bit-0 element as the first operand: level t of Psi_m and of the later stages pairs
// exactly those elements, and stage r's Psi_{m-r} on the second halves completes bit t
// for the remaining labels.  Each value passes through bits 0, 1, ..., m-1 in that order,
// so any schedule that keeps this order per value performs the same butterflies on the
// same operands and rounds exactly like the cascade in stage order.  The output index of
// label j is bitrev_m(j) (dyadic order; eq. (1) puts the first butterfly's output bit on
// the most significant row bit).
//
// A *phase* holds 64 values per thread in registers.  Its register-index bits, lane
// bits, warp bits and (in a cluster) CTA-rank bits each name one label bit.  A phase
// loads its 64 values from shared memory, runs the butterflies of its label-bit range in
// registers, and stores them back.  Shared-memory layouts are GF(2)-linear maps from
// labels to word positions (XOR swizzles), so each access is a per-thread base XOR a
// compile-time constant per register, and bank conflicts can be checked at compile time
// (static_assert below).
#pragma once

#include <cstdint>
#include <type_traits>
#include <utility>

#include "ptx.cuh"

namespace chw {

constexpr int kMaxBits = 24;

// ------------------------------------------------------------------ linear layouts
struct Lin {
  uint32_t img[kMaxBits];
};

constexpr Lin lin_identity() {
  Lin l{};
  for (int i = 0; i < kMaxBits; ++i) l.img[i] = 1u << i;
  return l;
}

constexpr uint32_t apply(const Lin& l, uint32_t x) {
  uint32_t p = 0;
  for (int i = 0; i < kMaxBits; ++i)
    if ((x >> i) & 1u) p ^= l.img[i];
  return p;
}

constexpr Lin compose(const Lin& outer, const Lin& inner) {
  Lin l{};
  for (int i = 0; i < kMaxBits; ++i) l.img[i] = apply(outer, inner.img[i]);
  return l;
}

// The TMA SWIZZLE_128B pattern on 4-byte words: the 16-byte chunk index (word bits 2..4)
// is XORed with the 128-byte row index modulo 8 (word bits 5..7).
constexpr Lin lin_tma128() {
  Lin l = lin_identity();
  for (int i = 5; i < 8; ++i) l.img[i] |= 1u << (i - 3);
  return l;
}

// Staging layout for the copy-out: chunk bits 2..4 XOR word bits s..s+2 (s >= 5).
constexpr Lin lin_stage(int s) {
  Lin l = lin_identity();
  for (int j = 0; j < 3; ++j) l.img[s + j] |= 1u << (2 + j);
  return l;
}

// ------------------------------------------------------------------ phases
struct Phase {
  int nreg = 6;
  int reg[6] = {};
  int lane[5] = {};
  int nwarp = 0;
  int warp[8] = {};
  int ncta = 0;
  int cta[4] = {};
};

constexpr uint32_t reg_label(const Phase& p, int k) {
  uint32_t l = 0;
  for (int i = 0; i < p.nreg; ++i)
    if ((k >> i) & 1) l |= 1u << p.reg[i];
  return l;
}
constexpr uint32_t lane_label(const Phase& p, int ln) {
  uint32_t l = 0;
  for (int i = 0; i < 5; ++i)
    if ((ln >> i) & 1) l |= 1u << p.lane[i];
  return l;
}
constexpr uint32_t warp_label(const Phase& p, int w) {
  uint32_t l = 0;
  for (int i = 0; i < p.nwarp; ++i)
    if ((w >> i) & 1) l |= 1u << p.warp[i];
  return l;
}
constexpr uint32_t cta_label(const Phase& p, int r) {
  uint32_t l = 0;
  for (int i = 0; i < p.ncta; ++i)
    if ((r >> i) & 1) l |= 1u << p.cta[i];
  return l;
}
constexpr int reg_index_of(const Phase& p, int b) {
  for (int i = 0; i < p.nreg; ++i)
    if (p.reg[i] == b) return i;
  return -1;
}
// Register index (in phase p's order) holding the value of the same label as index k of q.
constexpr int remap_index(const Phase& p, const Phase& q, int k) {
  const uint32_t lab = reg_label(q, k);
  for (int j = 0; j < (1 << p.nreg); ++j)
    if (reg_label(p, j) == lab) return j;
  return -1;
}

// Every label bit 0..nbits-1 is owned exactly once by a register, lane, warp or CTA bit.
constexpr bool phase_covers(const Phase& p, int nbits) {
  int seen[kMaxBits] = {};
  for (int i = 0; i < p.nreg; ++i) seen[p.reg[i]]++;
  for (int i = 0; i < 5; ++i) seen[p.lane[i]]++;
  for (int i = 0; i < p.nwarp; ++i) seen[p.warp[i]]++;
  for (int i = 0; i < p.ncta; ++i) seen[p.cta[i]]++;
  for (int b = 0; b < kMaxBits; ++b)
    if (seen[b] != (b < nbits ? 1 : 0)) return false;
  return true;
}

// Registers 0,1 are the two lowest word-position bits and nothing else touches them.
constexpr bool v4_ok(const Phase& p, const Lin& map, uint32_t lmask) {
  if (p.nreg < 2) return false;
  if (apply(map, (1u << p.reg[0]) & lmask) != 1u) return false;
  if (apply(map, (1u << p.reg[1]) & lmask) != 2u) return false;
  for (int i = 2; i < p.nreg; ++i)
    if (apply(map, (1u << p.reg[i]) & lmask) & 3u) return false;
  for (int i = 0; i < 5; ++i)
    if (apply(map, (1u << p.lane[i]) & lmask) & 3u) return false;
  for (int i = 0; i < p.nwarp; ++i)
    if (apply(map, (1u << p.warp[i]) & lmask) & 3u) return false;
  for (int i = 0; i < p.ncta; ++i)
    if (apply(map, (1u << p.cta[i]) & lmask) & 3u) return false;
  return true;
}

// Worst number of lanes of one warp instruction that hit the same bank (scalar 4-byte
// accesses) or the same 16-byte bank group within a quarter warp (128-bit accesses).
constexpr int conflict_degree(const Phase& p, const Lin& map, uint32_t lmask, bool vec) {
  int worst = 1;
  const int step = vec ? 4 : 1;
  for (int k = 0; k < (1 << p.nreg); k += step) {
    if (vec) {
      for (int q = 0; q < 4; ++q) {
        int count[8] = {};
        for (int ln = 8 * q; ln < 8 * q + 8; ++ln) {
          const uint32_t pos = apply(map, (reg_label(p, k) | lane_label(p, ln)) & lmask);
          count[(pos >> 2) & 7]++;
        }
        for (int b = 0; b < 8; ++b) worst = count[b] > worst ? count[b] : worst;
      }
    } else {
      int count[32] = {};
      for (int ln = 0; ln < 32; ++ln) {
        const uint32_t pos = apply(map, (reg_label(p, k) | lane_label(p, ln)) & lmask);
        count[pos & 31]++;
      }
      for (int b = 0; b < 32; ++b) worst = count[b] > worst ? count[b] : worst;
    }
  }
  return worst;
}

// ------------------------------------------------------------------ device helpers
template <int N, class F>
__device__ __forceinline__ void sfor(F&& f) {
  [&]<int... I>(std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
  }(std::make_integer_sequence<int, N>{});
}

// Per-thread part of a phase's word position: lane, warp and CTA-rank bits through `map`.
template <Phase P, Lin MAP, uint32_t LMASK>
__device__ __forceinline__ uint32_t thread_pos(uint32_t lane, uint32_t warp, uint32_t rank) {
  uint32_t pos = 0;
  sfor<5>([&](auto i) {
    constexpr uint32_t im = apply(MAP, (1u << P.lane[i]) & LMASK);
    if ((lane >> i) & 1u) pos ^= im;
  });
  sfor<P.nwarp>([&](auto i) {
    constexpr uint32_t im = apply(MAP, (1u << P.warp[i]) & LMASK);
    if ((warp >> i) & 1u) pos ^= im;
  });
  sfor<P.ncta>([&](auto i) {
    constexpr uint32_t im = apply(MAP, (1u << P.cta[i]) & LMASK);
    if ((rank >> i) & 1u) pos ^= im;
  });
  return pos;
}

// Label (not position) bits owned by this thread outside its registers.
template <Phase P>
__device__ __forceinline__ uint32_t thread_label(uint32_t lane, uint32_t warp, uint32_t rank) {
  uint32_t lab = 0;
  sfor<5>([&](auto i) { lab |= ((lane >> i) & 1u) << P.lane[i]; });
  sfor<P.nwarp>([&](auto i) { lab |= ((warp >> i) & 1u) << P.warp[i]; });
  sfor<P.ncta>([&](auto i) { lab |= ((rank >> i) & 1u) << P.cta[i]; });
  return lab;
}

// Load the 64 values of phase P from local shared memory laid out by MAP.
template <Phase P, Lin MAP, uint32_t LMASK>
__device__ __forceinline__ void load_phase(uint32_t (&v)[64], const uint32_t* buf, uint32_t base) {
  if constexpr (v4_ok(P, MAP, LMASK)) {
    sfor<16>([&](auto j) {
      constexpr int k = 4 * j;
      constexpr uint32_t kp = apply(MAP, reg_label(P, k) & LMASK);
      const uint4 q = *reinterpret_cast<const uint4*>(buf + (base ^ kp));
      v[k] = q.x;
      v[k + 1] = q.y;
      v[k + 2] = q.z;
      v[k + 3] = q.w;
    });
  } else {
    sfor<64>([&](auto k) {
      constexpr uint32_t kp = apply(MAP, reg_label(P, k) & LMASK);
      v[k] = buf[base ^ kp];
    });
  }
}

// Store the values (indexed in phase PR's register order) in phase PW's register order.
template <Phase PW, Phase PR, Lin MAP, uint32_t LMASK>
__device__ __forceinline__ void store_phase(const uint32_t (&v)[64], uint32_t* buf, uint32_t base) {
  if constexpr (v4_ok(PW, MAP, LMASK)) {
    sfor<16>([&](auto j) {
      constexpr int k = 4 * j;
      constexpr uint32_t kp = apply(MAP, reg_label(PW, k) & LMASK);
      constexpr int r0 = remap_index(PR, PW, k), r1 = remap_index(PR, PW, k + 1);
      constexpr int r2 = remap_index(PR, PW, k + 2), r3 = remap_index(PR, PW, k + 3);
      static_assert(r0 >= 0 && r1 >= 0 && r2 >= 0 && r3 >= 0, "write order must hold the same labels");
      *reinterpret_cast<uint4*>(buf + (base ^ kp)) = make_uint4(v[r0], v[r1], v[r2], v[r3]);
    });
  } else {
    sfor<64>([&](auto k) {
      constexpr uint32_t kp = apply(MAP, reg_label(PW, k) & LMASK);
      constexpr int r = remap_index(PR, PW, k);
      static_assert(r >= 0, "write order must hold the same labels");
      buf[base ^ kp] = v[r];
    });
  }
}

// Store the values (indexed in phase PR's order) with 16-byte stores into the shared memory
// of the cluster CTA whose buffer starts at cluster address `rbase`, at positions MAP(label).
template <Phase PW, Phase PR, Lin MAP>
__device__ __forceinline__ void store_phase_remote(const uint32_t (&v)[64], uint32_t rbase, uint32_t base) {
  static_assert(v4_ok(PW, MAP, ~0u), "remote stores move 16-byte chunks");
  sfor<16>([&](auto j) {
    constexpr int k = 4 * j;
    constexpr uint32_t kp = apply(MAP, reg_label(PW, k));
    constexpr int r0 = remap_index(PR, PW, k), r1 = remap_index(PR, PW, k + 1);
    constexpr int r2 = remap_index(PR, PW, k + 2), r3 = remap_index(PR, PW, k + 3);
    static_assert(r0 >= 0 && r1 >= 0 && r2 >= 0 && r3 >= 0, "write order must hold the same labels");
    st_dsmem_v4(rbase + 4u * (base ^ kp), v[r0], v[r1], v[r2], v[r3]);
  });
}

// Load phase P's values from the cluster: label bits >= TB pick the CTA rank whose shared
// memory (at the same layout MAP) holds them; rbase[r] is that CTA's buffer address.
template <Phase P, Lin MAP, int TB, int NR>
__device__ __forceinline__ void load_phase_cluster(uint32_t (&v)[64], const uint32_t (&rbase)[NR], uint32_t base) {
  constexpr uint32_t lmask = (1u << TB) - 1u;
  sfor<64>([&](auto k) {
    constexpr uint32_t lab = reg_label(P, k);
    constexpr uint32_t rank = lab >> TB;
    static_assert(rank < NR, "cluster rank out of range");
    constexpr uint32_t kp = apply(MAP, lab & lmask);
    v[k] = ld_dsmem_b32(rbase[rank] + 4u * (base ^ kp));
  });
}

// The butterflies of the Haar-Walsh head (a 2^HM-element prefix, see fused.cuh OUTMODE 6):
// the pair at bit b whose labels have no bit in [b+1, HM) set is stage 0's (the Haar
// transform's) and is skipped.  `tl` = the thread's label bits; reg bits are compile time.
template <Phase P, int LO, int HI, int HM, class BF>
__device__ __forceinline__ void butterflies_head(uint32_t (&v)[64], const BF& bf, uint32_t tl) {
  sfor<kMaxBits>([&](auto bb) {
    constexpr int b = bb;
    if constexpr (b >= LO && b < HI) {
      constexpr int i = reg_index_of(P, b);
      static_assert(i >= 0, "a butterfly bit must be a register bit of its phase");
      constexpr uint32_t above = ((1u << HM) - 1u) & ~((2u << b) - 1u);
      const bool live = (tl & above) != 0u;
      sfor<64>([&](auto kk) {
        constexpr int k = kk;
        constexpr bool s0 = (reg_label(P, k) & above) != 0u;
        if constexpr (BF::kPacked && i >= 1) {
          // registers k and k | 1 travel together (one f32x2 pair) where both are live or
          // both depend on the thread's label the same way
          constexpr bool s1 = (reg_label(P, k | 1) & above) != 0u;
          if constexpr (((k >> i) & 1) == 0 && (k & 1) == 0) {
            constexpr int j = 1 << i;
            if constexpr (s0 && s1) {
              bf.pair(v[k], v[k | 1], v[k | j], v[k | 1 | j]);
            } else if constexpr (!s0 && !s1) {
              if (live) bf.pair(v[k], v[k | 1], v[k | j], v[k | 1 | j]);
            } else {
              if (s0 || live) bf(v[k], v[k | j]);
              if (s1 || live) bf(v[k | 1], v[k | 1 | j]);
            }
          }
        } else if constexpr (((k >> i) & 1) == 0) {
          if constexpr (s0) {
            bf(v[k], v[k | (1 << i)]);
          } else {
            if (live) bf(v[k], v[k | (1 << i)]);
          }
        }
      });
    }
  });
}

// Butterflies of phase P on the label bits in [LO, HI), lowest bit first.  When the
// functor has a packed form (two butterflies in one f32x2 instruction pair) and register
// bit 0 is not the butterfly bit, registers k and k|1 travel together.
template <Phase P, int LO, int HI, class BF>
__device__ __forceinline__ void butterflies(uint32_t (&v)[64], const BF& bf) {
  sfor<kMaxBits>([&](auto bb) {
    constexpr int b = bb;
    if constexpr (b >= LO && b < HI) {
      constexpr int i = reg_index_of(P, b);
      static_assert(i >= 0, "a butterfly bit must be a register bit of its phase");
      if constexpr (BF::kPacked && i >= 1) {
        sfor<64>([&](auto kk) {
          constexpr int k = kk;
          if constexpr (((k >> i) & 1) == 0 && (k & 1) == 0)
            bf.pair(v[k], v[k | 1], v[k | (1 << i)], v[k | 1 | (1 << i)]);
        });
      } else {
        sfor<64>([&](auto kk) {
          constexpr int k = kk;
          if constexpr (((k >> i) & 1) == 0) bf(v[k], v[k | (1 << i)]);
        });
      }
    }
  });
}

// Butterfly (a, b) -> (a+b, a-b), values carried as 32-bit patterns.  The packed form
// runs two butterflies with f32x2 instructions (per-lane IEEE round to nearest even, no
// flush of subnormals: the same results as the scalar form).
// fp32(2^{-m/2}) for 0 <= m <= 252: 2^{-floor(m/2)} times 1 or fp32(1/sqrt2).  Scaling the
// correctly rounded constant by a power of two is exact in fp32's normal range, so the
// result is 2^{-m/2} correctly rounded.
__device__ __forceinline__ float end_scale_dev(int m) {
  const float r = (m & 1) ? 0.70710678118654752440f : 1.0f;
  return __fmul_rn(r, __uint_as_float(static_cast<uint32_t>(127 - m / 2) << 23));
}

struct BfF32Plain {
  static constexpr bool kPacked = true;
  __device__ __forceinline__ void operator()(uint32_t& a, uint32_t& b) const {
    const float x = __uint_as_float(a), y = __uint_as_float(b);
    a = __float_as_uint(__fadd_rn(x, y));
    b = __float_as_uint(__fsub_rn(x, y));
  }
  __device__ __forceinline__ void pair(uint32_t& a0, uint32_t& a1, uint32_t& b0, uint32_t& b1) const {
    asm("{\n\t.reg .b64 x, y, s, d;\n\t"
        "mov.b64 x, {%4, %5};\n\tmov.b64 y, {%6, %7};\n\t"
        "add.rn.f32x2 s, x, y;\n\tsub.rn.f32x2 d, x, y;\n\t"
        "mov.b64 {%0, %1}, s;\n\tmov.b64 {%2, %3}, d;\n\t}"
        : "=r"(a0), "=r"(a1), "=r"(b0), "=r"(b1)
        : "r"(a0), "r"(a1), "r"(b0), "r"(b1));
  }
};
// (a, b) -> ((a+b) c, (a-b) c), each operation rounded to nearest even.  The packed form
// adds and subtracts with f32x2 but multiplies with scalar mul.rn: a packed multiply feeding
// the next level's packed add was observed to be fused into one FMA by the assembler (a
// GB300 probe of chained levels), which would round differently from the cascade; built
// with -fmad=false (no contraction at all) the packed mul.rn still gave results differing
// from the cascade by a few ulps on most outputs (m = 17), while packed add and subtract
// are exact.
struct BfF32PerLevel {
  static constexpr bool kPacked = true;
  float c;
  __device__ __forceinline__ void operator()(uint32_t& a, uint32_t& b) const {
    const float x = __uint_as_float(a), y = __uint_as_float(b);
    a = __float_as_uint(__fmul_rn(__fadd_rn(x, y), c));
    b = __float_as_uint(__fmul_rn(__fsub_rn(x, y), c));
  }
  __device__ __forceinline__ void pair(uint32_t& a0, uint32_t& a1, uint32_t& b0, uint32_t& b1) const {
    BfF32Plain{}.pair(a0, a1, b0, b1);
    a0 = __float_as_uint(__fmul_rn(__uint_as_float(a0), c));
    a1 = __float_as_uint(__fmul_rn(__uint_as_float(a1), c));
    b0 = __float_as_uint(__fmul_rn(__uint_as_float(b0), c));
    b1 = __float_as_uint(__fmul_rn(__uint_as_float(b1), c));
  }
};
// int32 with two's-complement wrap (unsigned arithmetic).
struct BfI32 {
  static constexpr bool kPacked = false;
  __device__ __forceinline__ void operator()(uint32_t& a, uint32_t& b) const {
    const uint32_t x = a, y = b;
    a = x + y;
    b = x - y;
  }
  __device__ __forceinline__ void pair(uint32_t&, uint32_t&, uint32_t&, uint32_t&) const {}
};

}  // namespace chw
