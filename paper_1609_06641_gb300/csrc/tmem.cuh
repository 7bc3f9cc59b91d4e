// Whole-signal kernel for signals of 2^15 and 2^16 four-byte elements: one signal per SM
// at a time, with the SM's tensor memory holding the signal between its row and its
// column butterflies, so no element leaves the SM before it is final.
//
// A signal of 2^M elements is R = 2^(M-14) rows of 2^14 (label bits 0..13 within a row,
// bits 14..M-1 the row index).  Each row goes through the first three register phases of
// the fused 2^14 tile (TMA load into shared memory, phases 1-3: label bits 0..13, in
// order, exactly as fused.cuh runs them).  Phase 3 leaves every thread with 64 values that
// share its thread label bits 0..7 and differ in the register label bits 8..13.  The
// thread stores them into its own tensor-memory lane (32x32b shape: warp w reaches lanes
// 32 (w mod 4) .. +31, and warps w and w + 4 use the two halves of the columns), 64
// columns per row.  After the R rows the same thread reads them back: for each of its 64
// register labels it holds the R values that differ only in the row bits, and runs the
// cascade's last butterflies (bits 14..M-1) in registers, with no exchange between
// threads or SMs.  Results are staged in shared memory, one 2^14-value chunk at a time:
// in dyadic or natural order they leave by TMA tensor stores that drain while the SM
// transforms the next row; in sequency order the SM copies each aligned 32-element block
// to its gray^{-1} block.  Each output chunk of a signal is interleaved with a row of the
// next signal (alternating tensor-memory column layouts), so every step loads one row and
// stores one chunk.
//
// Tensor memory is 128 lanes x 512 columns x 4 bytes = 256 KB per SM: one 2^16-word
// signal.  Shared memory holds two 64 KB row buffers (the next rows' TMA loads overlap
// the current row and the column butterflies) and a 64 KB staging buffer, which keeps one
// CTA on each SM; the tensor-memory allocation therefore never waits for another CTA of
// this kernel.
#pragma once

#include "fused.cuh"

namespace chw {

constexpr int kTmemTB = 14;  // row bits
constexpr int kTmemThreads = 1 << (kTmemTB - 6);

constexpr uint32_t bitrev_bits(uint32_t x, int n) {
  uint32_t r = 0;
  for (int i = 0; i < n; ++i) r |= ((x >> i) & 1u) << (n - 1 - i);
  return r;
}

// Phase 3 of the row (label bits 11..13) with the registers on label bits 8..13 and the
// threads on bits 0..7; lane bits 0..2 carry label bits 7, 6, 5, which are the low bits of
// the thread's output run (the staging swizzle key, below).
constexpr Phase make_p3_tmem() {
  Phase p{};
  const int r[6] = {13, 12, 11, 10, 9, 8};
  const int l[5] = {7, 6, 5, 1, 0};
  const int w[3] = {2, 3, 4};
  p.nreg = 6;
  for (int i = 0; i < 6; ++i) p.reg[i] = r[i];
  for (int i = 0; i < 5; ++i) p.lane[i] = l[i];
  p.nwarp = 3;
  for (int i = 0; i < 3; ++i) p.warp[i] = w[i];
  return p;
}

// The thread label bits 0..7 and register bits 8..13 of phase 3 (the output mapping below
// depends on it).
constexpr bool tmem_p3_split(const Phase& p) {
  for (int i = 0; i < p.nreg; ++i)
    if (p.reg[i] < 8 || p.reg[i] > 13) return false;
  for (int i = 0; i < 5; ++i)
    if (p.lane[i] > 7) return false;
  for (int i = 0; i < p.nwarp; ++i)
    if (p.warp[i] > 7) return false;
  return p.nreg == 6 && p.ncta == 0;
}

// The staging key (bits 0..2 of a thread's output run, see below) differs between the
// eight lanes of every quarter warp: the 16-byte staging stores are conflict-free.
constexpr bool tmem_stage_key_ok(const Phase& p) {
  for (int q = 0; q < 4; ++q) {
    int seen = 0;
    for (int ln = 8 * q; ln < 8 * q + 8; ++ln) seen |= 1 << (bitrev_bits(lane_label(p, ln), 8) & 7u);
    if (seen != 0xff) return false;
  }
  return true;
}

// Natural order stages whole 32-word rows per warp: the lanes of phase 3 must carry label
// bits 0..4 (output bits 0..4), so that one scalar store per register is conflict-free.
constexpr bool tmem_natural_lanes_ok(const Phase& p) {
  int seen = 0;
  for (int i = 0; i < 5; ++i) seen |= 1 << p.lane[i];
  return seen == 0x1f;
}

// OM = 0: dyadic order; OM = 1: dyadic rows of the two-pass split's first pass, stored
// column-blocked (see below); OM = 2: natural (Sylvester) order, label j stored at j;
// OM = 3: sequency (Walsh) order, dyadic position p stored at gray^{-1}(p).
template <int M, int OM = 0>
struct TmemCfg {
  static_assert(M == 15 || M == 16, "tensor memory holds one signal of at most 2^16 words");
  static_assert(OM >= 0 && OM <= 3, "dyadic, column-blocked, natural or sequency order");
  static constexpr int TB = kTmemTB;
  static constexpr int R = 1 << (M - TB);  // rows per signal
  static constexpr int JW = 64 / R;        // registers per row in one output chunk
  static constexpr uint32_t NCOLS = 512;    // two column halves: two signals of 2^15 or one of 2^16
  // phases 1 and 2 of the fused 2^14 row tile; phase 3 and the exchange layout of our own
  static constexpr FusedPlan F = FusedCfg<0, TB, TB, 0, 0>::plan;
  static constexpr Phase P2 = F.p2;
  static constexpr Phase P3 = OM == 2 ? F.p3 : make_p3_tmem();
  static constexpr Lin LB = make_lin_b(P2, P3);
  static constexpr bool b_is_s = lin_equal(LB, F.lin_s);
  static_assert(F.has_p3 && phase_covers(P3, TB) && tmem_p3_split(P3), "phase 3 splits the label as 0..7 | 8..13");
  static_assert(conflict_degree(P2, LB, (1u << TB) - 1u, false) == 1, "phase 2 writes are conflict-free");
  static_assert(conflict_degree(P3, LB, (1u << TB) - 1u, false) == 1, "phase 3 reads are conflict-free");
  static_assert(OM == 2 ? tmem_natural_lanes_ok(P3) : tmem_stage_key_ok(P3), "staging stores are conflict-free");

  // Output bits the thread label does not fix: the dyadic output position of label L is
  // bitrev_M(L); the thread's label bits 0..7 give output bits M-8..M-1 (its "run" rho,
  // 2^(M-8) outputs apart), register k of row r gives the low M-8 bits.
  static constexpr uint32_t out_low(int r, int k) {
    return bitrev_bits(reg_label(P3, k) | (static_cast<uint32_t>(r) << TB), M);
  }
  // Output chunk q holds the low bits [64 q, 64 q + 64), i.e. registers [q JW, (q+1) JW) of
  // every row; src(q, w) is the index r JW + j in the chunk's register array of low bits
  // 64 q + w (-1 if none).
  static constexpr int src(int q, int w) {
    for (int r = 0; r < R; ++r)
      for (int j = 0; j < JW; ++j)
        if (out_low(r, q * JW + j) == static_cast<uint32_t>(64 * q + w)) return r * JW + j;
    return -1;
  }
  static constexpr bool chunks_ok() {
    for (int q = 0; q < R; ++q)
      for (int w = 0; w < 64; ++w)
        if (src(q, w) < 0) return false;
    return true;
  }
  static_assert(OM == 2 || chunks_ok(), "each output chunk is exactly one register range of every row");

  // Natural order: register k of row r holds output bits 8..M-1 = its label bits 8..M-1.
  // In output chunk q they are the row psi = bits M-6..M-1 (64 rows, 2^(M-6) words apart)
  // and the 256-word block qo = bits 8..M-7 of that row, the same for the whole chunk.
  static constexpr uint32_t nat_high(int r, int k) { return reg_label(P3, k) | (static_cast<uint32_t>(r) << TB); }
  static constexpr uint32_t nat_psi(int r, int k) { return nat_high(r, k) >> (M - 6); }
  static constexpr uint32_t nat_qo(int r, int k) { return (nat_high(r, k) >> 8) & ((1u << (M - 14)) - 1u); }
  static constexpr bool natural_ok() {
    for (int q = 0; q < R; ++q) {
      int seen[64] = {};
      for (int r = 0; r < R; ++r)
        for (int j = 0; j < JW; ++j) {
          if (nat_qo(r, q * JW + j) != nat_qo(0, q * JW)) return false;
          seen[nat_psi(r, q * JW + j)]++;
        }
      for (int i = 0; i < 64; ++i)
        if (seen[i] != 1) return false;
    }
    return true;
  }
  static_assert(OM == 0 || natural_ok(), "a natural-order chunk is 64 rows of one 256-word block");
};

constexpr int tmem_smem_bytes() {
  return (12 << kTmemTB) + 1024 + 64;  // two row buffers and the staging buffer, barriers, slot
}

// Output tensor map of the kernel's TMA stores, SWIZZLE_128B, boxes 32 words wide.  Dyadic
// order: the output as rows of 2^(M-8) words (one output run), boxes of 256 rows; the
// staging buffer holds one chunk as two boxes, words [0, 32) and [32, 64) of each of the
// 256 runs.  Natural order: rows of 2^(M-6) words, boxes of 64 rows; a chunk is eight
// boxes, words [32 b, 32 b + 32) of one 256-word block of each of 64 rows.

// Tensor-memory column of register k (a multiple of 16) of row r of a signal whose
// position in this CTA's sequence has parity `par`, within the thread's 256-column half.
// 2^16: even signals keep row r in the 64-column block r, odd signals keep register block
// k / 16 of every row in block k / 16 -- so the four registers blocks that the column
// chunk q of an even signal reads are exactly where row q of the next (odd) signal goes,
// and the other way round.  2^15: each parity has its own 128 columns.
template <int M>
__device__ __forceinline__ uint32_t tmem_col(uint32_t par, int r, int k) {
  if constexpr (M == 16) {
    return par ? 64u * (k >> 4) + 16u * r + (k & 15) : 64u * r + k;
  } else {
    return 128u * par + 64u * r + k;
  }
}

template <int M, class BF, bool SCALE, int OM>
__global__ void __launch_bounds__(kTmemThreads, 1)
    tmem_kernel(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout,
                const FusedArgs args, const int64_t units) {
  using T = TmemCfg<M, OM>;
  constexpr int TB = T::TB, R = T::R, JW = T::JW;
  constexpr uint32_t LMASK = (1u << TB) - 1u;
  constexpr Phase P2 = T::P2, P3 = T::P3;
  constexpr Lin LB = T::LB;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  uint32_t* bufs = reinterpret_cast<uint32_t*>(base);  // row buffers g mod 2
  uint32_t* stage = bufs + (2u << TB);
  uint64_t* bar = reinterpret_cast<uint64_t*>(stage + (1u << TB));
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 2);
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(slot, T::NCOLS);
    tmem_relinquish_alloc_permit();
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tmem = *slot;
  // this thread's lane and its warp's half of the columns
  const uint32_t taddr = tmem + ((32u * (warp & 3u)) << 16) + (T::NCOLS / 2) * (warp >> 2);

  const int64_t stride = gridDim.x;
  const int64_t first = blockIdx.x;
  const int64_t K = first < units ? (units - first + stride - 1) / stride : 0;
  const int64_t G = K * R;  // rows this CTA loads
  auto elem0 = [&](int64_t k) { return unit_elem<M>(args, args.in_off, first + k * stride); };
  auto row0 = [&](int64_t g) { return static_cast<int>((elem0(g / R) >> 5) + (g % R) * (1 << (TB - 5))); };
  if (tid == 0) {
    if (G > 0) tile_issue<TB>(&tin, row0(0), bufs, bar);
    if (G > 1) tile_issue<TB>(&tin, row0(1), bufs + (1u << TB), bar + 1);
  }
  BF bf{};
  if constexpr (std::is_same_v<BF, BfF32PerLevel>) bf.c = 0.70710678118654752440f;
  // A wait that gives up records CHW_ERR_TIMEOUT and turns this thread's later waits off.
  bool waiting = true;
  const uint32_t tries = args.wait_tries != 0 ? args.wait_tries : kWaitTries;
  // dyadic: output run of this thread (output bits M-8..M-1) and its staging swizzle;
  // natural: its label bits 0..7 are its output bits 0..7
  const uint32_t tl = thread_label<P3>(lane, warp, 0);
  const uint32_t rho = bitrev_bits(tl, 8);
  const uint32_t sxor = (rho & 7u) << 2;

  // Row r of signal k: label bits 0..13, then into tensor memory.
  auto row = [&](int64_t k, int r) {
    const int64_t g = k * R + r;
    uint32_t* buf = bufs + ((g & 1) << TB);
    if (waiting && !mbar_wait_bounded(bar + (g & 1), static_cast<uint32_t>((g >> 1) & 1), tries)) {
      waiting = false;
      if (lane == 0) atomicCAS(args.status, 0, kStatusTimeout);
    }
    uint32_t v[64];
    phases_1_2<0, TB, TB, 0, BF>(v, elem0(k) + (int64_t{r} << TB), args, buf, bf);
    if constexpr (!T::b_is_s) __syncthreads();
    store_phase<P2, P2, LB, LMASK>(v, buf, thread_pos<P2, LB, LMASK>(lane, warp, 0));
    __syncthreads();
    load_phase<P3, LB, LMASK>(v, buf, thread_pos<P3, LB, LMASK>(lane, warp, 0));
    butterflies<P3, 11, TB>(v, bf);
    __syncthreads();  // the row buffer is no longer read: refill it
    if (tid == 0 && g + 2 < G) tile_issue<TB>(&tin, row0(g + 2), buf, bar + (g & 1));
    const uint32_t par = static_cast<uint32_t>(k & 1);
    tmem_st16<0>(taddr + tmem_col<M>(par, r, 0), v);
    tmem_st16<16>(taddr + tmem_col<M>(par, r, 16), v);
    tmem_st16<32>(taddr + tmem_col<M>(par, r, 32), v);
    tmem_st16<48>(taddr + tmem_col<M>(par, r, 48), v);
    tmem_wait_st();
  };

  // Output chunk q of signal k: label bits 14..M-1 on registers [q JW, (q+1) JW) of every
  // row, staged in output order and stored by TMA.
  auto chunk = [&](int64_t k, auto qq) {
    constexpr int q = qq;
    const uint32_t par = static_cast<uint32_t>(k & 1);
    uint32_t u[64];  // u[r JW + j] = row r, register q JW + j
    sfor<R>([&](auto rr) {
      constexpr int r = rr;
      sfor<JW / 16>([&](auto jj) {
        constexpr int j = 16 * jj;
        tmem_ld16<r * JW + j>(taddr + tmem_col<M>(par, r, q * JW + j), u);
      });
    });
    tmem_wait_ld<0>(u);
    tmem_wait_ld<16>(u);
    tmem_wait_ld<32>(u);
    tmem_wait_ld<48>(u);
    sfor<M - TB>([&](auto bb) {  // label bit TB + b pairs rows r and r + 2^b
      constexpr int b = bb;
      sfor<R>([&](auto rr) {
        constexpr int r = rr;
        if constexpr (((r >> b) & 1) == 0) {
          sfor<JW>([&](auto j) { bf(u[r * JW + j], u[(r | (1 << b)) * JW + j]); });
        }
      });
    });
    if constexpr (SCALE) {
#pragma unroll
      for (int i = 0; i < 64; ++i) u[i] = __float_as_uint(__fmul_rn(__uint_as_float(u[i]), args.end_scale));
    }
    const int64_t ob = unit_elem<M>(args, args.out_off, first + k * stride);
    if constexpr (OM == 2) {
      constexpr uint32_t qo = T::nat_qo(0, q * JW);
      if (args.diag_out != nullptr) {  // D acts on the stored positions
        const int8_t* d = args.diag_out + (tl & args.diag_mask);
        sfor<64>([&](auto ii) {
          constexpr int r = ii / JW, j = ii % JW;
          constexpr int64_t o = T::nat_high(r, q * JW + j);  // output bits 8..M-1
          if (d[o & args.diag_mask] < 0) u[ii] = std::is_same_v<BF, BfI32> ? 0u - u[ii] : u[ii] ^ 0x80000000u;
        });
      }
      if (tid == 0) bulk_wait_read();  // the previous chunk's TMA stores have read the buffer
      __syncthreads();
      // word tl mod 32 of row psi in box tl / 32, 16-byte chunk XOR psi mod 8
      uint32_t* sb = stage + ((tl >> 5) << 11) + (tl & 3u);
      const uint32_t xc = (tl >> 2) & 7u;
      sfor<64>([&](auto ii) {
        constexpr int r = ii / JW, j = ii % JW;
        constexpr uint32_t psi = T::nat_psi(r, q * JW + j);
        sb[(psi << 5) | ((xc ^ (psi & 7u)) << 2)] = u[ii];
      });
      fence_proxy_async_smem();
      __syncthreads();
      if (tid == 0) {
        const int y = static_cast<int>(ob >> (M - 6));
#pragma unroll
        for (int b = 0; b < 8; ++b) tma_store_2d(&tout, stage + (b << 11), static_cast<int>(qo) * 256 + 32 * b, y);
        bulk_commit_group();
      }
    } else {
      if (OM == 0 && args.diag_out != nullptr) {  // D acts on the stored positions
        const int8_t* d = args.diag_out + ((static_cast<int64_t>(rho) << (M - 8)) & args.diag_mask);
        sfor<64>([&](auto ww) {
          constexpr int w = ww;
          constexpr int si = T::src(q, w);
          if (d[64 * q + w] < 0) u[si] = std::is_same_v<BF, BfI32> ? 0u - u[si] : u[si] ^ 0x80000000u;
        });
      }
      if (tid == 0) bulk_wait_read();  // the previous chunk's TMA stores have read the buffer
      __syncthreads();
      // Output low bits 64 q + w of run rho: box w / 32, row rho, 16-byte chunk (w mod 32) / 4
      // XOR rho mod 8 (the TMA's 128-byte swizzle).
      sfor<16>([&](auto cc) {
        constexpr int c = cc;
        constexpr int s0 = T::src(q, 4 * c), s1 = T::src(q, 4 * c + 1);
        constexpr int s2 = T::src(q, 4 * c + 2), s3 = T::src(q, 4 * c + 3);
        constexpr uint32_t box = (c >> 3) << (TB - 1);
        *reinterpret_cast<uint4*>(stage + box + ((rho << 5) | ((4u * (c & 7)) ^ sxor))) =
            make_uint4(u[s0], u[s1], u[s2], u[s3]);
      });
      if constexpr (OM == 0) {
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
          const int y = static_cast<int>(ob >> (M - 8));
          tma_store_2d(&tout, stage, 64 * q, y);
          tma_store_2d(&tout, stage + (1u << (TB - 1)), 64 * q + 32, y);
          bulk_commit_group();
        }
      } else {
        // Sequency order scatters the runs (gray^{-1} of their high bits), and the
        // column-blocked order of the first of two passes sends every 32-element segment of
        // a row to its own block, so the chunk goes out through the SM: a warp copies four
        // aligned 32-element blocks, each to one whole 128-byte line (gray^{-1} maps an
        // aligned block onto an aligned block, reordered inside).
        __syncthreads();
        uint32_t* out = static_cast<uint32_t*>(args.out);
        // OM = 1: row u is row r = u mod 2^a of signal u / 2^a (a = colblock_a); its element
        // k goes to signal * 2^(a+M) + (k / 32) 2^(a+5) + 32 r + k mod 32
        const int64_t u = first + k * stride;
        const int cba = args.colblock_a;
        const int64_t cb_base = ((u >> cba) << (cba + M)) + ((u & ((int64_t{1} << cba) - 1)) << 5);
#pragma unroll 4
        for (int i = static_cast<int>(tid); i < (1 << (TB - 2)); i += kTmemThreads) {
          const uint32_t h = static_cast<uint32_t>(i) >> (TB - 3), run = (static_cast<uint32_t>(i) >> 3) & 255u;
          const uint32_t c8 = static_cast<uint32_t>(i) & 7u;
          uint4 val = *reinterpret_cast<const uint4*>(stage + (h << (TB - 1)) + (run << 5) + ((c8 ^ (run & 7u)) << 2));
          // dyadic position / 4 within the signal
          const uint32_t p4 = (run << (M - 10)) | static_cast<uint32_t>(16 * q) | (h << 3) | c8;
          int64_t addr;
          if constexpr (OM == 1) {
            addr = cb_base + (static_cast<int64_t>(p4 >> 3) << (cba + 5)) + ((p4 & 7u) << 2);
          } else {
            uint32_t g = p4;  // gray^{-1}
            g ^= g >> 1;
            g ^= g >> 2;
            g ^= g >> 4;
            g ^= g >> 8;
            g ^= g >> 16;
            val = (__popc(p4) & 1) ? make_uint4(val.z, val.w, val.y, val.x) : make_uint4(val.x, val.y, val.w, val.z);
            addr = ob + (static_cast<int64_t>(g) << 2);
          }
          if (args.diag_out != nullptr) {  // D acts on the stored positions
            const int8_t* d = args.diag_out + (addr & args.diag_mask);
            if constexpr (std::is_same_v<BF, BfI32>) {
              if (d[0] < 0) val.x = 0u - val.x;
              if (d[1] < 0) val.y = 0u - val.y;
              if (d[2] < 0) val.z = 0u - val.z;
              if (d[3] < 0) val.w = 0u - val.w;
            } else {
              if (d[0] < 0) val.x ^= 0x80000000u;
              if (d[1] < 0) val.y ^= 0x80000000u;
              if (d[2] < 0) val.z ^= 0x80000000u;
              if (d[3] < 0) val.w ^= 0x80000000u;
            }
          }
          st_global_v4(out + addr, val.x, val.y, val.z, val.w);
        }
      }
    }
  };

  // Software pipeline: output chunk i of signal t-1 frees the tensor-memory columns that
  // row i of signal t fills, so every step reads one row and writes one chunk.
  for (int64_t t = 0; t <= K; ++t) {
#pragma unroll 1
    for (int i = 0; i < R; ++i) {
      if (t >= 1) {
        sfor<R>([&](auto qq) {
          if (static_cast<int>(qq) == i) chunk(t - 1, qq);
        });
      }
      if (t < K) row(t, i);
    }
  }
  // Leave no TMA load in flight into shared memory, even when a wait above gave up: wait
  // (bounded) for the last load issued on each barrier.
  if (tid == 0) {
    for (int64_t b = 0; b < 2 && b < G; ++b) {
      const int64_t gl = b + ((G - 1 - b) / 2) * 2;
      mbar_wait_bounded(bar + b, static_cast<uint32_t>((gl >> 1) & 1), kWaitTries);
    }
  }
  if (tid == 0) bulk_wait_all();  // the output stores have completed
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(tmem, T::NCOLS);
}

}  // namespace chw
