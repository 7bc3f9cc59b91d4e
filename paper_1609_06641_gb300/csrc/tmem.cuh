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
// in dyadic, natural or sequency order they leave by TMA tensor stores that drain while
// the SM transforms the next row (sequency order stages each chunk already permuted by
// gray^{-1}, see the output chunk below).  Each output chunk of a signal is interleaved with a row of the
// next signal (alternating tensor-memory column layouts), so every step loads one row and
// stores one chunk.
//
// The same kernel runs the column pass of the two-pass split y = H_b X^T H_a (CLO > 0): a
// unit is then a column block of 2^a rows x 2^CLO columns (M = a + CLO words, contiguous
// in the first pass's column-blocked output), label bits 0..CLO-1 the column and bits
// CLO..M-1 the row.  Only the row bits are transformed (the first phase starts at label
// bit CLO, or is skipped when CLO = 5), and column c's results form the contiguous output
// row c in dyadic order: label (c, r) is stored at c 2^a + bitrev_a(r).  Label bits 8..M-1
// then land on output bits M-1-b exactly as in the whole-signal case; only the run index
// of a thread (its output bits M-8..M-1) is formed differently.
//
// Signals of 2^17 words (XP = 1) spread over a cluster of two CTAs, one per SM: CTA c
// holds the 2^16 labels whose bit 16 equals c and runs label bits 0..15 exactly as above.
// Label bit 16 pairs values held by different SMs.  For every output chunk each thread
// keeps half of its 64 values (split by the dyadic output bit 5 of the chunk) and hands the
// other half to the same thread of the peer CTA through an L2-resident scratch slot: the
// CTA stages its 32 KB in shared memory and writes it with one bulk copy; while the CTA
// transforms its next input row, one thread waits for that copy and signals the peer, and
// another waits for the peer's signal and bulk-loads the peer's 32 KB into shared memory.
// Then the butterflies of label bit 16 run and 64 consecutive outputs per thread leave by
// TMA as above.  (The same exchange over distributed shared memory was measured slower on
// GB300: its per-SM bandwidth stalls the threads that issue it.)  Every value still meets
// label bits 0..16 in order, so the results equal the cascade's.
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

// gray^{-1}(x): bit i is the XOR of the bits i, i+1, ... of x (sequency order).
constexpr uint32_t gray_inverse(uint32_t x) {
  x ^= x >> 1;
  x ^= x >> 2;
  x ^= x >> 4;
  x ^= x >> 8;
  x ^= x >> 16;
  return x;
}

constexpr uint32_t parity_of(uint32_t x) { return gray_inverse(x) & 1u; }

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
  // Every chunk maps its registers to the same low output bits: src(q, w) = src(0, w), so
  // the chunk epilogue of the dyadic and sequency orders may take q at run time.
  static constexpr bool src_chunk_free() {
    for (int q = 1; q < R; ++q)
      for (int w = 0; w < 64; ++w)
        if (src(q, w) != src(0, w)) return false;
    return true;
  }
  static_assert(OM == 2 || src_chunk_free(), "the chunk's register map does not depend on the chunk");

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

// Phases 1 and 2 of a 2^14-word row with the butterflies of label bits LO..10 (LO <= 5):
// the fused row tile's phases, the first one restricted to bits LO..4 (skipped when LO = 5,
// phase 2 then reading the TMA layout directly).  On return v holds phase 2's values.
template <int LO, class BF>
__device__ __forceinline__ void row_phases_from(uint32_t (&v)[64], uint32_t* buf, const BF& bf) {
  using Cfg = FusedCfg<0, kTmemTB, kTmemTB, 0>;
  constexpr FusedPlan F = Cfg::plan;
  constexpr uint32_t LMASK = Cfg::LMASK;
  constexpr Phase P1 = F.p1, P2 = F.p2;
  constexpr Lin LS = F.lin_s;
  static_assert(LO >= 1 && LO <= 5, "column tiles start at label bit 1..5");
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  if constexpr (LO < 5) {
    const uint32_t base = thread_pos<P1, LS, LMASK>(lane, warp, 0);
    load_phase<P1, LS, LMASK>(v, buf, base);
    butterflies<P1, LO, 5>(v, bf);
    store_phase<P1, P1, LS, LMASK>(v, buf, base);
    __syncthreads();
  }
  load_phase<P2, LS, LMASK>(v, buf, thread_pos<P2, LS, LMASK>(lane, warp, 0));
  butterflies<P2, 5, 11>(v, bf);
}

// Two row buffers and the staging buffer, barriers and the allocation slot; a signal
// spread over 2^XP SMs (XP > 0) adds a 32 KB receive buffer and 2 XP barriers.
template <int XP = 0>
constexpr int tmem_smem_bytes() {
  return (12 << kTmemTB) + (XP > 0 ? (2 << kTmemTB) : 0) + 1024 + (XP > 0 ? 128 : 64);
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

template <int M, class BF, bool SCALE, int OM, int CLO = 0, bool HZ = false, int XP = 0>
__global__ void __launch_bounds__(kTmemThreads, 1)
    tmem_kernel(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout,
                const FusedArgs args, const int64_t units) {
  static_assert(CLO == 0 || (OM == 0 && CLO >= 2 && CLO <= 5 && M - CLO >= 10),
                "column tiles: dyadic rows of 2^(M-CLO) >= 2^10 outputs, 4..32 columns");
  using T = TmemCfg<M, OM>;
  constexpr int TB = T::TB, R = T::R, JW = T::JW;
  // Haar side output (FusedArgs::haar_z; the HZ instantiations, whole signals, dyadic order)
  static_assert(!HZ || (CLO == 0 && OM == 0), "side output of whole signals in dyadic order");
  constexpr int ZM = HZ ? M : 0;
  static_assert(ZM == 0 || reg_label(T::P3, 0) == 0u, "chunk 0, register 0 holds labels with bits 8..13 zero");
  static_assert(XP == 0 || (M == 16 && OM == 0 && CLO == 0 && !HZ && XP == 1),
                "a signal over two SMs: whole 2^17-word signals in dyadic order");
  constexpr uint32_t LMASK = (1u << TB) - 1u;
  constexpr Phase P2 = T::P2, P3 = T::P3;
  constexpr Lin LB = T::LB;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  uint32_t* bufs = reinterpret_cast<uint32_t*>(base);  // row buffers g mod 2
  uint32_t* stage = bufs + (2u << TB);
  uint32_t* xbuf = stage + (1u << TB);  // XP > 0: 32 KB of exchanged values, [piece j][thread]
  uint64_t* bar = reinterpret_cast<uint64_t*>(xbuf + (XP > 0 ? (1u << (TB - 1)) : 0u));
  // XP > 0: readyb[c & 1]: the peer's values of chunk c are in its scratch slot (a remote
  // arrival); loadb: the bulk load of the peer's values into xbuf has landed
  uint64_t* readyb = bar + 2;
  uint64_t* loadb = bar + 4;
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 5);
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
    if (XP > 0) {
      mbar_init(readyb, 1);
      mbar_init(readyb + 1, 1);
      mbar_init(loadb, 1);
    }
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
  const uint32_t rank = XP > 0 ? cluster_ctarank() : 0u;
  if constexpr (XP > 0) {
    cluster_arrive();  // every CTA's barriers exist before a peer signals them
    cluster_wait();
  }
  // this thread's lane and its warp's half of the columns
  const uint32_t taddr = tmem + ((32u * (warp & 3u)) << 16) + (T::NCOLS / 2) * (warp >> 2);

  const int64_t stride = gridDim.x >> XP;
  const int64_t first = blockIdx.x >> XP;
  const int64_t K = first < units ? (units - first + stride - 1) / stride : 0;
  const int64_t G = K * R;  // rows this CTA loads
  // first input element of this CTA's 2^M labels of unit k (signals of 2^(M+XP) words)
  auto elem0 = [&](int64_t k) {
    return unit_elem<M + XP>(args, args.in_off, first + k * stride) + (static_cast<int64_t>(rank) << M);
  };
  auto rowe = [&](int64_t g) { return elem0(g / R) + ((g % R) << TB); };  // first element of row g
  if (tid == 0) {
    if (G > 0) tile_issue_at<TB>(&tin, rowe(0), bufs, bar, args);
    if (G > 1) tile_issue_at<TB>(&tin, rowe(1), bufs + (1u << TB), bar + 1, args);
  }
  BF bf{};
  if constexpr (std::is_same_v<BF, BfF32PerLevel>) bf.c = 0.70710678118654752440f;
  // A wait that gives up records CHW_ERR_TIMEOUT and turns this thread's later waits off.
  bool waiting = true;
  const uint32_t tries = args.wait_tries != 0 ? args.wait_tries : kWaitTries;
  // dyadic: output run of this thread (output bits M-8..M-1) and its staging swizzle;
  // natural: its label bits 0..7 are its output bits 0..7
  const uint32_t tl = thread_label<P3>(lane, warp, 0);
  // column tiles: output bits M-8..M-1 are the column (label bits 0..CLO-1) above
  // bitrev of the row's label bits CLO..7
  const uint32_t rho = CLO == 0 ? bitrev_bits(tl, 8)
                                : ((tl & ((1u << CLO) - 1u)) << (8 - CLO)) | bitrev_bits(tl >> CLO, 8 - CLO);
  // staging swizzle: 16-byte piece c of run rho at piece c ^ (rho & skey) of its 128-byte
  // row -- the TMA's 128-byte swizzle (skey = 7), or for a first pass storing blocks of 16,
  // 8 or 4 columns by TMA, the 64-, 32-byte or no swizzle of their narrower box rows
  // (skey = 3, 1, 0), which permute the same pieces of the same rows
  const uint32_t skey = OM == 1 && args.tma_store ? (1u << ((args.colblock_c != 0 ? args.colblock_c : 5) - 2)) - 1u : 7u;
  const uint32_t sxor = (rho & skey) << 2;
  // The exchange of a signal over two SMs (XP = 1), one chunk at a time: xn is the chunk
  // (counted over this CTA's signals) whose exchange is under way, xstate its step --
  // 1: this CTA's values are being written to its scratch slot; 2: the peer has been told
  // they are there; 3: the load of the peer's values has been issued.  Every thread keeps
  // the same xn and xstate; threads 32 and 0 carry out steps 2 and 3.
  int64_t xn = 0;
  int xstate = 0;
  int64_t nload = 0;  // bulk loads issued on loadb (thread 0)
  auto xslot = [&](uint32_t r, int64_t n) {  // scratch slot of CTA rank r for chunk n
    return args.xscratch + ((((static_cast<int64_t>(first) * 2 + r) * 2 + (n & 1))) << 11);
  };
  auto signal_peer = [&]() {  // thread 32: this CTA's values of chunk xn are in L2
    bulk_wait_all();            // the bulk store of this thread has completed
    fence_proxy_async_global();
    mbar_remote_arrive(readyb + (xn & 1), rank ^ 1u);
  };
  auto load_peer = [&]() {  // thread 0: once the peer's values are in L2, load them into xbuf
    if (waiting && !mbar_wait_cluster_bounded(readyb + (xn & 1), static_cast<uint32_t>((xn >> 1) & 1), tries)) {
      waiting = false;
      atomicCAS(args.status, 0, kStatusTimeout);
    }
    fence_proxy_async_global();
    mbar_arrive_expect_tx(loadb, 32u << 10);
    bulk_load(xbuf, xslot(rank ^ 1u, xn), 32u << 10, loadb);
    ++nload;
  };

  // Row r of signal k: label bits 0..13, then into tensor memory.
  auto row = [&](int64_t k, int r) {
    const int64_t g = k * R + r;
    uint32_t* buf = bufs + ((g & 1) << TB);
    if (waiting && !mbar_wait_bounded(bar + (g & 1), static_cast<uint32_t>((g >> 1) & 1), tries)) {
      waiting = false;
      if (lane == 0) atomicCAS(args.status, 0, kStatusTimeout);
    }
    uint32_t v[64];
    // Haar side output of a whole signal: this row's labels carry the row number above bit 13
    HaarZ hz{};
    if constexpr (ZM > 0) {
      if (args.haar_z != nullptr) {
        hz.z = static_cast<uint32_t*>(args.haar_z) + unit_elem<M>(args, args.out_off, first + k * stride);
        hz.hi = static_cast<uint32_t>(r) << TB;
        hz.limit = 1u << M;
      }
    }
    if constexpr (CLO == 0) {
      phases_1_2<0, TB, TB, 0, BF, 0, ZM, SCALE>(v, elem0(k) + (int64_t{r} << TB), args, buf, bf, &hz);
    } else {
      row_phases_from<CLO>(v, buf, bf);
    }
    if constexpr (!T::b_is_s) __syncthreads();
    store_phase<P2, P2, LB, LMASK>(v, buf, thread_pos<P2, LB, LMASK>(lane, warp, 0));
    __syncthreads();
    if constexpr (XP > 0) {  // the exchange of the previous chunk advances during the row
      if (xstate == 1) {
        if (tid == 32) signal_peer();
        xstate = 2;
      }
    }
    load_phase<P3, LB, LMASK>(v, buf, thread_pos<P3, LB, LMASK>(lane, warp, 0));
    bfly<P3, 11, TB, 0, BF, ZM, SCALE>(v, bf, lane, warp, &hz);
    __syncthreads();  // the row buffer is no longer read: refill it
    if (tid == 0 && g + 2 < G) tile_issue_at<TB>(&tin, rowe(g + 2), buf, bar + (g & 1), args);
    if constexpr (XP > 0) {
      if (xstate == 2) {  // (thread 32's store has completed: the barrier above orders it)
        if (tid == 0) load_peer();
        xstate = 3;
      }
    }
    const uint32_t par = static_cast<uint32_t>(k & 1);
    tmem_st16<0>(taddr + tmem_col<M>(par, r, 0), v);
    tmem_st16<16>(taddr + tmem_col<M>(par, r, 16), v);
    tmem_st16<32>(taddr + tmem_col<M>(par, r, 32), v);
    tmem_st16<48>(taddr + tmem_col<M>(par, r, 48), v);
    tmem_wait_st();
  };

  // Label bit M (XP = 1) of output chunk q of signal k, in two steps around the next row's
  // phases so that the exchange overlaps them.  cross_send: u holds the chunk's values with
  // label bits 0..M-1 done; the value at dyadic position 64 q + w of the thread's run within
  // this CTA's 2^M labels is u[src(q, w)].  The thread keeps the 32 values of the half
  // w >> 5 = rank and writes the other half to xbuf (16-byte piece j of thread t at piece
  // 256 j + t), which thread 32 copies to this CTA's scratch slot.  cross_finish: the peer's
  // values of the kept half, loaded into xbuf the same way, are butterflied with the kept
  // ones (the rank-0 CTA's value first) and stored: the thread's 64 outputs are the
  // consecutive words
  //   2 (rho 2^8 + 64 q + 32 rank + j) + e = rho 2^9 + 64 (2 q + rank) + 2 j + e
  // of the signal (e = label bit M), staged and stored by TMA like the other chunks.
  auto cross_send = [&](int64_t k, int q, uint32_t (&u)[64], uint32_t (&keep)[32]) {
    const bool hi = rank != 0;
    uint32_t give[32];
    sfor<32>([&](auto jj) {
      constexpr int j = jj;
      const uint32_t lo = u[T::src(0, j)], up = u[T::src(0, 32 + j)];
      keep[j] = hi ? up : lo;
      give[j] = hi ? lo : up;
    });
    // xbuf is free: the previous chunk's values were read before the last barrier
#pragma unroll
    for (int j = 0; j < 8; ++j)
      *reinterpret_cast<uint4*>(xbuf + 4u * ((j << 8) + tid)) =
          make_uint4(give[4 * j], give[4 * j + 1], give[4 * j + 2], give[4 * j + 3]);
    fence_proxy_async_smem();
    __syncthreads();
    xn = k * R + q;
    if (tid == 32) {
      bulk_store(xslot(rank, xn), xbuf, 32u << 10);
      bulk_commit_group();
    }
    xstate = 1;
  };
  auto cross_finish = [&](int64_t k, int q, const uint32_t (&keep)[32]) {
    const bool hi = rank != 0;
    if (xstate == 1) {  // no row ran since cross_send (the last signal)
      if (tid == 32) signal_peer();
      __syncthreads();
      xstate = 2;
    }
    if (xstate == 2) {
      if (tid == 0) load_peer();
      xstate = 3;
    }
    if (waiting && !mbar_wait_bounded(loadb, static_cast<uint32_t>(xn & 1), tries)) {
      waiting = false;
      if (lane == 0) atomicCAS(args.status, 0, kStatusTimeout);
    }
    xstate = 0;
    uint32_t v[64];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint4 t = *reinterpret_cast<const uint4*>(xbuf + 4u * ((j << 8) + tid));
      const uint32_t g[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        uint32_t a = hi ? g[f] : keep[4 * j + f], b = hi ? keep[4 * j + f] : g[f];
        bf(a, b);
        v[8 * j + 2 * f] = a;
        v[8 * j + 2 * f + 1] = b;
      }
    }
    if constexpr (SCALE) {
#pragma unroll
      for (int i = 0; i < 64; ++i) v[i] = __float_as_uint(__fmul_rn(__uint_as_float(v[i]), args.end_scale));
    }
    const int64_t ob = unit_elem<M + XP>(args, args.out_off, first + k * stride);
    const uint32_t xr = 64u * ((static_cast<uint32_t>(q) << 1) | rank);  // within the output run
    if (args.diag_out != nullptr) {  // D acts on the stored positions (64 consecutive)
      const int64_t at = (static_cast<int64_t>(rho) << (M + XP - 8)) + xr;
      const int8_t* d = args.diag_out + (at & args.diag_mask);
      if (diag_v16_ok(args.diag_out, args.diag_mask)) {
        sfor<4>([&](auto gg) {
          constexpr int g = gg;
          diag16<BF>(v, d + 16 * g, [](int j) { return 16 * g + j; });
        });
      } else {
#pragma unroll
        for (int i = 0; i < 64; ++i)
          if (d[i] < 0) v[i] = std::is_same_v<BF, BfI32> ? 0u - v[i] : v[i] ^ 0x80000000u;
      }
    }
    if (tid == 0) bulk_wait_read();  // the previous chunk's TMA stores have read the buffer
    __syncthreads();                 // ... and every thread has read its values from xbuf
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const uint32_t box = static_cast<uint32_t>(c >> 3) << (TB - 1);
      *reinterpret_cast<uint4*>(stage + box + ((rho << 5) | ((4u * (c & 7)) ^ sxor))) =
          make_uint4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      if (args.checked && !range_ok(ob, int64_t{1} << (M + XP), args.out_total)) {
        check_fail(args.status, ob);
      } else {
        const int y = static_cast<int>(ob >> (M + XP - 8));
        tma_store_2d(&tout, stage, static_cast<int>(xr), y);
        tma_store_2d(&tout, stage + (1u << (TB - 1)), static_cast<int>(xr) + 32, y);
      }
      bulk_commit_group();
    }
  };

  // Output chunk q of signal k: label bits 14..M-1 on registers [q JW, (q+1) JW) of every
  // row, staged in output order and stored by TMA.
  // qq: the chunk index, a compile-time constant (one copy of the epilogue per chunk) or,
  // where the epilogue is long -- sequency order, the Haar side output, a signal over two
  // SMs -- a run-time int, so that the kernel's code stays within the instruction cache
  // (measured on GB300 at m = 16: sequency 78 -> 90 %, side output 63 -> 70 %, m = 17
  // 62 -> 66 %; the plain dyadic kernel runs 2.7 % faster with constants).
  constexpr bool kRunTimeChunk = OM == 3 || ZM > 0 || XP > 0;
  static_assert(!kRunTimeChunk || OM != 2, "natural-order staging needs the chunk index at compile time");
  auto chunk = [&](int64_t k, auto qq, uint32_t (&keep)[XP > 0 ? 32 : 1]) {
    const int q = static_cast<int>(qq);
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
    // Haar side output of the last label bits: the labels whose bits 0..13 are zero are
    // register 0 of output chunk 0 of the thread with label 0, one per row
    [[maybe_unused]] uint32_t* zs = nullptr;
    if constexpr (ZM > 0) {
      if (q == 0 && args.haar_z != nullptr && tl == 0u)
        zs = static_cast<uint32_t*>(args.haar_z) + unit_elem<M>(args, args.out_off, first + k * stride);
    }
    sfor<M - TB>([&](auto bb) {  // label bit TB + b pairs rows r and r + 2^b
      constexpr int b = bb;
      sfor<R>([&](auto rr) {
        constexpr int r = rr;
        if constexpr (((r >> b) & 1) == 0) {
          sfor<JW>([&](auto j) { bf(u[r * JW + j], u[(r | (1 << b)) * JW + j]); });
        }
      });
      if constexpr (ZM > 0) {
        if (zs != nullptr) {  // rows with bit b set and bits below it zero: level TB + b + 1
          sfor<R>([&](auto rr) {
            constexpr int r = rr;
            if constexpr ((r & ((2 << b) - 1)) == (1 << b)) {
              constexpr float sc = end_scale_const(TB + b + 1);
              uint32_t val = u[r * JW];
              if constexpr (SCALE) val = __float_as_uint(__fmul_rn(__uint_as_float(val), sc));
              zs[(1u << (M - TB - b - 1)) + (static_cast<uint32_t>(r) >> (b + 1))] = val;
            }
          });
        }
      }
    });
    if constexpr (ZM > 0) {
      if (zs != nullptr) {  // the approximation: label 0 after every level
        uint32_t val = u[0];
        if constexpr (SCALE) val = __float_as_uint(__fmul_rn(__uint_as_float(val), end_scale_const(M)));
        zs[0] = val;
      }
    }
    if constexpr (XP > 0) {
      cross_send(k, q, u, keep);
      return;
    }
    if constexpr (SCALE) {
#pragma unroll
      for (int i = 0; i < 64; ++i) u[i] = __float_as_uint(__fmul_rn(__uint_as_float(u[i]), args.end_scale));
    }
    const int64_t ob = unit_elem<M>(args, args.out_off, first + k * stride);
    if constexpr (OM == 2) {
      constexpr int qn = decltype(qq)::value;
      constexpr uint32_t qo = T::nat_qo(0, qn * JW);
      if (args.diag_out != nullptr) {  // D acts on the stored positions
        const int8_t* d = args.diag_out + (tl & args.diag_mask);
        sfor<64>([&](auto ii) {
          constexpr int r = ii / JW, j = ii % JW;
          constexpr int64_t o = T::nat_high(r, qn * JW + j);  // output bits 8..M-1
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
        constexpr uint32_t psi = T::nat_psi(r, qn * JW + j);
        sb[(psi << 5) | ((xc ^ (psi & 7u)) << 2)] = u[ii];
      });
      fence_proxy_async_smem();
      __syncthreads();
      if (tid == 0) {
        if (args.checked && !range_ok(ob, int64_t{1} << M, args.out_total)) {
          check_fail(args.status, ob);
        } else {
          const int y = static_cast<int>(ob >> (M - 6));
#pragma unroll
          for (int b = 0; b < 8; ++b) tma_store_2d(&tout, stage + (b << 11), static_cast<int>(qo) * 256 + 32 * b, y);
        }
        bulk_commit_group();
      }
    } else if constexpr (OM == 3) {
      // Sequency order: dyadic position p = rho 2^L + 64 q + w (L = M - 8) is stored at
      // gray^{-1}(p).  Its run is dr = gray^{-1}(rho); inside the run the 64-word segment is
      // gray^{-1}(q), complemented when dr is odd; inside the segment the 4-word group c of w
      // goes to gray^{-1}(c), complemented when parity(q) differs from dr's parity, and its
      // four words are reordered by parity(c) against that.  So the chunk is staged in its
      // final order as four TMA boxes (even or odd destination runs, 128 rows each, times the
      // two 32-word halves of the segment) and leaves through the 3-D view {2^L words, run
      // parity, run pair} of the output, like the other orders, off the SM's store path.
      constexpr uint32_t L = M - 8;
      constexpr uint32_t qmask = (1u << (L - 6)) - 1u;
      const uint32_t gq = gray_inverse(static_cast<uint32_t>(q)), pq = parity_of(static_cast<uint32_t>(q));
      const uint32_t dr = gray_inverse(rho);
      const uint32_t pd = dr & 1u, zr = dr >> 1, zx = zr & 7u;
      const uint32_t fx = pq ^ pd;                 // complement inside the segment
      const uint32_t qd = gq ^ (pd ? qmask : 0u);  // the segment in the destination run
      if (tid == 0) bulk_wait_read();  // the previous chunk's TMA stores have read the buffer
      __syncthreads();
      uint32_t* srow = stage + (pd << (TB - 2)) + (zr << 5);
      sfor<16>([&](auto cc) {
        constexpr int c = cc;
        constexpr int s0 = T::src(0, 4 * c), s1 = T::src(0, 4 * c + 1);
        constexpr int s2 = T::src(0, 4 * c + 2), s3 = T::src(0, 4 * c + 3);
        constexpr uint32_t gc = gray_inverse(c), pc = parity_of(c);
        const uint32_t C = gc ^ (fx ? 15u : 0u);
        uint4 val = (pc ^ fx) ? make_uint4(u[s2], u[s3], u[s1], u[s0]) : make_uint4(u[s0], u[s1], u[s3], u[s2]);
        if (args.diag_out != nullptr) {  // D acts on the stored positions
          const int64_t at = ob + ((static_cast<int64_t>(dr) << L) | (qd << 6) | (C << 2));
          const int8_t* dg = args.diag_out + (at & args.diag_mask);
          uint32_t* e[4] = {&val.x, &val.y, &val.z, &val.w};
#pragma unroll
          for (int f = 0; f < 4; ++f)
            if (dg[f] < 0) *e[f] = std::is_same_v<BF, BfI32> ? 0u - *e[f] : *e[f] ^ 0x80000000u;
        }
        *reinterpret_cast<uint4*>(srow + ((C >> 3) << (TB - 1)) + (((C & 7u) ^ zx) << 2)) = val;
      });
      fence_proxy_async_smem();
      __syncthreads();
      if (tid == 0 && args.checked && !range_ok(ob, int64_t{1} << M, args.out_total)) {
        check_fail(args.status, ob);
        bulk_commit_group();
      } else if (tid == 0) {
        const int z = static_cast<int>(ob >> (L + 1));
#pragma unroll
        for (int pp = 0; pp < 2; ++pp)
#pragma unroll
          for (int h = 0; h < 2; ++h)
            tma_store_3d(&tout, stage + (h << (TB - 1)) + (pp << (TB - 2)),
                         static_cast<int>(64 * (gq ^ (pp ? qmask : 0u)) + 32 * h), pp, z);
        bulk_commit_group();
      }
    } else {
      if (OM == 0 && args.diag_out != nullptr) {  // D acts on the stored positions
        // (a column tile's outputs are a part of a longer signal: its place in it counts);
        // the thread's 64 outputs of the chunk are consecutive: four 16-byte loads of D
        const int64_t at = (CLO > 0 ? ob : 0) + (static_cast<int64_t>(rho) << (M - 8));
        const int8_t* d = args.diag_out + (at & args.diag_mask) + 64 * q;
        if (diag_v16_ok(args.diag_out, args.diag_mask)) {
          sfor<4>([&](auto gg) {
            constexpr int g = gg;
            diag16<BF>(u, d + 16 * g, [](int j) { return T::src(0, 16 * g + j); });
          });
        } else {
          sfor<64>([&](auto ww) {
            constexpr int w = ww;
            constexpr int si = T::src(0, w);
            if (d[w] < 0) u[si] = std::is_same_v<BF, BfI32> ? 0u - u[si] : u[si] ^ 0x80000000u;
          });
        }
      }
      if (tid == 0) bulk_wait_read();  // the previous chunk's TMA stores have read the buffer
      __syncthreads();
      // Output low bits 64 q + w of run rho: box w / 32, row rho, 16-byte chunk (w mod 32) / 4
      // XOR rho mod 8 (the TMA's 128-byte swizzle).
      sfor<16>([&](auto cc) {
        constexpr int c = cc;
        constexpr int s0 = T::src(0, 4 * c), s1 = T::src(0, 4 * c + 1);
        constexpr int s2 = T::src(0, 4 * c + 2), s3 = T::src(0, 4 * c + 3);
        constexpr uint32_t box = (c >> 3) << (TB - 1);
        *reinterpret_cast<uint4*>(stage + box + ((rho << 5) | ((4u * (c & 7)) ^ sxor))) =
            make_uint4(u[s0], u[s1], u[s2], u[s3]);
      });
      if constexpr (OM == 0) {
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
          if (args.checked && !range_ok(ob, int64_t{1} << M, args.out_total)) {
            check_fail(args.status, ob);
          } else {
            const int y = static_cast<int>(ob >> (M - 8));
            tma_store_2d(&tout, stage, 64 * q, y);
            tma_store_2d(&tout, stage + (1u << (TB - 1)), 64 * q + 32, y);
          }
          bulk_commit_group();
        }
      } else if (OM == 1 && args.tma_store) {
        // Column blocks of 2^c (c = 2..5): the 2^c-word segment g of row r (signal s) lives
        // at s 2^(a+M) + g 2^(a+c) + 2^c r.  Box h of the staged chunk holds, for every run
        // rho, the segments g = rho 2^(M-8-c) + (64 q + 32 h) / 2^c + i, i < 2^(5-c), so each
        // box is one tensor store through the 5-D view {2^c words, r, g mod 2^(M-8-c), rho,
        // s} of the scratch.
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
          const int64_t u = first + k * stride;
          const int cba = args.colblock_a;
          const int64_t sig0 = (u >> cba) << (cba + M);
          if (args.checked && !range_ok(sig0, int64_t{1} << (cba + M), args.out_total)) {
            check_fail(args.status, sig0);
          } else {
            const int r = static_cast<int>(u & ((int64_t{1} << cba) - 1)), s = static_cast<int>(u >> cba);
            const int cw = args.colblock_c != 0 ? args.colblock_c : 5;
            tma_store_5d(&tout, stage, 0, r, (64 * q) >> cw, 0, s);
            tma_store_5d(&tout, stage + (1u << (TB - 1)), 0, r, (64 * q + 32) >> cw, 0, s);
          }
          bulk_commit_group();
        }
      } else {
        // The column-blocked order of the first of two passes sends every 2^w-element
        // segment of a row to its own block, so the chunk goes out through the SM: a warp
        // copies four aligned 32-element pieces of the staged chunk.
        static_assert(OM == 1, "dyadic, natural and sequency chunks leave by TMA stores");
        __syncthreads();
        uint32_t* out = static_cast<uint32_t*>(args.out);
        // OM = 1: row u is row r = u mod 2^a of signal u / 2^a (a = colblock_a); its element
        // k goes to signal * 2^(a+M) + (k / 2^w) 2^(a+w) + 2^w r + k mod 2^w, 2^w = the
        // column block's width (w = colblock_c, 32 columns by default)
        const int64_t u = first + k * stride;
        const int cba = args.colblock_a;
        const int cbw = args.colblock_c != 0 ? args.colblock_c : 5;
        const int64_t cb_base = ((u >> cba) << (cba + M)) + ((u & ((int64_t{1} << cba) - 1)) << cbw);
        // every address below lies in the signal's 2^(a+M) elements: checked once
        const int64_t sig0 = (u >> cba) << (cba + M);
        const bool skip = args.checked && !range_ok(sig0, int64_t{1} << (cba + M), args.out_total);
        if (skip && tid == 0) check_fail(args.status, sig0);
#pragma unroll 4
        for (int i = skip ? (1 << (TB - 2)) : static_cast<int>(tid); i < (1 << (TB - 2)); i += kTmemThreads) {
          const uint32_t h = static_cast<uint32_t>(i) >> (TB - 3), run = (static_cast<uint32_t>(i) >> 3) & 255u;
          const uint32_t c8 = static_cast<uint32_t>(i) & 7u;
          uint4 val = *reinterpret_cast<const uint4*>(stage + (h << (TB - 1)) + (run << 5) + ((c8 ^ (run & 7u)) << 2));
          // dyadic position / 4 within the signal
          const uint32_t p4 = (run << (M - 10)) | static_cast<uint32_t>(16 * q) | (h << 3) | c8;
          const uint32_t e = p4 << 2;  // a 4-word chunk never straddles a block (w >= 2)
          const int64_t addr = cb_base + (static_cast<int64_t>(e >> cbw) << (cba + cbw)) + (e & ((1u << cbw) - 1u));
          st_global_v4(out + addr, val.x, val.y, val.z, val.w);
        }
      }
    }
  };

  // Software pipeline: output chunk i of signal t-1 frees the tensor-memory columns that
  // row i of signal t fills, so every step reads one row and writes one chunk.
  // With XP = 1 the chunk's exchange with the peer runs while this CTA transforms the row.
  for (int64_t t = 0; t <= K; ++t) {
#pragma unroll 1
    for (int i = 0; i < R; ++i) {
      uint32_t keep[XP > 0 ? 32 : 1];
      if (t >= 1) {
        if constexpr (kRunTimeChunk) {
          chunk(t - 1, i, keep);
        } else {
          sfor<R>([&](auto qq) {
            if (static_cast<int>(qq) == i) chunk(t - 1, qq, keep);
          });
        }
      }
      if (t < K) row(t, i);
      if constexpr (XP > 0) {
        if (t >= 1) cross_finish(t - 1, i, keep);
      }
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
  if constexpr (XP > 0) {
    if (tid == 32) bulk_wait_all();  // the exchange stores too
    // and the last load into xbuf (already waited for, unless a wait above gave up)
    if (tid == 0 && nload > 0) mbar_wait_bounded(loadb, static_cast<uint32_t>((nload - 1) & 1), kWaitTries);
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(tmem, T::NCOLS);
  if constexpr (XP > 0) {
    cluster_arrive();  // no CTA leaves while a peer may still write into it or signal it
    cluster_wait();
  }
}

}  // namespace chw
