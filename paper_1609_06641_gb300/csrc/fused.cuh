// One-HBM-round-trip CHW kernel for 4-byte elements (fp32, int32).
//
// A CTA owns a tile of 2^TB consecutive elements; a thread-block cluster of 2^CB CTAs
// owns 2^(TB+CB).  The tile is brought into shared memory by TMA (SWIZZLE_128B), then
// up to three register phases run the butterflies (label bits 0-4, 5-10, 11+; see
// engine.cuh), the last of them reading the other CTAs' shared memory over DSMEM when
// the transform spans the cluster.  Results are staged in shared memory in output order
// and copied out with coalesced 16-byte stores.
//
// Two uses:
//   TLO = 0  row transform: each tile holds 2^(TB-M) whole signals of length 2^M (CB = 0)
//            or one 2^TB slice of a 2^(TB+CB) signal (CB > 0).  Output in dyadic order.
//   TLO = 5  column transform (second pass of the two-pass split): the tile is a
//            2^M x 32 block (32 columns of a row-transformed signal, stored contiguously
//            by the first pass); the transform runs over the 2^M rows of each column and
//            column c's results form the contiguous output row c (Y = H_b X^T H_a).
//
// Output modes (OUTMODE): where each result is stored.  The butterflies never change.
//   0  dyadic order (the paper's H_m): label j is output bitrev(j);
//   1  column-blocked scratch for the first pass of the two-pass split (dyadic rows);
//   2  natural (Sylvester) order: label j is output j.  Row tiles stage in natural order;
//      column tiles write each of their 32 columns as a stride-2^b run (the first pass ran
//      in mode 4), where b = FusedArgs::nat_b is the first pass's bit count;
//   3  sequency (Walsh) order: dyadic output p is sequency output gray^{-1}(p).  Tiles
//      stage in dyadic order; the copy-out sends each aligned 4-element chunk to
//      gray^{-1} of its position, which keeps the chunk together (reordered inside);
//   4  column-blocked scratch with natural row order (first pass of a natural two-pass);
//   6  the head of the Haar-Walsh transform (eq. (4)): positions [0, 2^M) of a signal of
//      Haar coefficients hold the scales k = 0..M-1 at [2^k, 2^{k+1}), each transformed by
//      its own H_k.  The tile runs the 2^M-point cascade with the pairs that belong to
//      stage 0 (no label bit above the butterfly bit) skipped, which leaves exactly the
//      per-scale transforms; dyadic staged position o (o != 0) is scale
//      k = M-1-ctz(o), entry o >> (ctz(o)+1), stored at 2^k + (o >> (ctz(o)+1)).
#pragma once

#include "engine.cuh"

namespace chw {

constexpr int kStatusTimeout = 6;      // CHW_ERR_TIMEOUT
constexpr int kStatusDeviceCheck = 7;  // CHW_ERR_DEVICE_CHECK
constexpr uint32_t kWaitTries = 1u << 22;

struct FusedArgs {
  void* out;                 // output array base (global)
  int64_t out_total;         // elements of `out` that may be written (tail tiles stop there)
  float end_scale;           // multiply applied to every result when the kernel's SCALE is set
  const int8_t* diag_in;     // +-1 applied to inputs (adjoint's D), or nullptr
  const int8_t* diag_out;    // +-1 applied to outputs (forward's D), or nullptr
  int64_t diag_mask;         // index within a signal = element index & diag_mask
  int* status;               // device status word (first error wins)
  int colblock_a;            // OUTMODE 1, 4: rows per signal = 2^colblock_a
  int colblock_c;            // tensor-memory rows of a first pass: 2^colblock_c columns per
                             //   column block (0: 32, the fused kernels' only width)
  int order_m;               // OUTMODE 3: bits of a signal (sequency order is per signal)
  int nat_b;                 // OUTMODE 2, column tiles: the first pass's bits (row stride 2^b)
  int head_end;              // OUTMODE 6: scale scale k by fp32(2^{-k/2}) on output (END)
  int64_t unit_stride;       // unit u's elements start at unit_base + u * unit_stride
  int64_t unit_base;         //   (0 = the default: units back to back, 2^(TB+CB) apart)
  // Signals at arbitrary offsets (ragged batches): when set, unit u belongs to signal
  // u >> sig_shift and starts 2^(TB+CB) * (u mod 2^sig_shift) elements into it, the
  // signal starting at in_off[] in the input and at out_off[] in the output.
  const int64_t* in_off;
  const int64_t* out_off;
  int sig_shift;
  // Test hook of the cluster kernel's failure detection: the CTA of rank stall_cta - 1
  // (0: none) withholds its first "full" signal, and waits give up after `wait_tries`
  // polls (0: kWaitTries), so the other CTAs' bounded waits run out and report
  // CHW_ERR_TIMEOUT while every CTA still finishes.
  int stall_cta;
  uint32_t wait_tries;
  // Output by TMA tensor stores (batched single-CTA tiles in dyadic order, outputs one
  // contiguous run per tile, no D): `tout` views the output as tile_store_map describes.
  int tma_store;
  // Checked mode (CHW_FLAG_CHECKED): every computed global index is range-checked before
  // it is used -- input rows against [0, in_total), output elements against
  // [0, out_total) -- and a bad one latches CHW_ERR_DEVICE_CHECK with the index into the
  // status words instead of being accessed (the access is skipped; the output is then
  // undefined).
  int checked;
  int64_t in_total;  // elements of the input that may be read (checked mode)
  // Haar side output (chw_forward_haar): z = Psi_m x (eq. (2)) of every signal, written
  // from the same pass at the signal's place in this array (the layout of y); nullptr: none.
  void* haar_z;
  // Signals over a pair of SMs (tensor-memory kernel, XP = 1): the exchange scratch in
  // global memory (L2-resident), four 32 KB slots per cluster (two per CTA, by the chunk
  // parity), room for `xclusters` clusters; the launch keeps its grid within it.
  uint4* xscratch;
  int64_t xclusters;
  CUtensorMap tout;  // the type carries the alignment TMA needs
};

// Checked mode: latch CHW_ERR_DEVICE_CHECK and the offending element index (the first one
// wins; status[2..3] hold the index as an int64).
__device__ __forceinline__ void check_fail(int* status, int64_t index) {
  if (atomicCAS(status, 0, kStatusDeviceCheck) == 0)
    atomicExch(reinterpret_cast<unsigned long long*>(status + 2), static_cast<unsigned long long>(index));
}

// Checked mode: elements [e0, e0 + n) lie inside [0, total).
__device__ __forceinline__ bool range_ok(int64_t e0, int64_t n, int64_t total) {
  return e0 >= 0 && e0 <= total - n;
}

// Element where unit u's input (or output) starts: from a per-signal offset table when
// one is given, else from the unit stride.
template <int UB>
__device__ __forceinline__ int64_t unit_elem(const FusedArgs& a, const int64_t* off, int64_t u) {
  if (off != nullptr) return off[u >> a.sig_shift] + ((u & ((int64_t{1} << a.sig_shift) - 1)) << UB);
  return a.unit_base + u * (a.unit_stride != 0 ? a.unit_stride : (int64_t{1} << UB));
}

// ------------------------------------------------------------------ phase plans
struct FusedPlan {
  bool has_p1, has_p3, p1_final, p2_final;
  Phase p1, p2, p3, fw;  // fw: the final phase in output-write register order
  Phase p2w;             // phase 2 in push order (clusters)
  Lin lin_s, lin_b, lin_final, lin_r;
  bool b_is_s;
  int stage_s;
  Lin omap;
  int rank_shift[4];  // o bit of each CTA-rank label bit (cluster output placement)
};

constexpr bool natural_mode(int OM) { return OM == 2 || OM == 4; }

constexpr Lin make_omap(int TLO, int M, int OM) {
  Lin l = lin_identity();
  if (natural_mode(OM)) return l;  // natural order: label j is output j
  if (TLO == 0) {
    for (int b = 0; b < M; ++b) l.img[b] = 1u << (M - 1 - b);
  } else {
    for (int b = 0; b < 5; ++b) l.img[b] = 1u << (M + b);
    for (int b = 5; b < 5 + M; ++b) l.img[b] = 1u << (M + 4 - b);
  }
  return l;
}

constexpr Phase make_p1(int TB) {
  Phase p{};
  p.nreg = 6;
  const int r[6] = {0, 1, 2, 3, 4, 10};
  for (int i = 0; i < 6; ++i) p.reg[i] = r[i];
  for (int i = 0; i < 5; ++i) p.lane[i] = 5 + i;
  p.nwarp = TB - 11;
  for (int i = 0; i < p.nwarp; ++i) p.warp[i] = 11 + i;
  return p;
}

constexpr Phase make_p2(int TB, int TLO, int M) {
  Phase p{};
  p.nreg = 6;
  const int top = TLO + M - 1;
  int n = 0;
  if (top <= 10 && top >= 5) {
    for (int b = top; b >= 5; --b) p.reg[n++] = b;
    for (int b = top + 1; b <= 10; ++b) p.reg[n++] = b;
  } else {
    for (int b = 5; b <= 10; ++b) p.reg[n++] = b;
  }
  const int l[5] = {4, 3, 2, 1, 0};
  for (int i = 0; i < 5; ++i) p.lane[i] = l[i];
  p.nwarp = TB - 11;
  for (int i = 0; i < p.nwarp; ++i) p.warp[i] = 11 + i;
  return p;
}

constexpr Phase make_p3(int TB, int CB, int TLO, int M) {
  Phase p{};
  const int nb = TB + CB;
  const int top = TLO + M - 1;
  // CTA-rank and lane bits per (TLO, CB).  Lane bits 0..2 (a quarter warp) set the staging
  // swizzle key; in a cluster two of the lanes are phase-2 register labels so that phase 2
  // can push 16-byte chunks to the CTA that finishes them.
  const int ctas[2][4][3] = {{{-1, -1, -1}, {0, -1, -1}, {0, 1, -1}, {0, 1, 2}},
                             {{-1, -1, -1}, {4, -1, -1}, {4, 3, -1}, {4, 3, 2}}};
  const int lanes[2][4][5] = {{{4, 3, 2, 1, 0}, {4, 3, 2, 5, 6}, {4, 3, 2, 5, 6}, {5, 4, 3, 6, 7}},
                              {{4, 3, 2, 1, 0}, {1, 2, 3, 5, 6}, {0, 1, 2, 5, 6}, {0, 1, 5, 6, 7}}};
  const int t = TLO == 0 ? 0 : 1;
  bool used[kMaxBits] = {};
  p.ncta = CB;
  for (int i = 0; i < CB; ++i) {
    p.cta[i] = ctas[t][CB][i];
    used[p.cta[i]] = true;
  }
  for (int i = 0; i < 5; ++i) {
    p.lane[i] = lanes[t][CB][i];
    used[p.lane[i]] = true;
  }
  p.nreg = 6;
  int n = 0;
  for (int b = top; b >= 11 && n < 6; --b) {
    p.reg[n++] = b;
    used[b] = true;
  }
  for (int b = 10; b >= 0 && n < 6; --b) {
    if (used[b]) continue;
    p.reg[n++] = b;
    used[b] = true;
  }
  p.nwarp = 0;
  for (int b = 0; b < nb; ++b)
    if (!used[b]) p.warp[p.nwarp++] = b;
  return p;
}

// Write order of a final phase: registers 0 and 1 hold output bits 0 and 1 if possible.
constexpr Phase write_order(const Phase& p, const Lin& omap) {
  int l0 = -1, l1 = -1;
  for (int b = 0; b < kMaxBits; ++b) {
    if (omap.img[b] == 1u) l0 = b;
    if (omap.img[b] == 2u) l1 = b;
  }
  const int i0 = reg_index_of(p, l0), i1 = reg_index_of(p, l1);
  if (i0 < 0 || i1 < 0) return p;
  Phase q = p;
  q.reg[0] = l0;
  q.reg[1] = l1;
  int n = 2;
  for (int i = 0; i < p.nreg; ++i)
    if (p.reg[i] != l0 && p.reg[i] != l1) q.reg[n++] = p.reg[i];
  return q;
}

// bank-XOR pairs for the P2 -> P3 exchange on top of the TMA layout
constexpr Lin make_lin_b(const Phase& p2, const Phase& p3) {
  Lin l = lin_tma128();
  int from[5] = {}, to[5] = {};
  int nf = 0, nt = 0;
  for (int i = 0; i < 5; ++i) {
    bool in3 = false;
    for (int j = 0; j < 5; ++j) in3 |= p3.lane[j] == p2.lane[i];
    if (!in3) to[nt++] = p2.lane[i];
  }
  for (int j = 0; j < 5; ++j) {
    bool in2 = false;
    for (int i = 0; i < 5; ++i) in2 |= p2.lane[i] == p3.lane[j];
    if (!in2) from[nf++] = p3.lane[j];
  }
  // sort both ascending
  for (int a = 0; a < nf; ++a)
    for (int b = a + 1; b < nf; ++b) {
      if (from[b] < from[a]) { int t = from[a]; from[a] = from[b]; from[b] = t; }
      if (to[b] < to[a]) { int t = to[a]; to[a] = to[b]; to[b] = t; }
    }
  for (int i = 0; i < nf; ++i) l.img[from[i]] |= 1u << to[i];
  return l;
}

// Receive layout of the cluster exchange (phase 2 -> phase 3), on the labels a CTA
// finishes (its CTA-rank labels map to nothing): word bits 0,1 hold two phase-3 lane labels
// that are phase-2 registers (16-byte pushes), bits 2..4 the other phase-3 lanes (conflict-
// free phase-3 reads), then the remaining labels in increasing order.
constexpr Lin make_lin_r(const Phase& p2, const Phase& p3, int nb) {
  Lin l{};
  int order[kMaxBits] = {};
  int n = 0, na = 0;
  int ab[2] = {-1, -1};
  for (int j = 0; j < 5 && na < 2; ++j)
    if (reg_index_of(p2, p3.lane[j]) >= 0) ab[na++] = p3.lane[j];
  if (na < 2) return lin_identity();  // rejected by the static checks of FusedCfg
  order[n++] = ab[0];
  order[n++] = ab[1];
  for (int j = 0; j < 5; ++j)
    if (p3.lane[j] != ab[0] && p3.lane[j] != ab[1]) order[n++] = p3.lane[j];
  for (int b = 0; b < nb; ++b) {
    bool skip = false;
    for (int i = 0; i < n; ++i) skip |= order[i] == b;
    for (int i = 0; i < p3.ncta; ++i) skip |= p3.cta[i] == b;
    if (!skip) order[n++] = b;
  }
  for (int i = 0; i < n; ++i) l.img[order[i]] = 1u << i;
  return l;
}

// Phase 2's write order for the pushes: registers 0 and 1 hold the labels at word bits 0, 1.
constexpr Phase push_order(const Phase& p2, const Lin& r) {
  int l0 = -1, l1 = -1;
  for (int i = 0; i < p2.nreg; ++i) {
    if (r.img[p2.reg[i]] == 1u) l0 = p2.reg[i];
    if (r.img[p2.reg[i]] == 2u) l1 = p2.reg[i];
  }
  Phase q = p2;
  if (l0 < 0 || l1 < 0) return q;
  q.reg[0] = l0;
  q.reg[1] = l1;
  int n = 2;
  for (int i = 0; i < p2.nreg; ++i)
    if (p2.reg[i] != l0 && p2.reg[i] != l1) q.reg[n++] = p2.reg[i];
  return q;
}

// Worst conflict degree of the 16-byte pushes: lanes of a quarter warp that go to the same
// CTA must hit distinct 16-byte bank groups.  `src` is the label bits of the pushing CTA.
constexpr int push_conflicts(const Phase& pw, const Lin& r, const Phase& p3) {
  int worst = 1;
  for (int k = 0; k < 64; k += 4)
    for (int q = 0; q < 4; ++q)
      for (int d = 0; d < 8; ++d) {
        int count[8] = {};
        for (int ln = 8 * q; ln < 8 * q + 8; ++ln) {
          const uint32_t lab = reg_label(pw, k) | lane_label(pw, ln);
          int dest = 0;
          for (int i = 0; i < p3.ncta; ++i) dest |= static_cast<int>((lab >> p3.cta[i]) & 1u) << i;
          if (dest != d) continue;
          count[(apply(r, lab) >> 2) & 7]++;
        }
        for (int b = 0; b < 8; ++b) worst = count[b] > worst ? count[b] : worst;
      }
  return worst;
}

// The CTA-rank labels of phase 3 are lane or warp labels of phase 2 (one destination per thread).
constexpr bool push_dest_per_thread(const Phase& p2, const Phase& p3) {
  for (int i = 0; i < p3.ncta; ++i)
    if (reg_index_of(p2, p3.cta[i]) >= 0) return false;
  return true;
}

constexpr bool lin_equal(const Lin& a, const Lin& b) {
  for (int i = 0; i < kMaxBits; ++i)
    if (a.img[i] != b.img[i]) return false;
  return true;
}

constexpr int pick_stage_key(const Phase& fw, const Lin& omap, int TB) {
  int ob[3] = {};
  for (int j = 0; j < 3; ++j) {
    const uint32_t im = omap.img[fw.lane[j]];
    int bit = 0;
    while ((1u << bit) != im) ++bit;
    ob[j] = bit;
  }
  for (int a = 0; a < 3; ++a)
    for (int b = a + 1; b < 3; ++b)
      if (ob[b] < ob[a]) { int t = ob[a]; ob[a] = ob[b]; ob[b] = t; }
  if (ob[0] >= 5 && ob[1] == ob[0] + 1 && ob[2] == ob[0] + 2 && ob[2] < TB) return ob[0];
  return 5;
}

// Tiles whose staged outputs form one contiguous run (dyadic order, single CTA) stage their
// 128-byte rows permuted so that the staging key -- output bits S..S+2, which XOR the
// 16-byte chunk index -- becomes the row index's low three bits: the layout of a TMA
// SWIZZLE_128B box over the 4-D view (32 words, bits S..S+2, bits 5..S-1, bits S+3..) of
// the output (tile_store_map).  The identity when S = 5.
constexpr bool tile_store_layout(int OM, int CB) { return OM == 0 && CB == 0; }

constexpr Lin lin_stage_rows(int s) {
  Lin l = lin_identity();
  for (int b = 5; b < kMaxBits; ++b) {
    if (b >= s && b < s + 3) {
      l.img[b] = 1u << (5 + b - s);
    } else if (b < s) {
      l.img[b] = 1u << (b + 3);
    }
  }
  return l;
}

// Staged position of output o (within a tile) for staging key s: the chunk swizzle, then
// (tile-store layout) the row permutation of lin_stage_rows.
__host__ __device__ constexpr uint32_t staged_pos(uint32_t o, int s, bool rows) {
  uint32_t p = o ^ (((o >> s) & 7u) << 2);
  if (rows && s > 5)
    p = (p & 31u) | (((p >> s) & 7u) << 5) | (((p >> 5) & ((1u << (s - 5)) - 1u)) << 8) | ((p >> (s + 3)) << (s + 3));
  return p;
}

constexpr FusedPlan make_plan(int TLO, int M, int TB, int CB, int OM) {
  FusedPlan f{};
  const int top = TLO + M;  // one past the last transform bit
  f.has_p1 = TLO == 0;
  f.p1_final = TLO == 0 && top <= 5;
  f.p2_final = !f.p1_final && top <= 11;
  f.has_p3 = top > 11;
  f.p1 = make_p1(TB);
  f.p2 = make_p2(TB, TLO, M);
  f.p3 = make_p3(TB, CB, TLO, M);
  f.omap = make_omap(TLO, M, OM);
  f.lin_s = lin_tma128();
  f.lin_b = make_lin_b(f.p2, f.p3);
  f.lin_r = CB > 0 ? make_lin_r(f.p2, f.p3, TB + CB) : lin_identity();
  f.p2w = push_order(f.p2, f.lin_r);
  f.b_is_s = lin_equal(f.lin_b, f.lin_s);
  const Phase fin = f.p1_final ? f.p1 : (f.p2_final ? f.p2 : f.p3);
  f.fw = write_order(fin, f.omap);
  f.stage_s = pick_stage_key(f.fw, f.omap, TB);
  Lin fl = compose(lin_stage(f.stage_s), f.omap);
  if (tile_store_layout(OM, CB)) fl = compose(lin_stage_rows(f.stage_s), fl);
  for (int i = 0; i < kMaxBits; ++i) fl.img[i] &= (1u << TB) - 1u;
  f.lin_final = fl;
  for (int i = 0; i < 4; ++i) f.rank_shift[i] = 0;
  for (int i = 0; i < CB; ++i) {
    int bit = 0;
    while ((1u << bit) != f.omap.img[f.p3.cta[i]]) ++bit;
    f.rank_shift[i] = bit;
  }
  return f;
}

template <int TLO, int M, int TB, int CB, int OM = 0>
struct FusedCfg {
  static constexpr FusedPlan plan = make_plan(TLO, M, TB, CB, OM);
  static constexpr int NB = TB + CB;
  static constexpr uint32_t LMASK = (1u << TB) - 1u;
  static_assert(TB >= 11 && TB <= 15, "tile must hold 64 values x 32 lanes x >=1 warp");
  static_assert(TLO == 0 || TLO == 5, "transform starts at label bit 0 (rows) or 5 (columns)");
  static_assert((OM >= 0 && OM <= 4) || OM == 6, "output modes 0..4 and 6");
  static_assert(OM != 6 || (TLO == 0 && CB == 0), "the Haar-Walsh head is a single-CTA row tile");
  static_assert(!natural_mode(OM) || CB == 0, "natural order is staged by single-CTA tiles");
  static_assert(OM != 4 || TLO == 0, "mode 4 is a first (row) pass");
  static_assert(CB == 0 || TLO + M == NB, "a cluster tile holds exactly one transform");
  static_assert(TLO + M <= NB && M >= 0, "transform must fit the tile");
  static_assert(TLO + M <= 17, "at most three register phases");
  static_assert(CB == 0 || plan.has_p3, "cluster bits are finished by the third phase");
  static_assert(!plan.has_p1 || phase_covers(plan.p1, TB), "phase 1 covers the tile");
  static_assert(phase_covers(plan.p2, TB), "phase 2 covers the tile");
  static_assert(!plan.has_p3 || phase_covers(plan.p3, NB), "phase 3 covers the cluster tile");
  // bank-conflict freedom of every shared-memory access
  static_assert(!plan.has_p1 || (v4_ok(plan.p1, plan.lin_s, LMASK) &&
                                 conflict_degree(plan.p1, plan.lin_s, LMASK, true) == 1),
                "phase 1 reads the TMA tile with conflict-free 16-byte loads");
  static_assert(conflict_degree(plan.p2, plan.lin_s, LMASK, false) == 1, "phase 2 reads are conflict-free");
  static_assert(!plan.has_p3 || CB > 0 || conflict_degree(plan.p2, plan.lin_b, LMASK, false) == 1,
                "phase 2 writes are conflict-free");
  static_assert(!plan.has_p3 || CB > 0 || conflict_degree(plan.p3, plan.lin_b, LMASK, false) == 1,
                "phase 3 reads are conflict-free");
  // clusters: 16-byte pushes from phase 2 to the finishing CTA, local phase-3 reads
  static_assert(CB == 0 || push_dest_per_thread(plan.p2, plan.p3), "one push destination per thread");
  static_assert(CB == 0 || v4_ok(plan.p2w, plan.lin_r, ~0u), "pushes are 16-byte chunks");
  static_assert(CB == 0 || push_conflicts(plan.p2w, plan.lin_r, plan.p3) == 1, "pushes are conflict-free");
  static_assert(CB == 0 || conflict_degree(plan.p3, plan.lin_r, ~0u, false) == 1, "phase 3 reads are conflict-free");
  // The final phase writes every value it holds (labels from other CTAs included) into
  // its own staging buffer, so no label bit is masked there.
  static constexpr bool final_v4 = v4_ok(plan.fw, plan.lin_final, ~0u);
  static constexpr int final_conflicts = conflict_degree(plan.fw, plan.lin_final, ~0u, final_v4);
  static_assert(final_conflicts <= (TLO + M <= 6 ? 2 : 1), "staging writes are conflict-free");
  static_assert(plan.stage_s + 3 <= TB, "staging key inside the tile");
};

// ------------------------------------------------------------------ one tile
// Issue the TMA load of a (CTA's part of a) tile: rows [in_row0, in_row0 + 2^(TB-5)) of
// 32 words into `buf`, completing on `bar`.  One thread calls this.  Earlier
// generic-proxy accesses to `buf` must be ordered before it by a barrier.
template <int TB>
__device__ __forceinline__ void tile_issue(const CUtensorMap* tin, int in_row0, uint32_t* buf, uint64_t* bar) {
  constexpr int BOXR = (1 << (TB - 5)) < 256 ? (1 << (TB - 5)) : 256;
  constexpr int NBOX = (1 << (TB - 5)) / BOXR;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  const uint64_t pol = policy_evict_first();
  mbar_arrive_expect_tx(bar, 4u << TB);
#pragma unroll
  for (int j = 0; j < NBOX; ++j) tma_load_2d(buf + j * BOXR * 32, tin, bar, 0, in_row0 + j * BOXR, pol);
}

// tile_issue for a tile whose first input element is e0: in checked mode a tile that does
// not start on a 32-element row inside [0, in_total) is not loaded -- the index is latched
// and the barrier's phase completed by a plain arrival, so the waits still end (the tile
// then holds stale data).  A tile may run past in_total: the tensor map reads zeros there
// (the tail tile of a batch whose length is not a multiple of the tile).
template <int TB>
__device__ __forceinline__ void tile_issue_at(const CUtensorMap* tin, int64_t e0, uint32_t* buf, uint64_t* bar,
                                              const FusedArgs& args) {
  if (args.checked && (e0 < 0 || e0 >= args.in_total || (e0 & 31) != 0)) {
    check_fail(args.status, e0);
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
    return;
  }
  tile_issue<TB>(tin, static_cast<int>(e0 >> 5), buf, bar);
}

// Copy the staged tile (output order, staging swizzle) to global memory with coalesced
// 16-byte stores; `out_base` is the element index of the (cluster) tile's first output.
template <int TLO, int M, int TB, int CB, class BF, int OUTMODE>
__device__ __forceinline__ void copy_out(const uint32_t* buf, int64_t out_base, uint32_t rank, const FusedArgs& args) {
  using Cfg = FusedCfg<TLO, M, TB, CB, OUTMODE>;
  constexpr FusedPlan F = Cfg::plan;
  constexpr int NT = 1 << (TB - 6);
  if constexpr (CB > 0) {
    uint32_t ro = 0;
#pragma unroll
    for (int i = 0; i < CB; ++i) ro |= ((rank >> i) & 1u) << (F.rank_shift[i] - TB);
    out_base += static_cast<int64_t>(ro) << TB;
  }
  uint32_t* out = static_cast<uint32_t*>(args.out);
  constexpr int NCH = 1 << (TB - 2);
  constexpr int S = F.stage_s;
  constexpr bool ROWS = tile_store_layout(OUTMODE, CB);
  if constexpr (OUTMODE == 6) {
    // Haar-Walsh head: the staged tile holds every signal of 2^M words in dyadic order of
    // its labels, and final position p >= 1 (scale k = the top bit of p) takes staged
    // element ((p - 2^k) << (M - k)) | 2^(M-1-k), p = 0 element 0.  Each thread gathers the
    // four staged elements of four consecutive final positions and stores them as 16 bytes.
    constexpr uint32_t mask = (1u << M) - 1u;
    for (int c = threadIdx.x; c < NCH; c += NT) {
      const uint32_t o = static_cast<uint32_t>(c) << 2;  // final position within the tile
      const int64_t at = out_base + o;
      if (at >= args.out_total) continue;
      uint32_t e[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const uint32_t pf = (o + t) & mask, so = (o + t) & ~mask;
        uint32_t qe = 0;
        int k = 0;
        if (pf != 0) {
          k = 31 - __clz(pf);
          qe = ((pf - (1u << k)) << (M - k)) | (1u << (M - 1 - k));
        }
        e[t] = buf[staged_pos(so + qe, S, ROWS)];
        if (args.head_end && pf != 0) e[t] = __float_as_uint(__fmul_rn(__uint_as_float(e[t]), end_scale_dev(k)));
      }
      const int64_t nv = args.out_total - at < 4 ? args.out_total - at : 4;  // a tail chunk holds fewer
      if (args.checked && !range_ok(at, nv, args.out_total)) {
        check_fail(args.status, at);
      } else if (at + 3 < args.out_total) {
        st_global_v4(out + at, e[0], e[1], e[2], e[3]);
      } else {
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (at + t < args.out_total) out[at + t] = e[t];
      }
    }
    return;
  }
  // the same loop with and without the checked mode's range checks, chosen once
  auto loop = [&](auto checked_c) {
  constexpr bool CHECKED = decltype(checked_c)::value;
#pragma unroll 4
  for (int c = threadIdx.x; c < NCH; c += NT) {
    const uint32_t o = static_cast<uint32_t>(c) << 2;
    const uint32_t pos = staged_pos(o, S, ROWS);
    uint4 q = *reinterpret_cast<const uint4*>(buf + pos);
    const int64_t og = out_base + o;  // position in the staged (dyadic or natural) order
    if (og >= args.out_total) continue;
    int64_t addr;
    if constexpr (OUTMODE == 0 || (OUTMODE == 2 && TLO == 0)) {
      addr = og;
    } else if constexpr (OUTMODE == 1 || OUTMODE == 4) {
      // Column-blocked scratch for the two-pass split: element k of row R of a signal with
      // 2^a rows goes to signal*2^(a+M) + (k/32)*2^(a+5) + (R mod 2^a)*32 + k mod 32.
      const int a = args.colblock_a;
      const int64_t R = og >> M;
      const int64_t k = og & ((int64_t{1} << M) - 1);
      const int64_t sig = R >> a, r = R & ((int64_t{1} << a) - 1);
      addr = (sig << (a + M)) + ((k >> 5) << (a + 5)) + (r << 5) + (k & 31);
    } else if constexpr (OUTMODE == 2) {
      // natural column tile: staged element c + 32 R + 2^(5+M) blk is row label R of column
      // 32 cb + c of signal sig, where blk = sig 2^(b-5) + cb numbers the column blocks
      const int b = args.nat_b;
      const int64_t blk = og >> (5 + M);
      const int64_t sig = blk >> (b - 5), cb = blk & ((int64_t{1} << (b - 5)) - 1);
      const int64_t R = (og >> 5) & ((int64_t{1} << M) - 1);
      addr = (sig << (M + b)) + (R << b) + (cb << 5) + (og & 31);
    } else if constexpr (OUTMODE == 6) {
      // Haar-Walsh head: each element goes to its scale's block
      uint32_t e[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int64_t qe = (og + t) & ((int64_t{1} << M) - 1);  // position within the signal
        int64_t pos = 0;
        if (qe != 0) {
          const int c = __ffsll(qe) - 1;
          pos = (int64_t{1} << (M - 1 - c)) | (qe >> (c + 1));
          if (args.head_end) e[t] = __float_as_uint(__fmul_rn(__uint_as_float(e[t]), end_scale_dev(M - 1 - c)));
        }
        const int64_t at = (og + t) - qe + pos;
        if (CHECKED && !range_ok(at, 1, args.out_total)) {
          check_fail(args.status, at);
          continue;
        }
        out[at] = e[t];
      }
      continue;
    } else {
      // sequency: dyadic position p = 4h + e (within the signal) goes to gray^{-1}(p)
      // = 4 gray^{-1}(h) + (e-th entry of {0,1,3,2}, or of {3,2,0,1} when h has odd parity)
      const int64_t p0 = og & ((int64_t{1} << args.order_m) - 1);
      const uint32_t h = static_cast<uint32_t>(p0 >> 2);
      uint32_t g = h;
      g ^= g >> 1;
      g ^= g >> 2;
      g ^= g >> 4;
      g ^= g >> 8;
      g ^= g >> 16;
      addr = (og - p0) + (static_cast<int64_t>(g) << 2);
      q = (__popc(h) & 1) ? make_uint4(q.z, q.w, q.y, q.x) : make_uint4(q.x, q.y, q.w, q.z);
    }
    if (CHECKED && !range_ok(addr, 4, args.out_total)) {
      check_fail(args.status, addr);
      continue;
    }
    if (args.diag_out != nullptr) diag4_at<BF>(q, args, addr);  // D acts on the stored (final) positions
    st_global_v4(out + addr, q.x, q.y, q.z, q.w);
  }
  };
  if (args.checked) {
    loop(std::true_type{});
  } else {
    loop(std::false_type{});
  }
}

// ------------------------------------------------------------------ the diagonal D
// D is an int8 array of +-1: a value's sign flips where its byte is negative (int32:
// negated), i.e. where the byte's top bit is set.
template <class BF>
__device__ __forceinline__ uint32_t diag_apply(uint32_t v, uint32_t top) {  // top: 0 or bit 31
  if constexpr (std::is_same_v<BF, BfI32>) {
    const uint32_t s = static_cast<uint32_t>(static_cast<int32_t>(top) >> 31);
    return (v ^ s) - s;
  } else {
    return v ^ top;
  }
}
// The top bit of byte j (0..3) of w, moved to bit 31.
__device__ __forceinline__ uint32_t byte_top(uint32_t w, int j) { return (w << (24 - 8 * j)) & 0x80000000u; }
// D read as 16-byte vectors: base pointer 16-byte aligned and positions taken modulo at
// least 16 (so a run of 16 never wraps).
__device__ __forceinline__ bool diag_v16_ok(const int8_t* d, int64_t mask) {
  return (reinterpret_cast<uintptr_t>(d) & 15u) == 0u && (mask & 15) == 15;
}
// D on a run of 16 values at consecutive positions, from one 16-byte load (d 16-aligned).
template <class BF, int N, class IDX>
__device__ __forceinline__ void diag16(uint32_t (&v)[N], const int8_t* d, IDX idx) {
  const uint4 w = *reinterpret_cast<const uint4*>(d);
  const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
  sfor<16>([&](auto jj) {
    constexpr int j = jj;
    v[idx(j)] = diag_apply<BF>(v[idx(j)], byte_top(ws[j >> 2], j & 3));
  });
}

// D on four consecutive output positions from `pos` (a multiple of 4): one 4-byte load of
// D where the array allows it.
template <class BF>
__device__ __forceinline__ void diag4_at(uint4& q, const FusedArgs& args, int64_t pos) {
  const int8_t* d = args.diag_out;
  const int64_t di = pos & args.diag_mask;
  if ((reinterpret_cast<uintptr_t>(d) & 3u) == 0u && (args.diag_mask & 3) == 3) {
    const uint32_t w = *reinterpret_cast<const uint32_t*>(d + di);
    q.x = diag_apply<BF>(q.x, byte_top(w, 0));
    q.y = diag_apply<BF>(q.y, byte_top(w, 1));
    q.z = diag_apply<BF>(q.z, byte_top(w, 2));
    q.w = diag_apply<BF>(q.w, byte_top(w, 3));
  } else {
    q.x = diag_apply<BF>(q.x, d[di] < 0 ? 0x80000000u : 0u);
    q.y = diag_apply<BF>(q.y, d[(di + 1) & args.diag_mask] < 0 ? 0x80000000u : 0u);
    q.z = diag_apply<BF>(q.z, d[(di + 2) & args.diag_mask] < 0 ? 0x80000000u : 0u);
    q.w = diag_apply<BF>(q.w, d[(di + 3) & args.diag_mask] < 0 ? 0x80000000u : 0u);
  }
}

// D on the inputs of phase 1 (the adjoint's D): register k holds label tl | reg_label(k),
// and registers 16 g .. 16 g + 15 hold 16 consecutive positions (phase 1 keeps label bits
// 0..3 on register bits 0..3), so each group takes one 16-byte load of D.
template <Phase P, class BF>
__device__ __forceinline__ void diag_in_phase1(uint32_t (&v)[64], const FusedArgs& args, int64_t in_elem0,
                                               uint32_t tl) {
  static_assert((reg_label(P, 1) | reg_label(P, 2) | reg_label(P, 4) | reg_label(P, 8)) == 15u &&
                    reg_label(P, 1) == 1u && reg_label(P, 2) == 2u && reg_label(P, 4) == 4u && reg_label(P, 8) == 8u,
                "phase 1 holds label bits 0..3 on register bits 0..3");
  const int8_t* d = args.diag_in;
  if (diag_v16_ok(d, args.diag_mask) && ((in_elem0 + tl) & 15) == 0) {
    sfor<4>([&](auto gg) {
      constexpr int g = gg;
      const int64_t at = (in_elem0 + (tl | reg_label(P, 16 * g))) & args.diag_mask;
      diag16<BF>(v, d + at, [](int j) { return 16 * g + j; });
    });
  } else {
    sfor<64>([&](auto k) {
      constexpr uint32_t kl = reg_label(P, k);
      const int64_t idx = in_elem0 + (tl | kl);
      if (d[idx & args.diag_mask] < 0) v[k] = std::is_same_v<BF, BfI32> ? 0u - v[k] : v[k] ^ 0x80000000u;
    });
  }
}

// ------------------------------------------------------------------ Haar side output
// Stage 0 of Theorem 1 is the Haar transform Psi_m of eq. (2), and its levels are the
// cascade's butterflies restricted to labels whose lower bits are zero: right after the
// butterfly on label bit t, the label L with bits 0..t-1 zero and bit t one holds its
// level-(t+1) detail, which eq. (2) places at z[2^(m-t-1) + (L >> (t+1))]; after the last
// bit, label 0 holds the approximation z[0].  So z leaves the same pass as y, from the
// registers, bit-identical to chw_haar (END: each coefficient multiplied once by
// fp32(2^(-L/2)), L the levels behind it).
struct HaarZ {
  uint32_t* z;     // z element of the tile's label 0 (nullptr: no side output)
  uint32_t hi;     // label bits of the tile above its own (tensor-memory rows), else 0
  uint32_t limit;  // z elements of the tile that belong to its signals (tail tiles)
};

// fp32(2^(-L/2)), exactly as end_scale_dev forms it.
constexpr float end_scale_const(int L) {
  float r = (L & 1) ? 0.70710678118654752440f : 1.0f;
  for (int i = 0; i < L / 2; ++i) r *= 0.5f;
  return r;
}

// Register k of phase P holds a label captured after bit T (T == ZM: the approximation).
template <int T, int ZM>
constexpr bool z_hit(const Phase& p, int k) {
  const uint32_t rl = reg_label(p, k), smask = (1u << ZM) - 1u;
  return T < ZM ? (rl & ((2u << T) - 1u)) == (1u << T) : (rl & smask) == 0u;
}
// Its z position within the tile, less the thread's part.
template <int T, int ZM>
constexpr uint32_t z_rpart(const Phase& p, int k) {
  const uint32_t rl = reg_label(p, k), smask = (1u << ZM) - 1u;
  return ((rl >> ZM) << ZM) + (T < ZM ? (1u << (ZM - T - 1)) + ((rl & smask) >> (T + 1)) : 0u);
}
// The register holding the captured label at z position `at` (less the thread's part), or -1.
template <int T, int ZM>
constexpr int z_reg_at(const Phase& p, uint32_t at) {
  for (int k = 0; k < (1 << p.nreg); ++k)
    if (z_hit<T, ZM>(p, k) && z_rpart<T, ZM>(p, k) == at) return k;
  return -1;
}
// The thread's part of a z position is a multiple of 4 (no thread-owned label bit lands on
// its two low bits), so four consecutive register positions can leave as one 16-byte store.
template <int T, int ZM>
constexpr bool z_v4_ok(const Phase& p) {
  if (T >= ZM) return false;
  uint32_t tb = 0;
  for (int i = 0; i < 5; ++i) tb |= 1u << p.lane[i];
  for (int i = 0; i < p.nwarp; ++i) tb |= 1u << p.warp[i];
  for (int i = 0; i < p.ncta; ++i) tb |= 1u << p.cta[i];
  return ((tb >> (T + 1)) & 3u) == 0u && ZM - T - 1 >= 2;
}
// The same for eight consecutive positions (one 32-byte store).
template <int T, int ZM>
constexpr bool z_v8_ok(const Phase& p) {
  if (T >= ZM) return false;
  uint32_t tb = 0;
  for (int i = 0; i < 5; ++i) tb |= 1u << p.lane[i];
  for (int i = 0; i < p.nwarp; ++i) tb |= 1u << p.warp[i];
  for (int i = 0; i < p.ncta; ++i) tb |= 1u << p.cta[i];
  return ((tb >> (T + 1)) & 7u) == 0u && ZM - T - 1 >= 3;
}
// All eight positions from `at` (a multiple of 8) are captured in registers.
template <int T, int ZM>
constexpr bool z_full8(const Phase& p, uint32_t at) {
  for (uint32_t i = 0; i < 8; ++i)
    if (z_reg_at<T, ZM>(p, at | i) < 0) return false;
  return true;
}

// The captures after the butterflies of label bit T (T == ZM: the approximation, after the
// last bit) for signals of 2^ZM labels; tl = the thread's label bits (with hz.hi).  Eight
// (four) captures at consecutive z positions leave as one 32-byte (16-byte) store where
// the layout allows; the 32-byte stores need z on a 32-byte boundary, else two 16-byte
// stores are issued.
template <Phase P, int T, int ZM, bool ZEND>
__device__ __forceinline__ void haar_capture(const uint32_t (&v)[64], uint32_t tl, const HaarZ& hz) {
  constexpr uint32_t smask = (1u << ZM) - 1u;
  constexpr uint32_t below = T < ZM ? (1u << T) - 1u : smask;  // label bits that must be zero
  if ((tl & below) != 0u) return;
  const uint32_t tpart = ((tl >> ZM) << ZM) + (T < ZM ? ((tl & smask) >> (T + 1)) : 0u);
  constexpr float sc = end_scale_const(T < ZM ? T + 1 : ZM);
  constexpr bool V4 = z_v4_ok<T, ZM>(P);
  constexpr bool V8 = z_v8_ok<T, ZM>(P);
  const bool a32 = (reinterpret_cast<uintptr_t>(hz.z) & 31u) == 0u;
  auto scaled = [&](uint32_t x) {
    if constexpr (ZEND) x = __float_as_uint(__fmul_rn(__uint_as_float(x), sc));
    return x;
  };
  sfor<64>([&](auto kk) {
    constexpr int k = kk;
    if constexpr (z_hit<T, ZM>(P, k)) {
      constexpr uint32_t rp = z_rpart<T, ZM>(P, k);
      constexpr bool in8 = V8 && z_full8<T, ZM>(P, rp & ~7u);  // part of a complete group of eight
      if constexpr (in8) {
        if constexpr ((rp & 7u) == 0u) {
          constexpr int r1 = z_reg_at<T, ZM>(P, rp | 1u), r2 = z_reg_at<T, ZM>(P, rp | 2u),
                        r3 = z_reg_at<T, ZM>(P, rp | 3u), r4 = z_reg_at<T, ZM>(P, rp | 4u),
                        r5 = z_reg_at<T, ZM>(P, rp | 5u), r6 = z_reg_at<T, ZM>(P, rp | 6u),
                        r7 = z_reg_at<T, ZM>(P, rp | 7u);
          const uint32_t at = tpart + rp;
          if (at + 7u < hz.limit) {
            if (a32) {
              st_global_v8(hz.z + at, scaled(v[k]), scaled(v[r1]), scaled(v[r2]), scaled(v[r3]), scaled(v[r4]),
                           scaled(v[r5]), scaled(v[r6]), scaled(v[r7]));
            } else {
              st_global_v4(hz.z + at, scaled(v[k]), scaled(v[r1]), scaled(v[r2]), scaled(v[r3]));
              st_global_v4(hz.z + at + 4u, scaled(v[r4]), scaled(v[r5]), scaled(v[r6]), scaled(v[r7]));
            }
          } else {
            const uint32_t w[8] = {scaled(v[k]), scaled(v[r1]), scaled(v[r2]), scaled(v[r3]),
                                   scaled(v[r4]), scaled(v[r5]), scaled(v[r6]), scaled(v[r7])};
#pragma unroll
            for (uint32_t i = 0; i < 8; ++i)
              if (at + i < hz.limit) hz.z[at + i] = w[i];
          }
        }
        return;
      }
      constexpr int k1 = z_reg_at<T, ZM>(P, rp | 1u), k2 = z_reg_at<T, ZM>(P, rp | 2u),
                    k3 = z_reg_at<T, ZM>(P, rp | 3u);
      constexpr bool group = V4 && (rp & 3u) == 0u && k1 >= 0 && k2 >= 0 && k3 >= 0;
      constexpr bool member = V4 && (rp & 3u) != 0u && z_reg_at<T, ZM>(P, rp & ~3u) >= 0 &&
                              z_reg_at<T, ZM>(P, (rp & ~3u) | 1u) >= 0 && z_reg_at<T, ZM>(P, (rp & ~3u) | 2u) >= 0 &&
                              z_reg_at<T, ZM>(P, (rp & ~3u) | 3u) >= 0;
      const uint32_t at = tpart + rp;
      if constexpr (group) {
        if (at + 3u < hz.limit)
          st_global_v4(hz.z + at, scaled(v[k]), scaled(v[k1]), scaled(v[k2]), scaled(v[k3]));
      } else if constexpr (!member) {
        if (at < hz.limit) hz.z[at] = scaled(v[k]);
      }
    }
  });
}

// Butterflies of a phase; masked for the Haar-Walsh head when HM > 0; with the Haar side
// output captured bit by bit when ZM > 0 and hz names an output.
template <Phase P, int LO, int HI, int HM, class BF, int ZM = 0, bool ZEND = false>
__device__ __forceinline__ void bfly(uint32_t (&v)[64], const BF& bf, uint32_t lane, uint32_t warp,
                                     const HaarZ* hz = nullptr) {
  if constexpr (HM > 0) {
    butterflies_head<P, LO, HI, HM>(v, bf, thread_label<P>(lane, warp, 0));
  } else if constexpr (ZM > 0) {
    if (hz == nullptr || hz->z == nullptr) {
      butterflies<P, LO, HI>(v, bf);
      return;
    }
    const uint32_t tl = thread_label<P>(lane, warp, 0) | hz->hi;
    sfor<kMaxBits>([&](auto bb) {
      constexpr int b = bb;
      if constexpr (b >= LO && b < HI) {
        butterflies<P, b, b + 1>(v, bf);
        if constexpr (b < ZM) haar_capture<P, b, ZM, ZEND>(v, tl, *hz);
        if constexpr (b == ZM - 1) haar_capture<P, ZM, ZM, ZEND>(v, tl, *hz);
      }
    });
  } else {
    butterflies<P, LO, HI>(v, bf);
  }
}

// Phases 1 and 2 of a tile in `buf` (TMA complete): on return v holds phase 2's values and
// no thread reads `buf` any more once the caller has synchronised.  Only for tiles that
// have a third phase.  ZM, ZEND, hz: the Haar side output (see bfly).
template <int TLO, int M, int TB, int CB, class BF, int HM = 0, int ZM = 0, bool ZEND = false>
__device__ __forceinline__ void phases_1_2(uint32_t (&v)[64], int64_t in_elem0, const FusedArgs& args, uint32_t* buf,
                                           const BF& bf, const HaarZ* hz = nullptr) {
  using Cfg = FusedCfg<TLO, M, TB, CB>;
  constexpr FusedPlan F = Cfg::plan;
  static_assert(F.has_p3, "tiles with a third phase");
  constexpr uint32_t LMASK = Cfg::LMASK;
  constexpr Phase P1 = F.p1, P2 = F.p2;
  constexpr Lin LS = F.lin_s;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  if constexpr (F.has_p1) {
    const uint32_t base = thread_pos<P1, LS, LMASK>(lane, warp, 0);
    load_phase<P1, LS, LMASK>(v, buf, base);
    if (args.diag_in != nullptr) diag_in_phase1<P1, BF>(v, args, in_elem0, thread_label<P1>(lane, warp, 0));
    bfly<P1, 0, 5, HM, BF, ZM, ZEND>(v, bf, lane, warp, hz);
    store_phase<P1, P1, LS, LMASK>(v, buf, base);
    __syncthreads();
  }
  load_phase<P2, LS, LMASK>(v, buf, thread_pos<P2, LS, LMASK>(lane, warp, 0));
  bfly<P2, (TLO > 5 ? TLO : 5), 11, HM, BF, ZM, ZEND>(v, bf, lane, warp, hz);
}

// Push phase 2's values of a cluster tile to the CTAs that finish them (16-byte DSMEM
// stores into their `buf`, receive layout lin_r).
template <int TLO, int M, int TB, int CB>
__device__ __forceinline__ void push_to_finishers(const uint32_t (&v)[64], uint32_t* buf, uint32_t rank) {
  constexpr FusedPlan F = FusedCfg<TLO, M, TB, CB>::plan;
  constexpr Phase P2 = F.p2, P2W = F.p2w, P3 = F.p3;
  constexpr Lin LR = F.lin_r;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t tl = thread_label<P2>(lane, warp, 0) | (rank << TB);
  uint32_t dest = 0;
#pragma unroll
  for (int i = 0; i < CB; ++i) dest |= ((tl >> P3.cta[i]) & 1u) << i;
  uint32_t base = 0;
#pragma unroll
  for (int b = 0; b < TB + CB; ++b)
    if ((tl >> b) & 1u) base ^= LR.img[b];
  store_phase_remote<P2W, P2, LR>(v, mapa_shared(smem_u32(buf), dest), base);
}

// Phase 3 of a cluster tile from the local receive layout, then staging and copy-out.
template <int TLO, int M, int TB, int CB, class BF, bool SCALE, int OUTMODE>
__device__ __forceinline__ void phase_3_out(int64_t out_base, const FusedArgs& args, uint32_t* buf, uint32_t rank,
                                            const BF& bf) {
  constexpr FusedPlan F = FusedCfg<TLO, M, TB, CB, OUTMODE>::plan;
  constexpr Phase P3 = F.p3, FW = F.fw;
  constexpr Lin LR = F.lin_r, LF = F.lin_final;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint32_t v[64];
  load_phase<P3, LR, ~0u>(v, buf, thread_pos<P3, LR, ~0u>(lane, warp, rank));
  butterflies<P3, 11, TLO + M>(v, bf);
  if constexpr (SCALE) {
#pragma unroll
    for (int k = 0; k < 64; ++k) v[k] = __float_as_uint(__fmul_rn(__uint_as_float(v[k]), args.end_scale));
  }
  __syncthreads();
  store_phase<FW, P3, LF, ~0u>(v, buf, thread_pos<FW, LF, ~0u>(lane, warp, rank));
  __syncthreads();
  copy_out<TLO, M, TB, CB, BF, OUTMODE>(buf, out_base, rank, args);
}

// Transform the tile held in `buf` (one CTA, no cluster) once `bar` completes phase
// `parity`: the input's first element is `in_elem0` (for the adjoint's diagonal) and the
// outputs start at element `out_base`.  All threads of the CTA call this; it returns with
// the CTA's output stores issued (a barrier is still needed before `buf` is refilled).
template <int TLO, int M, int TB, int CB, class BF, bool SCALE, int OUTMODE, bool TS = false, bool HZ = false>
__device__ __forceinline__ void tile_compute(int64_t in_elem0, int64_t out_base, const FusedArgs& args,
                                             uint32_t* buf, uint64_t* bar, uint32_t parity) {
  static_assert(CB == 0, "cluster tiles run in the pipelined cluster kernel");
  using Cfg = FusedCfg<TLO, M, TB, CB, OUTMODE>;
  constexpr FusedPlan F = Cfg::plan;
  constexpr uint32_t LMASK = Cfg::LMASK;
  constexpr Phase P1 = F.p1, P2 = F.p2, P3 = F.p3, FW = F.fw;
  constexpr Lin LS = F.lin_s, LB = F.lin_b, LF = F.lin_final;
  constexpr int HM = OUTMODE == 6 ? M : 0;

  const uint32_t tid = threadIdx.x;
  const uint32_t lane = tid & 31u, warp = tid >> 5;
  BF bf{};
  if constexpr (std::is_same_v<BF, BfF32PerLevel>) bf.c = 0.70710678118654752440f;

  if (!mbar_wait_bounded(bar, parity, kWaitTries)) {
    if (lane == 0) atomicCAS(args.status, 0, kStatusTimeout);
  }

  // Haar side output (the HZ instantiations): row tiles of whole signals in dyadic order
  static_assert(!HZ || (TLO == 0 && CB == 0 && OUTMODE == 0 && M >= 1), "side output of whole-signal row tiles");
  constexpr int ZM = HZ ? M : 0;
  constexpr bool ZEND = SCALE;
  HaarZ hz{};
  if constexpr (ZM > 0) {
    if (args.haar_z != nullptr) {
      hz.z = static_cast<uint32_t*>(args.haar_z) + out_base;
      const int64_t left = args.out_total - out_base;
      hz.limit = left < (int64_t{1} << TB) ? static_cast<uint32_t>(left) : (1u << TB);
    }
  }

  uint32_t v[64];
  auto scale_all = [&]() {
    if constexpr (SCALE) {
#pragma unroll
      for (int k = 0; k < 64; ++k) v[k] = __float_as_uint(__fmul_rn(__uint_as_float(v[k]), args.end_scale));
    }
  };

  if constexpr (F.has_p3) {
    phases_1_2<TLO, M, TB, CB, BF, HM, ZM, ZEND>(v, in_elem0, args, buf, bf, &hz);
    if constexpr (!F.b_is_s) __syncthreads();
    store_phase<P2, P2, LB, LMASK>(v, buf, thread_pos<P2, LB, LMASK>(lane, warp, 0));
    __syncthreads();
    load_phase<P3, LB, LMASK>(v, buf, thread_pos<P3, LB, LMASK>(lane, warp, 0));
    bfly<P3, 11, TLO + M, HM, BF, ZM, ZEND>(v, bf, lane, warp, &hz);
    scale_all();
    __syncthreads();
    store_phase<FW, P3, LF, ~0u>(v, buf, thread_pos<FW, LF, ~0u>(lane, warp, 0));
    __syncthreads();
  } else if constexpr (F.has_p1) {
    const uint32_t base = thread_pos<P1, LS, LMASK>(lane, warp, 0);
    load_phase<P1, LS, LMASK>(v, buf, base);
    if (args.diag_in != nullptr) diag_in_phase1<P1, BF>(v, args, in_elem0, thread_label<P1>(lane, warp, 0));
    bfly<P1, 0, (TLO + M < 5 ? TLO + M : 5), HM, BF, ZM, ZEND>(v, bf, lane, warp, &hz);
    if constexpr (F.p1_final) {
      scale_all();
      __syncthreads();
      store_phase<FW, P1, LF, ~0u>(v, buf, thread_pos<FW, LF, ~0u>(lane, warp, 0));
      __syncthreads();
    } else {
      store_phase<P1, P1, LS, LMASK>(v, buf, base);
      __syncthreads();
      load_phase<P2, LS, LMASK>(v, buf, thread_pos<P2, LS, LMASK>(lane, warp, 0));
      bfly<P2, 5, TLO + M, HM, BF, ZM, ZEND>(v, bf, lane, warp, &hz);
      scale_all();
      __syncthreads();
      store_phase<FW, P2, LF, ~0u>(v, buf, thread_pos<FW, LF, ~0u>(lane, warp, 0));
      __syncthreads();
    }
  } else {
    load_phase<P2, LS, LMASK>(v, buf, thread_pos<P2, LS, LMASK>(lane, warp, 0));
    butterflies<P2, (TLO > 5 ? TLO : 5), TLO + M>(v, bf);
    scale_all();
    __syncthreads();
    store_phase<FW, P2, LF, ~0u>(v, buf, thread_pos<FW, LF, ~0u>(lane, warp, 0));
    __syncthreads();
  }
  if constexpr (TS && tile_store_layout(OUTMODE, CB)) {
    if (args.tma_store) {
      // the staged tile goes out as one TMA box (args.tout); every thread orders its staging
      // writes before the async-proxy read, then one thread issues the store
      fence_proxy_async_smem();
      __syncthreads();
      if (tid == 0) {
        if (args.checked && !range_ok(out_base, int64_t{1} << TB, args.out_total)) {
          check_fail(args.status, out_base);
        } else {
          tma_store_4d(&args.tout, buf, 0, 0, 0, static_cast<int>(out_base >> (F.stage_s + 3)));
        }
        bulk_commit_group();
      }
      return;
    }
  }
  copy_out<TLO, M, TB, CB, BF, OUTMODE>(buf, out_base, 0, args);
}

// Load + transform one tile (the persistent ragged kernel's form: no prefetch).
template <int TLO, int M, int TB, int CB, class BF, bool SCALE, int OUTMODE>
__device__ __forceinline__ void fused_tile(const CUtensorMap* tin, int in_row0, int64_t out_base,
                                           const FusedArgs& args, uint32_t* buf, uint64_t* bar, uint32_t parity) {
  if (threadIdx.x == 0) tile_issue<TB>(tin, in_row0, buf, bar);
  tile_compute<TLO, M, TB, CB, BF, SCALE, OUTMODE>(static_cast<int64_t>(in_row0) * 32, out_base, args, buf, bar,
                                                     parity);
}

// 1024-byte aligned start of the dynamic shared buffer (SWIZZLE_128B needs it).
__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  const uint32_t a = smem_u32(p);
  return p + ((1024u - (a & 1023u)) & 1023u);
}

// CTAs per SM the batched kernel is compiled for: two 2^TB-word buffers per CTA.
template <int TB>
constexpr int fused_ctas_per_sm() {
  return TB >= 14 ? 1 : 3;
}

// ------------------------------------------------------------------ the batched kernel
// Persistent: each CTA walks the units u = first, first + stride, ... with two shared
// buffers; the TMA load of unit k+1 is issued before unit k is transformed, so HBM reads
// overlap the butterflies and the stores of the previous unit.
template <int TLO, int M, int TB, int CB, class BF, bool SCALE, int OUTMODE, bool HZ = false>
__global__ void __launch_bounds__(1 << (TB - 6), fused_ctas_per_sm<TB>())
    fused_kernel(const __grid_constant__ CUtensorMap tin, const __grid_constant__ FusedArgs args,
                 const int64_t units) {
  static_assert(CB == 0, "cluster shapes use cluster_kernel");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  uint32_t* buf0 = reinterpret_cast<uint32_t*>(base);
  uint32_t* buf1 = buf0 + (1u << TB);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + (8u << TB));
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const int64_t stride = gridDim.x;
  const int64_t first = blockIdx.x;
  auto elem0 = [&](int64_t u) { return unit_elem<TB>(args, args.in_off, u); };
  if (threadIdx.x == 0 && first < units) tile_issue_at<TB>(&tin, elem0(first), buf0, bar, args);
  int k = 0;
  for (int64_t u = first; u < units; u += stride, ++k) {
    uint32_t* cur = (k & 1) ? buf1 : buf0;
    uint32_t* nxt = (k & 1) ? buf0 : buf1;
    const int64_t un = u + stride;
    if (threadIdx.x == 0 && un < units) {
      if (args.tma_store) bulk_wait_read();  // the previous unit's TMA store has read `nxt`
      tile_issue_at<TB>(&tin, elem0(un), nxt, bar + ((k + 1) & 1), args);
    }
    tile_compute<TLO, M, TB, CB, BF, SCALE, OUTMODE, true, HZ>(elem0(u), unit_elem<TB>(args, args.out_off, u), args,
                                                               cur, bar + (k & 1), (k >> 1) & 1);
    __syncthreads();
  }
  // no TMA load or store left in flight on shared memory, even after a wait gave up
  if (threadIdx.x == 0) {
    if (args.tma_store) bulk_wait_all();
    for (int b = 0; b < 2 && b < k; ++b) {
      const int kl = b + ((k - 1 - b) / 2) * 2;  // this CTA's last unit on buffer b
      mbar_wait_bounded(bar + b, (kl >> 1) & 1, kWaitTries);
    }
  }
}

// ------------------------------------------------------------------ the cluster kernel
// A cluster of 2^CB CTAs owns one unit (a 2^(TB+CB)-element tile) at a time and walks its
// units persistently with three shared buffers per CTA, rotating roles:
//   unit u's input S_u is loaded by TMA into buffer u mod 3;
//   phases 1-2 of unit u read it, after which it receives the pushes R_{u+1} of unit u+1;
//   phase 3, staging and copy-out of unit u+1 then use it, and the TMA load of unit u+3
//   refills it.
// Iteration k: finish unit k-1 (wait "full" for R_{k-1}, phase 3, staging, copy-out),
// issue the TMA load of unit k+1 into the buffer that just became free, then run phases
// 1-2 of unit k, signal every CTA that this buffer may now receive R_{k+1} ("free"), wait
// until every CTA's buffer for R_k is free (signalled an iteration earlier), push, and
// signal "full" for R_k.  Signals are remote mbarrier arrivals with release/acquire at
// cluster scope; every wait is bounded.
constexpr int kClusterBufs = 3;

template <int TB>
constexpr int cluster_smem_bytes() {
  return kClusterBufs * (4 << TB) + 1024 + 128;
}

template <int TLO, int M, int TB, int CB, class BF, bool SCALE, int OUTMODE>
__global__ void __launch_bounds__(1 << (TB - 6), 1)
    cluster_kernel(const __grid_constant__ CUtensorMap tin, const FusedArgs args, const int64_t units) {
  static_assert(CB > 0, "cluster shapes only");
  constexpr int NR = 1 << CB;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  uint32_t* bufs = reinterpret_cast<uint32_t*>(base);
  uint64_t* tma = reinterpret_cast<uint64_t*>(base + kClusterBufs * (4u << TB));
  uint64_t* freeb = tma + kClusterBufs;    // freeb[u % 3]: every CTA's buffer for R_u is free
  uint64_t* fullb = freeb + kClusterBufs;  // fullb[u % 3]: every CTA has pushed R_u here
  const uint32_t tid = threadIdx.x, lane = tid & 31u;
  if (tid == 0) {
    for (int i = 0; i < kClusterBufs; ++i) {
      mbar_init(tma + i, 1);
      mbar_init(freeb + i, NR);
      mbar_init(fullb + i, NR);
    }
    fence_mbar_init();
  }
  cluster_arrive();  // every CTA's barriers exist before any peer signals them
  cluster_wait();
  const uint32_t rank = cluster_ctarank();
  const int64_t stride = gridDim.x >> CB;
  const int64_t first = blockIdx.x >> CB;
  const int64_t K = first < units ? (units - first + stride - 1) / stride : 0;
  auto buf = [&](int64_t i) { return bufs + (i % kClusterBufs) * (int64_t{1} << TB); };  // S_i; R_{i+1}
  // first input / output element of the unit of iteration k
  auto elem0 = [&](int64_t k) { return unit_elem<TB + CB>(args, args.in_off, first + k * stride); };
  auto oelem0 = [&](int64_t k) { return unit_elem<TB + CB>(args, args.out_off, first + k * stride); };
  auto cta_elem0 = [&](int64_t k) { return elem0(k) + (int64_t{rank} << TB); };
  auto row0 = [&](int64_t k) { return static_cast<int>(cta_elem0(k) >> 5); };
  auto par = [](int64_t u) { return static_cast<uint32_t>((u / kClusterBufs) & 1); };
  BF bf{};
  if constexpr (std::is_same_v<BF, BfF32PerLevel>) bf.c = 0.70710678118654752440f;
  // A wait that gives up records CHW_ERR_TIMEOUT and turns every later wait of this thread
  // off, so a broken schedule costs one bounded wait per thread, not one per unit.
  bool waiting = true;
  const uint32_t tries = args.wait_tries != 0 ? args.wait_tries : kWaitTries;
  auto wait_local = [&](uint64_t* b, uint32_t parity) {
    if (waiting && !mbar_wait_bounded(b, parity, tries)) {
      waiting = false;
      if (lane == 0) atomicCAS(args.status, 0, kStatusTimeout);
    }
  };
  auto wait_cluster = [&](uint64_t* b, uint32_t parity) {
    if (waiting && !mbar_wait_cluster_bounded(b, parity, tries)) {
      waiting = false;
      if (lane == 0) atomicCAS(args.status, 0, kStatusTimeout);
    }
  };

  if (tid == 0 && K > 0) tile_issue_at<TB>(&tin, cta_elem0(0), buf(0), tma, args);
  if (tid == 0 && K > 1) tile_issue_at<TB>(&tin, cta_elem0(1), buf(1), tma + 1, args);
  if (tid < NR && K > 0) mbar_remote_arrive(freeb + 0, tid);  // buffer 2 (R_0) starts free
  for (int64_t k = 0; k <= K; ++k) {
    if (k >= 1) {
      // ---- finish unit k-1: its pushes R_{k-1} sit in buffer (k-2) mod 3
      const int64_t u = k - 1;
      wait_cluster(fullb + u % kClusterBufs, par(u));
      phase_3_out<TLO, M, TB, CB, BF, SCALE, OUTMODE>(oelem0(u), args, buf(u + 2), rank, bf);
      __syncthreads();  // buffer (k+1) mod 3 is free: the copy-out has read it
      if (tid == 0 && k + 1 < K) tile_issue_at<TB>(&tin, cta_elem0(k + 1), buf(k + 1), tma + (k + 1) % kClusterBufs, args);
    }
    if (k < K) {
      // ---- phases 1-2 of unit k, then push R_k
      wait_local(tma + k % kClusterBufs, par(k));
      uint32_t v[64];
      phases_1_2<TLO, M, TB, CB, BF>(v, static_cast<int64_t>(row0(k)) * 32, args, buf(k), bf);
      __syncthreads();  // buffer k mod 3 is no longer read: it may receive R_{k+1}
      if (tid < NR) mbar_remote_arrive(freeb + (k + 1) % kClusterBufs, tid);
      wait_cluster(freeb + k % kClusterBufs, par(k));
      push_to_finishers<TLO, M, TB, CB>(v, buf(k + 2), rank);
      __syncthreads();  // every push of this CTA is issued
      if (tid < NR && !(k == 0 && static_cast<int>(rank) + 1 == args.stall_cta)) {
        fence_acq_rel_cluster();
        mbar_remote_arrive(fullb + k % kClusterBufs, tid);
      }
    }
  }
  // Leave no TMA load in flight into this CTA's shared memory, even when a wait above gave
  // up: wait (bounded) for the last load issued on each barrier.
  if (tid == 0) {
    for (int64_t i = 0; i < kClusterBufs && i < K; ++i) {
      const int64_t u = i + ((K - 1 - i) / kClusterBufs) * kClusterBufs;
      mbar_wait_bounded(tma + i, par(u), kWaitTries);
    }
  }
  cluster_arrive();  // no CTA leaves while a peer may still push into it or signal it
  cluster_wait();
}

}  // namespace chw
