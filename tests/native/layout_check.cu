// Host-only check of the staging layouts the kernels' TMA stores rely on, computed with the
// kernels' own constexpr plans and, for the column-blocked first pass of a two-pass split,
// the plan's own tensor view (no GPU): every staged position is hit exactly once, the TMA
// box that reads it fits the buffer it is read from and writes the output position the
// cascade defines.  Prints "ALL OK".
#include <cstdio>
#include <vector>

#include "colblock.h"
#include "tmem.cuh"

using namespace chw;

static bool g_ok = true;
#define CHECK(cond, ...)           \
  do {                             \
    if (!(cond)) {                 \
      std::printf(__VA_ARGS__);    \
      std::printf("\n");           \
      g_ok = false;                \
      return;                      \
    }                              \
  } while (0)

// Fused single-CTA tile in dyadic order: staged position of label L, and the 4-D box
// {32 words, bits S..S+2, bits 5..S-1, bits S+3..} with SWIZZLE_128B that the tile store uses.
template <int TLO, int M, int TB>
void fused_tile_store() {
  constexpr FusedPlan F = make_plan(TLO, M, TB, 0, 0);
  const int S = F.stage_s;
  const uint32_t N = 1u << TB;
  std::vector<int> seen(N, 0);
  for (uint32_t L = 0; L < N; ++L) {
    const uint32_t o = apply(F.omap, L) & (N - 1);
    const uint32_t pos = apply(F.lin_final, L);
    CHECK(pos == staged_pos(o, S, true), "fused TLO=%d M=%d: staged position of L=%u", TLO, M, L);
    const uint32_t c0 = o & 31u, c1 = (o >> S) & 7u, c2 = (o >> 5) & ((1u << (S - 5)) - 1u), c3 = o >> (S + 3);
    const uint32_t row = c1 + 8u * c2 + (8u << (S - 5)) * c3;
    CHECK(row * 32u + ((((c0 >> 2) ^ (row & 7u)) << 2)) + (c0 & 3u) == pos, "fused TLO=%d M=%d: box of o=%u", TLO, M, o);
    CHECK(c0 + (c1 << S) + (c2 << 5) + (c3 << (S + 3)) == o, "fused: global coordinates of o=%u", o);
    seen[pos]++;
  }
  for (uint32_t i = 0; i < N; ++i) CHECK(seen[i] == 1, "fused TLO=%d M=%d: position %u staged %d times", TLO, M, i, seen[i]);
  std::printf("fused tile store TLO=%d M=%2d TB=%d S=%2d ok\n", TLO, M, TB, S);
}

// Thread label bits of phase P (lanes and warps), as the kernels' thread_label computes them.
uint32_t thread_label_host(const Phase& p, uint32_t lane, uint32_t warp) {
  return lane_label(p, static_cast<int>(lane)) | warp_label(p, static_cast<int>(warp));
}

// Tensor-memory kernel, dyadic order (output modes 0 and 1): the labels staged for output
// chunk q.  Run rho's 16-byte piece c (0..15: half c / 8 of its 64 outputs) lands at piece
// (c mod 8) ^ (rho & skey) of row rho of half c / 8 of the staging buffer; -1 where nothing
// is staged; *ok turns false if two values share a word.
template <int M>
std::vector<int64_t> stage_dyadic(int q, uint32_t skey, bool* ok) {
  using T = TmemCfg<M, 0>;
  std::vector<int64_t> stage(1u << kTmemTB, -1);
  for (uint32_t warp = 0; warp < 8; ++warp)
    for (uint32_t lane = 0; lane < 32; ++lane) {
      const uint32_t tl = thread_label_host(T::P3, lane, warp);
      const uint32_t rho = bitrev_bits(tl, 8), sxor = (rho & skey) << 2;
      for (int c = 0; c < 16; ++c)
        for (int e = 0; e < 4; ++e) {
          const int si = T::src(q, 4 * c + e);
          const int r = si / T::JW, j = si % T::JW;
          const uint32_t label = tl | reg_label(T::P3, q * T::JW + j) | (static_cast<uint32_t>(r) << kTmemTB);
          const uint32_t p = ((c >> 3) << (kTmemTB - 1)) + (((rho << 5) | (4u * (c & 7))) ^ sxor) + e;
          if (stage[p] >= 0) {
            std::printf("tmem M=%d q=%d: staged twice at %u\n", M, q, p);
            *ok = false;
          }
          stage[p] = label;
        }
    }
  return stage;
}

// Tensor-memory kernel, dyadic order: chunk q's staging (two 32-word x 256-row boxes,
// SWIZZLE_128B) against the dyadic output position bitrev_M(label).
template <int M>
void tmem_dyadic() {
  using T = TmemCfg<M, 0>;
  const uint32_t n = 1u << M;
  std::vector<int> out(n, 0);
  for (int q = 0; q < T::R; ++q) {
    bool ok = true;
    const std::vector<int64_t> stage = stage_dyadic<M>(q, 7u, &ok);
    CHECK(ok, "tmem M=%d: staging", M);
    for (uint32_t h = 0; h < 2; ++h)
      for (uint32_t row = 0; row < 256; ++row)
        for (uint32_t x = 0; x < 32; ++x) {
          const uint32_t sm = (h << (kTmemTB - 1)) + row * 32u + ((((x >> 2) ^ (row & 7u))) << 2) + (x & 3u);
          const uint32_t pos = (row << (M - 8)) + 64u * q + 32u * h + x;
          CHECK(stage[sm] >= 0 && pos == bitrev_bits(static_cast<uint32_t>(stage[sm]), M), "tmem M=%d: box of pos %u", M, pos);
          out[pos]++;
        }
  }
  for (uint32_t i = 0; i < n; ++i) CHECK(out[i] == 1, "tmem M=%d: output %u written %d times", M, i, out[i]);
  std::printf("tmem dyadic M=%d ok\n", M);
}

// Tensor-memory kernel, sequency order: dyadic position p goes to gray^{-1}(p) (the s with
// s ^ (s >> 1) = p, from a table built from that definition).  The kernel stages run rho's
// 16-byte group c of chunk q at group C = gray^{-1}(c), complemented when parity(q) differs
// from the destination run's parity, with its words reordered by parity(c) against that,
// in box (destination run parity, C / 8) at row (destination run / 2); four TMA stores,
// each 32 words x 1 x 128 run pairs with the 128-byte swizzle, write the boxes at segment
// gray^{-1}(q) (complemented for odd destination runs) of the 3-D view {2^(M-8) words,
// run parity, run pair}.  Every output is written once, with the right value.
template <int M>
void tmem_sequency() {
  using T = TmemCfg<M, 3>;
  constexpr uint32_t L = M - 8, qmask = (1u << (L - 6)) - 1u;
  const uint32_t n = 1u << M;
  std::vector<uint32_t> ginv(n);
  for (uint32_t x = 0; x < n; ++x) ginv[x ^ (x >> 1)] = x;
  std::vector<int> out(n, 0);
  for (int q = 0; q < T::R; ++q) {
    std::vector<int64_t> stage(1u << kTmemTB, -1);
    const uint32_t gq = gray_inverse(static_cast<uint32_t>(q)), pq = parity_of(static_cast<uint32_t>(q));
    for (uint32_t warp = 0; warp < 8; ++warp)
      for (uint32_t lane = 0; lane < 32; ++lane) {
        const uint32_t tl = thread_label_host(T::P3, lane, warp);
        const uint32_t rho = bitrev_bits(tl, 8);
        const uint32_t dr = gray_inverse(rho), pd = dr & 1u, zr = dr >> 1, zx = zr & 7u, fx = pq ^ pd;
        for (uint32_t c = 0; c < 16; ++c) {
          const uint32_t C = gray_inverse(c) ^ (fx ? 15u : 0u);
          const int order[2][4] = {{0, 1, 3, 2}, {2, 3, 1, 0}};  // value word e' <- group word
          for (int e = 0; e < 4; ++e) {
            const int si = T::src(q, 4 * static_cast<int>(c) + order[parity_of(c) ^ fx][e]);
            const int r = si / T::JW, j = si % T::JW;
            const uint32_t label = tl | reg_label(T::P3, q * T::JW + j) | (static_cast<uint32_t>(r) << kTmemTB);
            const uint32_t sm = (pd << (kTmemTB - 2)) + (zr << 5) + ((C >> 3) << (kTmemTB - 1)) + (((C & 7u) ^ zx) << 2) + e;
            CHECK(stage[sm] < 0, "sequency M=%d q=%d: staged twice at %u", M, q, sm);
            stage[sm] = label;
          }
        }
      }
    for (uint32_t pp = 0; pp < 2; ++pp)
      for (uint32_t h = 0; h < 2; ++h)
        for (uint32_t zl = 0; zl < 128; ++zl)
          for (uint32_t x = 0; x < 32; ++x) {
            const uint32_t sm = (h << (kTmemTB - 1)) + (pp << (kTmemTB - 2)) + zl * 32u + (((x >> 2) ^ (zl & 7u)) << 2) + (x & 3u);
            const uint32_t xc = 64u * (gq ^ (pp ? qmask : 0u)) + 32u * h + x;  // the view's coordinates
            const uint32_t pos = ((2u * zl + pp) << L) + xc;
            CHECK(stage[sm] >= 0, "sequency M=%d: box reads an unstaged word", M);
            CHECK(pos == ginv[bitrev_bits(static_cast<uint32_t>(stage[sm]), M)], "sequency M=%d: box of pos %u", M, pos);
            out[pos]++;
          }
  }
  for (uint32_t i = 0; i < n; ++i) CHECK(out[i] == 1, "sequency M=%d: output %u written %d times", M, i, out[i]);
  std::printf("tmem sequency M=%d ok\n", M);
}

// Tensor-memory kernel as the first pass of a two-pass split (output mode 1), its chunks
// written by TMA stores through the column-blocked view `colblock_view` (the plan's own
// encoding).  The kernel stages with key 2^(c-2) - 1 for blocks of 2^c columns.  The box is
// laid out in shared memory as the TMA lays it out: rows of 2^c words at a pitch of the
// swizzle span when the row is narrower than it, and the span's XOR of the 16-byte piece
// bits with the bits above 128 bytes.  It must fit the 32 KB half of the staging buffer it
// is read from, and read every staged element into the place the column-blocked layout
// gives its dyadic output position k: s 2^(a+M) + (k >> c) 2^(a+c) + 2^c r + (k mod 2^c)
// for row r of signal s.  Every word of the scratch is written once.
template <int M>
void tmem_colblock(int a, int c) {
  using T = TmemCfg<M, 1>;
  static_assert(T::R == TmemCfg<M, 0>::R && T::JW == TmemCfg<M, 0>::JW, "modes 0 and 1 share the row layout");
  const int64_t sigs = 2, total = sigs << (a + M);
  const ColblockView v = colblock_view(total, M, a, c);
  const uint32_t row_bytes = 4u * v.box[0];
  const uint32_t span = v.swizzle == CU_TENSOR_MAP_SWIZZLE_128B  ? 128u
                        : v.swizzle == CU_TENSOR_MAP_SWIZZLE_64B ? 64u
                        : v.swizzle == CU_TENSOR_MAP_SWIZZLE_32B ? 32u
                                                                 : 0u;
  const uint32_t pitch = span > row_bytes ? span : row_bytes;
  const uint32_t box_bytes = pitch * v.box[1] * v.box[2] * v.box[3] * v.box[4];
  CHECK(box_bytes <= (4u << (kTmemTB - 1)), "colblock M=%d c=%d: a box takes %u bytes of shared memory, more than %u",
        M, c, box_bytes, 4u << (kTmemTB - 1));
  const uint32_t pbits = span == 128u ? 3u : span == 64u ? 2u : span == 32u ? 1u : 0u;  // piece bits the span permutes
  std::vector<int> hits(static_cast<size_t>(total), 0);
  for (int q = 0; q < T::R; ++q) {
    bool ok = true;
    const std::vector<int64_t> stage = stage_dyadic<M>(q, (1u << (c - 2)) - 1u, &ok);
    CHECK(ok, "colblock M=%d c=%d: staging", M, c);
    for (int64_t s = 0; s < sigs; ++s)
      for (int64_t r = 0; r < (int64_t{1} << a); ++r)
        for (uint32_t h = 0; h < 2; ++h)
          for (uint32_t rho = 0; rho < v.box[3]; ++rho)
            for (uint32_t gl = 0; gl < v.box[2]; ++gl)
              for (uint32_t w = 0; w < v.box[0]; ++w) {
                const uint32_t o = (rho * v.box[2] + gl) * pitch + 4u * w;  // byte in the box before the swizzle
                const uint32_t phys = o ^ (((o >> 7) & ((1u << pbits) - 1u)) << 4);
                const int64_t label = stage[(h << (kTmemTB - 1)) + phys / 4u];
                CHECK(label >= 0, "colblock M=%d c=%d: the box reads an unstaged word", M, c);
                const uint64_t k = bitrev_bits(static_cast<uint32_t>(label), M);
                const uint64_t x[5] = {w, static_cast<uint64_t>(r), ((64u * q + 32u * h) >> c) + gl, rho,
                                       static_cast<uint64_t>(s)};
                for (int i = 0; i < 5; ++i) CHECK(x[i] < v.dims[i], "colblock M=%d c=%d: coordinate %d out of range", M, c, i);
                const uint64_t addr =
                    x[0] + (x[1] * v.strides[0] + x[2] * v.strides[1] + x[3] * v.strides[2] + x[4] * v.strides[3]) / 4u;
                const uint64_t want = (static_cast<uint64_t>(s) << (a + M)) + ((k >> c) << (a + c)) +
                                      (static_cast<uint64_t>(r) << c) + (k & ((1u << c) - 1u));
                CHECK(addr == want, "colblock M=%d a=%d c=%d: label %lld stored at %llu, defined at %llu", M, a, c,
                      static_cast<long long>(label), static_cast<unsigned long long>(addr),
                      static_cast<unsigned long long>(want));
                hits[addr]++;
              }
  }
  for (int64_t i = 0; i < total; ++i) CHECK(hits[i] == 1, "colblock M=%d c=%d: word %lld written %d times", M, c,
                                             static_cast<long long>(i), hits[i]);
  std::printf("tmem column blocks M=%d a=%d c=%d (%u-byte box rows, swizzle span %u) ok\n", M, a, c, row_bytes, span);
}

// Tensor-memory kernel, natural order: eight 32-word x 64-row boxes per chunk.
template <int M>
void tmem_natural() {
  using T = TmemCfg<M, 2>;
  const uint32_t n = 1u << M;
  std::vector<int> out(n, 0);
  for (int q = 0; q < T::R; ++q) {
    const uint32_t qo = T::nat_qo(0, q * T::JW);
    std::vector<int64_t> stage(1u << kTmemTB, -1);
    for (uint32_t warp = 0; warp < 8; ++warp)
      for (uint32_t lane = 0; lane < 32; ++lane) {
        const uint32_t tl = thread_label_host(T::P3, lane, warp);
        for (int ii = 0; ii < 64; ++ii) {
          const int r = ii / T::JW, j = ii % T::JW;
          const uint32_t psi = T::nat_psi(r, q * T::JW + j);
          const uint32_t p = ((tl >> 5) << 11) + (tl & 3u) + ((psi << 5) | (((((tl >> 2) & 7u)) ^ (psi & 7u)) << 2));
          CHECK(stage[p] < 0, "tmem natural M=%d: staged twice at %u", M, p);
          stage[p] = tl | T::nat_high(r, q * T::JW + j);
        }
      }
    for (uint32_t b = 0; b < 8; ++b)
      for (uint32_t row = 0; row < 64; ++row)
        for (uint32_t x = 0; x < 32; ++x) {
          const uint32_t sm = (b << 11) + row * 32u + ((((x >> 2) ^ (row & 7u))) << 2) + (x & 3u);
          const uint32_t pos = (row << (M - 6)) + qo * 256u + 32u * b + x;
          CHECK(stage[sm] >= 0 && pos == static_cast<uint32_t>(stage[sm]), "tmem natural M=%d: box of pos %u", M, pos);
          out[pos]++;
        }
  }
  for (uint32_t i = 0; i < n; ++i) CHECK(out[i] == 1, "tmem natural M=%d: output %u written %d times", M, i, out[i]);
  std::printf("tmem natural M=%d ok\n", M);
}

// Haar-Walsh head (output mode 6): the copy-out gathers final position p of a signal of
// 2^M words from staged (dyadic-order) element qe = ((p - 2^k) << (M - k)) | 2^(M-1-k),
// k = the top bit of p (p = 0: qe = 0), restated from the kernel.  By eq. (4) scale k
// holds H_k of the signal's block [2^k, 2^(k+1)) in dyadic order, so final position
// 2^k + bitrev_k(j) is the block's label 2^k + j, staged at dyadic position
// bitrev_M(2^k + j).  Every final position must take that element, each exactly once.
static uint32_t bitrev(uint32_t x, int n) {
  uint32_t r = 0;
  for (int i = 0; i < n; ++i) r |= ((x >> i) & 1u) << (n - 1 - i);
  return r;
}
void head_gather(int M) {
  const uint32_t n = 1u << M;
  std::vector<int> used(n, 0);
  for (uint32_t p = 0; p < n; ++p) {
    uint32_t qe = 0;
    if (p != 0) {
      int k = 31;
      while (((p >> k) & 1u) == 0) --k;
      qe = ((p - (1u << k)) << (M - k)) | (1u << (M - 1 - k));
    }
    // the definition: the label whose final position is p
    uint32_t label = 0;
    if (p != 0) {
      int k = 31;
      while (((p >> k) & 1u) == 0) --k;
      label = (1u << k) + bitrev(p - (1u << k), k);
    }
    CHECK(qe < n && qe == bitrev(label, M), "head M=%d: final %u gathers %u, expected %u", M, p, qe, bitrev(label, M));
    used[qe]++;
  }
  for (uint32_t i = 0; i < n; ++i) CHECK(used[i] == 1, "head M=%d: staged %u used %d times", M, i, used[i]);
  std::printf("head M=%d ok\n", M);
}

int main() {
  for (int M = 0; M <= 14; ++M) head_gather(M);
  // every single-CTA dyadic shape the library instantiates: rows of m = 0..14 and the
  // two-pass column tiles of 2^a rows x 32 columns, a = 6..9
  fused_tile_store<0, 0, 13>();
  fused_tile_store<0, 1, 13>();
  fused_tile_store<0, 2, 13>();
  fused_tile_store<0, 3, 13>();
  fused_tile_store<0, 4, 13>();
  fused_tile_store<0, 5, 13>();
  fused_tile_store<0, 6, 13>();
  fused_tile_store<0, 7, 13>();
  fused_tile_store<0, 8, 13>();
  fused_tile_store<0, 9, 13>();
  fused_tile_store<0, 10, 13>();
  fused_tile_store<0, 11, 13>();
  fused_tile_store<0, 12, 13>();
  fused_tile_store<0, 13, 13>();
  fused_tile_store<0, 14, 14>();
  fused_tile_store<5, 6, 13>();
  fused_tile_store<5, 7, 13>();
  fused_tile_store<5, 8, 13>();
  fused_tile_store<5, 9, 14>();
  tmem_dyadic<15>();
  tmem_dyadic<16>();
  tmem_natural<15>();
  tmem_natural<16>();
  tmem_sequency<15>();
  tmem_sequency<16>();
  for (int c = 2; c <= 5; ++c) {
    tmem_colblock<15>(2, c);
    tmem_colblock<16>(3, c);
  }
  std::printf(g_ok ? "ALL OK\n" : "FAILED\n");
  return g_ok ? 0 : 1;
}
