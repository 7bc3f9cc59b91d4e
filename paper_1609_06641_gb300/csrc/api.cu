// C ABI of the CHW library: plans, validation, tier choice, launches, host pipeline.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/chw.h"
#include "colblock.h"
#include "launch.cuh"
#include "ragged.cuh"
#include "simple.cuh"
#include "lowp.cuh"
#include "tune.h"

namespace chw {
using LowpLaunchFn = cudaError_t (*)(const CUtensorMap*, const CUtensorMap*, const LowpArgs&, int64_t, cudaStream_t);
LowpLaunchFn lookup_lowp(int m, bool f16, bool end);
using RowstackLaunchFn = cudaError_t (*)(const CUtensorMap*, const FusedArgs&, uint32_t*, int64_t, int64_t,
                                         cudaStream_t);
RowstackLaunchFn lookup_rowstack(int m, int var);
int64_t haar_scratch_words(int m, int64_t batch);
cudaError_t haar_forward(int var, int m, int64_t batch, const void* x, void* z, uint32_t* scratch, int* status,
                         cudaStream_t st);
cudaError_t haar_inverse(int var, int m, int64_t batch, const void* z, void* x, uint32_t* scratch, cudaStream_t st);
}  // namespace chw

namespace {

thread_local std::string g_err;

chw_status_t fail(chw_status_t s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define CHW_CUDA(expr)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess) return fail(CHW_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

enum Tier {
  kTierSimple = 0,
  kTierFused = 1,
  kTierCluster = 2,
  kTierTwoPass = 3,
  kTierRagged = 4,
  kTierLowp = 5,
  kTierRowStack = 6,
  kTierTmem = 7,
  kTierTmemCross = 8
};

struct Shape {
  int tb, cb;
};

// Tile bits preferred for cluster shapes: 14 (64 KiB tiles, one CTA per SM) or 13
// (32 KiB tiles in twice as many CTAs, three per SM); CHW_CLUSTER_TILE_BITS overrides.
int cluster_tile_bits() {
  static const int v = [] {
    const char* e = std::getenv("CHW_CLUSTER_TILE_BITS");
    return (e && std::atoi(e) == 13) ? 13 : 14;
  }();
  return v;
}

// Column bits a of the two-pass split y = H_b X^T H_a for m = 18..30 (b = m - a row bits).
// Measured on GB300 (fp32, 1 GiB per call): single-CTA tiles in both passes are fastest
// up to m = 23 (a = 9); beyond, the first pass runs rows of 2^15 or 2^16 words on the
// tensor-memory kernel, so b = m - a is kept at 15..16 with the column pass as small as
// that allows: a = max(9, m - 16).  Column passes of a = 10..14 bits run on the
// tensor-memory kernel as well (column blocks of 2^a rows x 2^min(5, 16-a) columns, at
// most 2^16 words); the fused and cluster column kernels take a <= 12, so sequency order
// (whose column pass they run) keeps a <= 12.  CHW_TWO_PASS_A (6..14, m - a in 5..17)
// overrides it (tuning).
int two_pass_col_bits(int m, int order = 0) {
  static const int v = [] {
    const char* e = std::getenv("CHW_TWO_PASS_A");
    return e ? std::atoi(e) : 0;
  }();
  const int amax = order == 2 ? 12 : 14;
  if (v >= 6 && v <= amax && m - v <= 17 && m - v >= 5) return v;
  if (m <= 23) return 9;
  const int a = m - 16 > 9 ? m - 16 : 9;
  return a < amax ? a : amax;
}

// One-pass row kernel shape for a transform of M bits; `tb` = preferred CTA tile bits for
// shapes that span more than a 2^13-word tile (13 or 14; 0: the default above).
Shape row_shape(int M, int tb = 0) {
  if (tb == 0) tb = cluster_tile_bits();
  if (M <= 13) return {13, 0};
  if (M <= 16 && tb == 13) return {13, M - 13};
  if (M == 14) return {14, 0};
  return {14, M - 14};
}
// Second-pass column kernel shape for A row bits (32 columns per block).
Shape col_shape(int A, int tb = 0) {
  if (tb == 0) tb = cluster_tile_bits();
  if (A <= 8) return {13, 0};
  if (A <= 11 && tb == 13) return {13, A - 8};
  if (A == 9) return {14, 0};
  return {14, A - 9};
}

bool is_lowp(chw_dtype_t d) { return d == CHW_BF16 || d == CHW_F16; }
size_t elem_bytes(chw_dtype_t d) { return is_lowp(d) ? 2 : 4; }

// fp32(2^{-m/2}): 2^{-floor(m/2)} times (1 or fp32(1/sqrt2)); exact power-of-two scaling of
// the correctly rounded constant is itself correctly rounded in fp32's normal range.
float end_scale_f32(int m) {
  const float r = (m & 1) ? 0.70710678118654752440f : 1.0f;
  return std::ldexp(r, -(m / 2));
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// View `total` 4-byte words at `ptr` as rows of 32 words (128 B); box of `boxr` rows,
// SWIZZLE_128B, out-of-bounds rows read as zero.
chw_status_t make_rows_map(CUtensorMap* map, const void* ptr, int64_t total, int tb) {
  auto enc = tensor_map_encoder();
  if (!enc) return fail(CHW_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  if (total % 32 != 0) return fail(CHW_ERR_INVALID_ARG, "internal: tensor rows need a multiple of 32 words");
  const int boxr = (1 << (tb - 5)) < 256 ? (1 << (tb - 5)) : 256;
  cuuint64_t dims[2] = {32, static_cast<cuuint64_t>(total / 32)};
  cuuint64_t strides[1] = {128};
  cuuint32_t box[2] = {32, static_cast<cuuint32_t>(boxr)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(CHW_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
  return CHW_OK;
}

// View `total` 4-byte words at `ptr` as rows of 2^run_bits words; boxes of 32 words x
// `box_rows` rows, SWIZZLE_128B (the tensor-memory kernel's output stores).
chw_status_t make_runs_map(CUtensorMap* map, const void* ptr, int64_t total, int run_bits, int box_rows) {
  auto enc = tensor_map_encoder();
  if (!enc) return fail(CHW_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  if (total % (int64_t{box_rows} << run_bits) != 0) return fail(CHW_ERR_INVALID_ARG, "internal: output runs");
  cuuint64_t dims[2] = {cuuint64_t{1} << run_bits, static_cast<cuuint64_t>(total >> run_bits)};
  cuuint64_t strides[1] = {cuuint64_t{4} << run_bits};
  cuuint32_t box[2] = {32, static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(CHW_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
  return CHW_OK;
}

// Sequency-order stores of the tensor-memory kernel: `total` words at `ptr` viewed in 3-D as
// {2^run_bits words, run parity (2), run pair}; boxes of 32 words x 1 x 128 run pairs,
// SWIZZLE_128B (one box holds 128 runs of one parity).
chw_status_t make_seq_map(CUtensorMap* map, const void* ptr, int64_t total, int run_bits) {
  auto enc = tensor_map_encoder();
  if (!enc) return fail(CHW_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  if (total % (int64_t{256} << run_bits) != 0) return fail(CHW_ERR_INVALID_ARG, "internal: sequency runs");
  cuuint64_t dims[3] = {cuuint64_t{1} << run_bits, 2, static_cast<cuuint64_t>(total >> (run_bits + 1))};
  cuuint64_t strides[2] = {cuuint64_t{4} << run_bits, cuuint64_t{8} << run_bits};
  cuuint32_t box[3] = {32, 1, 128};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, const_cast<void*>(ptr), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(CHW_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
  return CHW_OK;
}

// The column-blocked scratch of a two-pass split as the 5-D view `colblock_view` gives: boxes
// of 256 runs of 128 bytes, with the 16-byte pieces of run rho XOR-permuted by rho mod 8,
// 4, 2 or 1 for 32-, 16-, 8- or 4-column blocks -- the layout in which the tensor-memory
// kernel stages such a first pass.  False if the driver rejects the view.
bool make_colblock_map(CUtensorMap* map, const void* ptr, int64_t total, int M, int a, int c) {
  auto enc = tensor_map_encoder();
  if (!enc || M < 13 || c < 2 || c > 5 || total % (int64_t{1} << (a + M)) != 0) return false;
  const chw::ColblockView v = chw::colblock_view(total, M, a, c);
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 5, const_cast<void*>(ptr), v.dims, v.strides, v.box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, v.swizzle, CU_TENSOR_MAP_L2_PROMOTION_NONE,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

namespace chw {
int64_t persistent_cap_override() {
  static const int64_t v = [] {
    const char* e = std::getenv("CHW_MAX_RESIDENT_UNITS");
    return e ? std::atoll(e) : int64_t{0};
  }();
  return v;
}
}  // namespace chw

struct chw_plan_s {
  int device = 0;
  int m = 0;
  int64_t batch = 0;
  chw_dtype_t dtype = CHW_F32;
  chw_norm_t norm = CHW_NORM_PER_LEVEL;
  uint32_t flags = 0;
  int tier = kTierSimple;
  int passes = 1;
  int row_bits = 0;  // two-pass: b (pass 1 rows); a = m - b
  int64_t rowstack_slots = 0;  // row-stack tier: scratch slots of 2^m words (one per CTA)
  int order = 0;               // 0 dyadic, 1 natural, 2 sequency
  int tile_bits = 0;           // fused / cluster CTA tile bits (0: the default)
  int tuned = 0;               // 0 built-in choice, 1 timed by the autotuner, 2 from its cache
  float tune_us = 0.f;         // the autotuner's time for the chosen configuration
  int64_t total = 0;
  void* workspace = nullptr;
  size_t workspace_bytes = 0;
  int* d_status = nullptr;
  // host pipeline (chw_forward_host), allocated on first use
  int64_t h_chunk = 0;  // signals per chunk
  cudaStream_t h_stream[3] = {};
  void* h_buf[3] = {};
  void* h_ws[3] = {};
  int32_t* h_exp[3][2] = {};
  int8_t* h_diag = nullptr;
  // ragged
  chw::RaggedPlan* ragged = nullptr;
  // Haar transforms: row approximations between passes (m > 13)
  uint32_t* haar_ws = nullptr;
  size_t haar_ws_bytes = 0;
  // Haar-Walsh (CHW_FLAG_HAAR_WALSH): every Haar scale of every signal as one ragged task
  // set (scales up to 2^20), and a one-signal plan per larger scale k
  chw::RaggedPlan* hw = nullptr;  // only for tiny totals that are not whole 32-word rows
  bool hw_ready = false;
  chw_plan_s* hw_big[CHW_MAX_M] = {};
  // the scale launches of one call run on branches forked from the caller's stream
  cudaStream_t hw_side[2] = {};
  cudaEvent_t hw_ev[3] = {};
  // chw_forward_haar: the Haar side output of the current call (fused tiers only), else null
  void* call_haar_z = nullptr;
};

namespace {

int fused_variant(const chw_plan_s* p, bool last_pass) {
  if (p->dtype == CHW_I32) return chw::kVarI32;
  switch (p->norm) {
    case CHW_NORM_PER_LEVEL: return chw::kVarPerLevel;
    case CHW_NORM_END: return last_pass ? chw::kVarEnd : chw::kVarPlain;
    default: return chw::kVarPlain;
  }
}

// Output mode of a final pass (fused.cuh): 0 dyadic, 2 natural, 3 sequency.  For m <= 1 the
// three orders coincide.
int final_outmode(const chw_plan_s* p) {
  if (p->m <= 1) return 0;
  return p->order == 1 ? 2 : (p->order == 2 ? 3 : 0);
}

// Checked mode (CHW_FLAG_CHECKED): the launch range-checks its indices against these bounds.
void set_checks(chw::FusedArgs* a, const chw_plan_s* p, int64_t in_total) {
  a->checked = (p->flags & CHW_FLAG_CHECKED) != 0;
  a->in_total = in_total;
}

// Device status block of a plan: int code, int (unused), int64 first offending index.
constexpr size_t kStatusBytes = 16;

chw_status_t validate_data_ptr(const void* p, const char* name) {
  if (p == nullptr) return fail(CHW_ERR_INVALID_ARG, "%s is NULL", name);
  if (reinterpret_cast<uintptr_t>(p) % 16 != 0) return fail(CHW_ERR_ALIGNMENT, "%s is not 16-byte aligned", name);
  return CHW_OK;
}

// Let a batched single-CTA launch in dyadic order write each tile with one TMA store (the
// kernel's tile-store layout) when its outputs are whole tiles and carry no D; otherwise, or
// if the driver rejects the 4-D view, the tiles go out through the SM (which applies D while
// copying).  Measured on GB300 at m = 14 x 16384 with D: the SM copy-out 4700 GB/s; a pass
// over the staged tile before the TMA store 4290; D applied to the registers before
// staging (one 4-byte load of D per 16-byte staged word) 3560.
void enable_tile_store(chw::FusedArgs* a, void* out, int64_t total, int tlo, int M, int tb, int om) {
  if (om != 0 || a->diag_out != nullptr || total % (int64_t{1} << tb) != 0) return;
  auto enc = tensor_map_encoder();
  if (!enc) return;
  const int S = chw::stage_key(tlo, M, tb, 0, om);
  cuuint64_t dims[4] = {32, 8, cuuint64_t{1} << (S - 5), static_cast<cuuint64_t>(total >> (S + 3))};
  cuuint64_t strides[3] = {cuuint64_t{4} << S, 128, cuuint64_t{4} << (S + 3)};
  cuuint32_t box[4] = {32, 8, 1u << (S - 5), 1u << (tb - S - 3)};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  if (enc(&a->tout, CU_TENSOR_MAP_DATA_TYPE_UINT32, 4, out, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
    a->tma_store = 1;
}

chw_status_t launch_tmem_units(chw_plan_s* p, int M, int om, int var, const void* in, void* out, int64_t total,
                               int64_t units, int64_t ustride, int64_t ubase, const int8_t* diag_in,
                               const int8_t* diag_out, float scale, cudaStream_t st, int colblock_a = 0,
                               int64_t diag_mask = 0, int colblock_c = 0);

// The first pass of a two-pass split takes the tensor-memory kernel for rows of 2^15 and
// 2^16 words (unless the plan asks for 2^13-word cluster tiles).
bool tmem_row_pass_tb(int tile_bits, int M, int om) { return om == 1 && (M == 15 || M == 16) && tile_bits != 13; }
bool tmem_row_pass(const chw_plan_s* p, int M, int om) { return tmem_row_pass_tb(p->tile_bits, M, om); }

// log2 of the columns per block of a tensor-memory column pass of A row bits after a first
// pass of B bits (dyadic output), or 0 when the fused / cluster column kernels run it:
// column blocks of 2^A x 32 for A = 10, 11 (2^15, 2^16 words), and narrower blocks of
// 2^(16 - A) columns for A = 12..14, which only the tensor-memory first pass can write.
int tmem_col_bits_tb(int tile_bits, int A, int B, int om) {
  if (om != 0 || A < 10 || A > 14 || tile_bits == 13) return 0;
  if (A <= 11) return 5;
  return tmem_row_pass_tb(tile_bits, B, 1) ? 16 - A : 0;
}
int tmem_col_bits(const chw_plan_s* p, int A, int B, int om) { return tmem_col_bits_tb(p->tile_bits, A, B, om); }

chw_status_t launch_row_pass(chw_plan_s* p, int M, int om, int var, const void* in, void* out, int64_t total,
                             const int8_t* diag_in, const int8_t* diag_out, int64_t diag_mask, int colblock_a,
                             float scale, cudaStream_t st, int colblock_c = 0) {
  if (tmem_row_pass(p, M, om) && diag_out == nullptr)
    return launch_tmem_units(p, M, 1, var, in, out, total, total >> M, 0, 0, diag_in, nullptr, scale, st, colblock_a,
                             diag_mask, colblock_c);
  if (colblock_c != 0 && colblock_c != 5)
    return fail(CHW_ERR_UNSUPPORTED, "internal: column blocks narrower than 32 need the tensor-memory first pass");
  const Shape s = row_shape(M, p->tile_bits);
  const bool hz = p->call_haar_z != nullptr && om == 0 && s.cb == 0;  // chw_forward_haar
  chw::FusedLaunchFn fn = hz ? chw::lookup_fused_hz(M, s.tb, var) : chw::lookup_fused(0, M, s.tb, s.cb, var, om);
  if (!fn) return fail(CHW_ERR_UNSUPPORTED, "no row kernel for M=%d tb=%d cb=%d out=%d", M, s.tb, s.cb, om);
  CUtensorMap map;
  chw_status_t r = make_rows_map(&map, in, total, s.tb);
  if (r != CHW_OK) return r;
  chw::FusedArgs a{};
  a.out = out;
  a.out_total = total;
  a.end_scale = scale;
  a.diag_in = diag_in;
  a.diag_out = diag_out;
  a.diag_mask = diag_mask;
  a.status = p->d_status;
  set_checks(&a, p, total);
  a.colblock_a = colblock_a;
  a.order_m = M;
  a.nat_b = 0;
  a.haar_z = p->call_haar_z;  // (used by whole-signal row tiles in a final order only)
  a.stall_cta = (p->flags & CHW_FLAG_TEST_STALL) != 0 ? 2 : 0;  // rank 1 withholds its signal
  a.wait_tries = (p->flags & CHW_FLAG_TEST_STALL) != 0 ? 4096u : 0u;
  if (s.cb == 0) enable_tile_store(&a, out, total, 0, M, s.tb, om);
  const int64_t unit = int64_t{1} << (s.tb + s.cb);
  const int64_t units = s.cb > 0 ? total / unit : (total + unit - 1) / unit;
  CHW_CUDA(fn(&map, a, units, st));
  return CHW_OK;
}

// Tensor-memory kernel (M = 15, 16, any order) over `units` signals of 2^M
// words: unit u at element ubase + u * ustride of `in` and `out` (ustride 0: 2^M).
chw_status_t launch_tmem_units(chw_plan_s* p, int M, int om, int var, const void* in, void* out, int64_t total,
                               int64_t units, int64_t ustride, int64_t ubase, const int8_t* diag_in,
                               const int8_t* diag_out, float scale, cudaStream_t st, int colblock_a,
                               int64_t diag_mask, int colblock_c) {
  const bool hz = p->call_haar_z != nullptr && om == 0;  // chw_forward_haar
  chw::TmemLaunchFn fn = hz ? chw::lookup_tmem_hz(M, var) : chw::lookup_tmem(M, var, om);
  if (!fn) return fail(CHW_ERR_UNSUPPORTED, "no tensor-memory kernel for m=%d out=%d", M, om);
  CUtensorMap map, omap;
  chw_status_t r = make_rows_map(&map, in, total, 14);
  if (r != CHW_OK) return r;
  bool cb_tma = false;  // the column-blocked first pass by tensor stores
  if (om == 2) {
    r = make_runs_map(&omap, out, total, M - 6, 64);
  } else if (om == 3) {
    r = make_seq_map(&omap, out, total, M - 8);
  } else if (om == 1) {
    r = CHW_OK;
    cb_tma = make_colblock_map(&omap, out, total, M, colblock_a, colblock_c != 0 ? colblock_c : 5);
  } else {
    r = make_runs_map(&omap, out, total, M - 8, 256);
  }
  if (r != CHW_OK) return r;
  chw::FusedArgs a{};
  a.out = out;
  a.out_total = total;
  a.end_scale = scale;
  a.diag_in = diag_in;
  a.diag_out = diag_out;
  a.diag_mask = diag_mask != 0 ? diag_mask : (int64_t{1} << M) - 1;
  a.status = p->d_status;
  set_checks(&a, p, total);
  a.unit_stride = ustride;
  a.unit_base = ubase;
  a.colblock_a = colblock_a;
  a.colblock_c = colblock_c;
  a.tma_store = cb_tma ? 1 : 0;
  a.haar_z = p->call_haar_z;  // (used by whole signals in a final order only)
  CHW_CUDA(fn(&map, &omap, a, units, st));
  return CHW_OK;
}

// Second pass of a two-pass split on the tensor-memory kernel: column blocks of 2^A rows x
// 2^clo columns (2^(A+clo) words each, back to back in `in`), output rows contiguous.
chw_status_t launch_tmem_col_pass(chw_plan_s* p, int A, int clo, int var, const void* in, void* out, int64_t total,
                                  const int8_t* diag_out, int64_t diag_mask, float scale, cudaStream_t st) {
  const int M = A + clo;
  chw::TmemLaunchFn fn = chw::lookup_tmem_col(M, clo, var);
  if (!fn) return fail(CHW_ERR_UNSUPPORTED, "no tensor-memory column kernel for A=%d", A);
  CUtensorMap map, omap;
  chw_status_t r = make_rows_map(&map, in, total, 14);
  if (r != CHW_OK) return r;
  r = make_runs_map(&omap, out, total, M - 8, 256);
  if (r != CHW_OK) return r;
  chw::FusedArgs a{};
  a.out = out;
  a.out_total = total;
  a.end_scale = scale;
  a.diag_out = diag_out;
  a.diag_mask = diag_mask;
  a.status = p->d_status;
  set_checks(&a, p, total);
  CHW_CUDA(fn(&map, &omap, a, total >> M, st));
  return CHW_OK;
}

// Exchange scratch of the tensor-memory tier over SM pairs (m = 17).
size_t cross_scratch_bytes(int device) { return static_cast<size_t>(chw::tmem_cross_clusters(device)) << 17; }

// Tensor-memory tier over a cluster (m = 17: two SMs per signal, each holding half of it);
// `ws` holds at least cross_scratch_bytes().
chw_status_t launch_tmem_cross(chw_plan_s* p, const void* in, void* out, int64_t total, const int8_t* diag_in,
                               const int8_t* diag_out, void* ws, cudaStream_t st) {
  const int M = p->m;
  chw::TmemLaunchFn fn = chw::lookup_tmem_cross(M, fused_variant(p, true));
  if (!fn) return fail(CHW_ERR_UNSUPPORTED, "no cross-SM tensor-memory kernel for m=%d", M);
  CUtensorMap map, omap;
  chw_status_t r = make_rows_map(&map, in, total, 14);
  if (r != CHW_OK) return r;
  r = make_runs_map(&omap, out, total, M - 8, 256);
  if (r != CHW_OK) return r;
  chw::FusedArgs a{};
  a.out = out;
  a.out_total = total;
  a.end_scale = end_scale_f32(M);
  a.diag_in = diag_in;
  a.diag_out = diag_out;
  a.diag_mask = (int64_t{1} << M) - 1;
  a.status = p->d_status;
  set_checks(&a, p, total);
  if (ws == nullptr) return fail(CHW_ERR_INVALID_ARG, "internal: no exchange scratch");
  a.xscratch = static_cast<uint4*>(ws);
  a.xclusters = static_cast<int64_t>(cross_scratch_bytes(p->device) >> 17);
  CHW_CUDA(fn(&map, &omap, a, total >> M, st));
  return CHW_OK;
}

// Tensor-memory tier: the plan's batch, one signal per SM at a time.
chw_status_t launch_tmem_pass(chw_plan_s* p, const void* in, void* out, int64_t total, const int8_t* diag_in,
                              const int8_t* diag_out, cudaStream_t st) {
  return launch_tmem_units(p, p->m, final_outmode(p), fused_variant(p, true), in, out, total, total >> p->m, 0, 0,
                           diag_in, diag_out, end_scale_f32(p->m), st);
}

chw_status_t launch_col_pass(chw_plan_s* p, int A, int var, int om, const void* in, void* out, int64_t total,
                             const int8_t* diag_out, int64_t diag_mask, float scale, cudaStream_t st) {
  const Shape s = om == 2 ? Shape{A <= 8 ? 13 : 14, 0} : col_shape(A, p->tile_bits);
  chw::FusedLaunchFn fn = chw::lookup_fused(5, A, s.tb, s.cb, var, om);
  if (!fn) return fail(CHW_ERR_UNSUPPORTED, "no column kernel for A=%d", A);
  CUtensorMap map;
  chw_status_t r = make_rows_map(&map, in, total, s.tb);
  if (r != CHW_OK) return r;
  chw::FusedArgs a{};
  a.out = out;
  a.out_total = total;
  a.end_scale = scale;
  a.diag_in = nullptr;
  a.diag_out = diag_out;
  a.diag_mask = diag_mask;
  a.status = p->d_status;
  set_checks(&a, p, total);
  a.colblock_a = 0;
  a.order_m = p->m;
  a.nat_b = p->m - A;
  if (s.cb == 0) enable_tile_store(&a, out, total, 5, A, s.tb, om);
  const int64_t unit = int64_t{1} << (s.tb + s.cb);
  const int64_t units = s.cb > 0 ? total / unit : (total + unit - 1) / unit;
  CHW_CUDA(fn(&map, a, units, st));
  return CHW_OK;
}

// `batch` signals of 2^m 2-byte codes viewed as rows of 64 codes (128 B), SWIZZLE_128B.
chw_status_t make_codes_map(CUtensorMap* map, const void* ptr, int64_t batch, int m) {
  auto enc = tensor_map_encoder();
  if (!enc) return fail(CHW_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  cuuint64_t dims[2] = {64, static_cast<cuuint64_t>((batch << m) / 64)};
  cuuint64_t strides[1] = {128};
  cuuint32_t box[2] = {64, static_cast<cuuint32_t>(1 << (m - 6))};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(CHW_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
  return CHW_OK;
}

chw_status_t launch_lowp_fused(chw_plan_s* p, const void* x, void* y, int64_t batch, const int32_t* exp_in,
                               int32_t* exp_out, const int8_t* diag_in, const int8_t* diag_out, cudaStream_t st) {
  chw::LowpLaunchFn fn = chw::lookup_lowp(p->m, p->dtype == CHW_F16, p->norm == CHW_NORM_END);
  if (!fn) return fail(CHW_ERR_UNSUPPORTED, "no fused 16-bit kernel for m=%d", p->m);
  CUtensorMap map, omap;
  chw_status_t r = make_codes_map(&map, x, batch, p->m);
  if (r != CHW_OK) return r;
  r = make_codes_map(&omap, y, batch, p->m);  // the one-warp kernel's output stores
  if (r != CHW_OK) return r;
  chw::LowpArgs a{};
  a.out = y;
  a.exp_in = exp_in;
  a.exp_out = exp_out;
  a.end_scale = end_scale_f32(p->m);
  a.diag_in = diag_in;
  a.diag_out = diag_out;
  a.status = p->d_status;  // (the 16-bit kernel indexes by signal number only: no checks)
  CHW_CUDA(fn(&map, &omap, a, batch, st));
  return CHW_OK;
}

// Row-stack tier: one CTA per signal, rows through an L2-resident scratch slot per CTA.
chw_status_t launch_rowstack(chw_plan_s* p, const void* x, void* y, int64_t batch, const int8_t* diag_in,
                             const int8_t* diag_out, void* ws, int64_t slots, cudaStream_t st) {
  chw::RowstackLaunchFn fn = chw::lookup_rowstack(p->m, fused_variant(p, true));
  if (!fn) return fail(CHW_ERR_UNSUPPORTED, "no row-stack kernel for m=%d", p->m);
  CUtensorMap map;
  const int64_t total = batch << p->m;
  chw_status_t r = make_rows_map(&map, x, total, 14);
  if (r != CHW_OK) return r;
  chw::FusedArgs a{};
  a.out = y;
  a.out_total = total;
  a.end_scale = end_scale_f32(p->m);
  a.diag_in = diag_in;
  a.diag_out = diag_out;
  a.diag_mask = (int64_t{1} << p->m) - 1;
  a.status = p->d_status;
  set_checks(&a, p, total);
  const int64_t grid = batch < slots ? batch : slots;
  CHW_CUDA(fn(&map, a, static_cast<uint32_t*>(ws), grid, batch, st));
  return CHW_OK;
}

chw_status_t launch_simple(chw_plan_s* p, const void* x, void* y, int64_t batch, const int32_t* exp_in,
                           int32_t* exp_out, const int8_t* diag_in, const int8_t* diag_out, cudaStream_t st) {
  chw::SimpleArgs a{};
  a.x = x;
  a.y = y;
  a.m = p->m;
  a.batch = batch;
  a.norm = static_cast<int>(p->norm);
  a.end_scale = end_scale_f32(p->m);
  a.exp_in = exp_in;
  a.exp_out = exp_out;
  a.diag_in = diag_in;
  a.diag_out = diag_out;
  a.order = p->order;
  const int64_t n = int64_t{1} << p->m;
  const int threads = n >= 512 ? 256 : (n >= 64 ? static_cast<int>(n / 2) : 32);
  const size_t smem = static_cast<size_t>(n) * 4;
  const dim3 grid(static_cast<unsigned>(batch));
  switch (p->dtype) {
    case CHW_I32: chw::simple_kernel<chw::kSimpleI32><<<grid, threads, smem, st>>>(a); break;
    case CHW_F32: chw::simple_kernel<chw::kSimpleF32><<<grid, threads, smem, st>>>(a); break;
    case CHW_BF16: chw::simple_kernel<chw::kSimpleBF16><<<grid, threads, smem, st>>>(a); break;
    case CHW_F16: chw::simple_kernel<chw::kSimpleF16><<<grid, threads, smem, st>>>(a); break;
  }
  CHW_CUDA(cudaGetLastError());
  return CHW_OK;
}

// y = D_out H x D_in for `batch` signals (x, y device; ws = scratch for the two-pass tier)
chw_status_t run_transform(chw_plan_s* p, const void* x, void* y, int64_t batch, const int32_t* exp_in,
                           int32_t* exp_out, const int8_t* diag_in, const int8_t* diag_out, void* ws,
                           cudaStream_t st) {
  const int m = p->m;
  const int64_t n = int64_t{1} << m;
  const int64_t total = batch * n;
  const int64_t dmask = n - 1;
  switch (p->tier) {
    case kTierSimple:
      return launch_simple(p, x, y, batch, exp_in, exp_out, diag_in, diag_out, st);
    case kTierLowp:
      return launch_lowp_fused(p, x, y, batch, exp_in, exp_out, diag_in, diag_out, st);
    case kTierRowStack:
      return launch_rowstack(p, x, y, batch, diag_in, diag_out, ws, p->rowstack_slots, st);
    case kTierTmem:
      return launch_tmem_pass(p, x, y, total, diag_in, diag_out, st);
    case kTierTmemCross:
      return launch_tmem_cross(p, x, y, total, diag_in, diag_out, ws, st);
    case kTierFused:
    case kTierCluster:
      return launch_row_pass(p, m, final_outmode(p), fused_variant(p, true), x, y, total, diag_in, diag_out, dmask,
                             0, end_scale_f32(m), st);
    case kTierTwoPass: {
      const int b = p->row_bits, a = m - b;
      const int om2 = final_outmode(p);
      const int clo = tmem_col_bits(p, a, b, om2);
      chw_status_t r = launch_row_pass(p, b, om2 == 2 ? 4 : 1, fused_variant(p, false), x, ws, total, diag_in,
                                       nullptr, dmask, a, 1.0f, st, clo);
      if (r != CHW_OK) return r;
      if (clo != 0)
        return launch_tmem_col_pass(p, a, clo, fused_variant(p, true), ws, y, total, diag_out, dmask,
                                    end_scale_f32(m), st);
      return launch_col_pass(p, a, fused_variant(p, true), om2, ws, y, total, diag_out, dmask, end_scale_f32(m), st);
    }
    default:
      return fail(CHW_ERR_INVALID_ARG, "plan is not a batched plan");
  }
}

chw_status_t check_plan_args(int m, int64_t batch, chw_dtype_t dtype, chw_norm_t norm) {
  if (m < 0 || m > CHW_MAX_M) return fail(CHW_ERR_INVALID_ARG, "m=%d outside 0..%d", m, CHW_MAX_M);
  if (batch < 1) return fail(CHW_ERR_INVALID_ARG, "batch=%lld must be >= 1", static_cast<long long>(batch));
  if (dtype < CHW_I32 || dtype > CHW_F16) return fail(CHW_ERR_INVALID_ARG, "unknown dtype %d", static_cast<int>(dtype));
  if (norm < CHW_NORM_NONE || norm > CHW_NORM_END) return fail(CHW_ERR_INVALID_ARG, "unknown norm %d", static_cast<int>(norm));
  if (dtype == CHW_I32 && norm != CHW_NORM_NONE) return fail(CHW_ERR_INVALID_ARG, "int32 is unnormalised only (CHW_NORM_NONE)");
  if (is_lowp(dtype) && norm == CHW_NORM_NONE)
    return fail(CHW_ERR_INVALID_ARG, "bf16/fp16 take CHW_NORM_END or CHW_NORM_PER_LEVEL");
  const int64_t n = int64_t{1} << m;
  if (batch > (int64_t{1} << 40) / n) return fail(CHW_ERR_INVALID_ARG, "batch * 2^m exceeds 2^40 elements");
  return CHW_OK;
}

// The Haar-Walsh transform of eq. (4): for every signal, z[0] (H = 1) and the Haar scale
// k = 0..m-1 at [2^k, 2^{k+1}) (H_k).  The scales below 2^14 together fill the signal's
// first 2^min(m,14) positions and run in one single-CTA "head" launch (output mode 6);
// scales k = 14..17 run as batched launches over strided units (one unit per signal,
// 2^m apart, at offset 2^k; k = 15, 16 on the tensor-memory kernel, 14 and 17 on the
// fused and cluster kernels); each scale k >= 18 gets a one-signal two-pass plan.  Totals
// that are not whole 32-word rows (m < 5) take a ragged task set over the same offsets.
chw_status_t build_haar_walsh(chw_plan_s* p) {
  if (is_lowp(p->dtype)) return fail(CHW_ERR_UNSUPPORTED, "Haar-Walsh takes int32 or fp32");
  if (p->m > 29) return fail(CHW_ERR_UNSUPPORTED, "Haar-Walsh takes m <= 29");
  const int m = p->m;
  if (p->total % 32 == 0) {
    for (int k = 18; k < m; ++k) {
      chw_status_t r = chw_plan(&p->hw_big[k], k, 1, p->dtype, p->norm, 0);
      if (r != CHW_OK) return r;
    }
    for (int i = 0; i < 2; ++i)
      if (cudaStreamCreateWithFlags(&p->hw_side[i], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return fail(CHW_ERR_CUDA, "Haar-Walsh branch streams");
      }
    for (int i = 0; i < 3; ++i)
      if (cudaEventCreateWithFlags(&p->hw_ev[i], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return fail(CHW_ERR_CUDA, "Haar-Walsh branch events");
      }
    p->hw_ready = true;
    return CHW_OK;
  }
  const int kr = m - 1 < chw::kRaggedMaxM ? m - 1 : chw::kRaggedMaxM;
  std::vector<uint8_t> ms;
  std::vector<int64_t> off;
  ms.reserve(static_cast<size_t>(p->batch) * (kr + 2));
  off.reserve(ms.capacity());
  for (int64_t s = 0; s < p->batch; ++s) {
    const int64_t base = s << m;
    ms.push_back(0);
    off.push_back(base);
    for (int k = 0; k <= kr; ++k) {
      ms.push_back(static_cast<uint8_t>(k));
      off.push_back(base + (int64_t{1} << k));
    }
  }
  std::string why;
  p->hw = chw::ragged_create_at(ms.data(), off.data(), static_cast<int64_t>(ms.size()), p->total,
                                p->dtype == CHW_I32 ? chw::kVarI32 : fused_variant(p, true), p->d_status, false,
                                &why, (p->flags & CHW_FLAG_CHECKED) != 0);
  if (p->hw == nullptr) return fail(CHW_ERR_CUDA, "Haar-Walsh task set: %s", why.c_str());
  for (int k = chw::kRaggedMaxM + 1; k < m; ++k) {
    chw_status_t r = chw_plan(&p->hw_big[k], k, 1, p->dtype, p->norm, 0);
    if (r != CHW_OK) return r;
  }
  return CHW_OK;
}

// One launch of fused row tiles over `units` units of 2^(tb+cb) elements, unit u at
// ubase + u * ustride (ustride 0: back to back), in and out both `total` words long.
chw_status_t launch_units(chw_plan_s* p, int M, int om, int var, const void* in, void* out, int64_t total,
                          int64_t units, int64_t ustride, int64_t ubase, float scale, int head_end,
                          cudaStream_t st) {
  const Shape s = row_shape(M);
  chw::FusedLaunchFn fn = chw::lookup_fused(0, M, s.tb, s.cb, var, om);
  if (!fn) return fail(CHW_ERR_UNSUPPORTED, "no row kernel for M=%d tb=%d cb=%d out=%d", M, s.tb, s.cb, om);
  CUtensorMap map;
  chw_status_t r = make_rows_map(&map, in, total, s.tb);
  if (r != CHW_OK) return r;
  chw::FusedArgs a{};
  a.out = out;
  a.out_total = total;
  a.end_scale = scale;
  a.diag_mask = (int64_t{1} << p->m) - 1;
  a.status = p->d_status;
  set_checks(&a, p, total);
  a.order_m = M;
  a.head_end = head_end;
  a.unit_stride = ustride;
  a.unit_base = ubase;
  CHW_CUDA(fn(&map, a, units, st));
  return CHW_OK;
}

// y = H_m Psi_m^T z (eq. (4)) with the launches described at build_haar_walsh.
chw_status_t run_haar_walsh(chw_plan_s* p, const void* z, void* y, cudaStream_t st) {
  const int m = p->m;
  const int64_t total = p->total, n = int64_t{1} << m;
  // the head's butterflies are unscaled for END (each scale is scaled once on output)
  const int vh = p->dtype == CHW_I32 ? chw::kVarI32 : (p->norm == CHW_NORM_PER_LEVEL ? chw::kVarPerLevel : chw::kVarPlain);
  const int head_end = p->dtype == CHW_F32 && p->norm == CHW_NORM_END;
  chw_status_t r;
  if (m <= 14) {
    const Shape s = row_shape(m);
    const int64_t tile = int64_t{1} << s.tb;
    return launch_units(p, m, 6, vh, z, y, total, (total + tile - 1) / tile, 0, 0, 1.0f, head_end, st);
  }
  // The head and the scales 2^14..2^17 read and write disjoint parts of every signal, so
  // they run as parallel branches (the caller's stream and two forked streams, joined
  // again before the call returns its work to the caller's stream): one launch's ramp-down
  // leaves SMs to the others.
  CHW_CUDA(cudaEventRecord(p->hw_ev[0], st));
  for (cudaStream_t h : p->hw_side) CHW_CUDA(cudaStreamWaitEvent(h, p->hw_ev[0], 0));
  r = launch_units(p, 14, 6, vh, z, y, total, p->batch, n, 0, 1.0f, head_end, p->hw_side[0]);
  for (int k = 14; k < m && k <= 17 && r == CHW_OK; ++k) {
    cudaStream_t bs = k == 14 ? p->hw_side[1] : (k == 15 ? p->hw_side[0] : st);
    if (k == 15 || k == 16) {
      r = launch_tmem_units(p, k, 0, fused_variant(p, true), z, y, total, p->batch, n, int64_t{1} << k, nullptr,
                            nullptr, end_scale_f32(k), bs);
    } else {
      r = launch_units(p, k, 0, fused_variant(p, true), z, y, total, p->batch, n, int64_t{1} << k, end_scale_f32(k),
                       0, bs);
    }
  }
  for (int i = 0; i < 2; ++i) {  // join the branches (also after a failed launch)
    CHW_CUDA(cudaEventRecord(p->hw_ev[1 + i], p->hw_side[i]));
    CHW_CUDA(cudaStreamWaitEvent(st, p->hw_ev[1 + i], 0));
  }
  if (r != CHW_OK) return r;
  for (int k = 18; k < m; ++k) {
    chw_plan_s* b = p->hw_big[k];
    for (int64_t s = 0; s < p->batch; ++s) {
      const int64_t o = (s << m) + (int64_t{1} << k);
      r = run_transform(b, static_cast<const uint32_t*>(z) + o, static_cast<uint32_t*>(y) + o, 1, nullptr, nullptr,
                        nullptr, nullptr, b->workspace, st);
      if (r != CHW_OK) return r;
    }
  }
  return CHW_OK;
}

// Read and clear a device status word (after a device synchronisation).
chw_status_t take_status(int* d_status, int* out, int64_t* index = nullptr) {
  int32_t block[4] = {};
  CHW_CUDA(cudaMemcpy(block, d_status, kStatusBytes, cudaMemcpyDeviceToHost));
  CHW_CUDA(cudaMemset(d_status, 0, kStatusBytes));
  *out = block[0];
  if (index != nullptr) std::memcpy(index, block + 2, sizeof(int64_t));
  return CHW_OK;
}

// Two device ranges of `bytes` each overlap.
bool overlaps(const void* a, const void* b, size_t bytes) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + bytes && y < x + bytes;
}

chw_status_t check_haar_call(chw_plan_s* p, const void* in, const void* out, const char* in_name,
                             const char* out_name) {
  if (p == nullptr) return fail(CHW_ERR_INVALID_ARG, "plan is NULL");
  if (p->ragged) return fail(CHW_ERR_INVALID_ARG, "Haar transforms take a batched plan, not a ragged one");
  if (is_lowp(p->dtype)) return fail(CHW_ERR_UNSUPPORTED, "Haar transforms take int32 or fp32");
  chw_status_t r = validate_data_ptr(in, in_name);
  if (r != CHW_OK) return r;
  return validate_data_ptr(out, out_name);
}

void destroy_host_pipeline(chw_plan_s* p) {
  for (int i = 0; i < 3; ++i) {
    if (p->h_stream[i]) cudaStreamDestroy(p->h_stream[i]);
    if (p->h_buf[i]) cudaFree(p->h_buf[i]);
    if (p->h_ws[i]) cudaFree(p->h_ws[i]);
    for (int j = 0; j < 2; ++j)
      if (p->h_exp[i][j]) cudaFree(p->h_exp[i][j]);
    p->h_stream[i] = nullptr;
    p->h_buf[i] = p->h_ws[i] = nullptr;
    p->h_exp[i][0] = p->h_exp[i][1] = nullptr;
  }
  if (p->h_diag) cudaFree(p->h_diag);
  p->h_diag = nullptr;
  p->h_chunk = 0;
}

// ---------------------------------------------------------------- autotuner
// The configurations a plan of this shape can run, every one of them compiled: for m = 14
// the 2^14-word tile or a 2-CTA cluster of 2^13-word tiles; for m = 17 the 8-CTA cluster;
// for m >= 17 every two-pass split
// y = H_b X^T H_a with a = 6..12 (b = m - a in 5..17) and either tile size.  Empty when the
// plan has a single configuration (m <= 13, 16-bit storage, or a flag that fixes the tier).
std::vector<chw::TuneChoice> tune_candidates(int m, chw_dtype_t dtype, chw_norm_t norm, uint32_t flags) {
  std::vector<chw::TuneChoice> c;
  const uint32_t fixed = CHW_FLAG_FORCE_SIMPLE | CHW_FLAG_FORCE_MULTIPASS | CHW_FLAG_ROWSTACK | CHW_FLAG_CLUSTER |
                         CHW_FLAG_TEST_STALL;
  if (is_lowp(dtype) || (flags & fixed) != 0 || m < 14 || m > CHW_MAX_M) return c;
  const int order = (flags & CHW_FLAG_ORDER_NATURAL) != 0 ? 1 : ((flags & CHW_FLAG_ORDER_SEQUENCY) != 0 ? 2 : 0);
  const int om = m <= 1 ? 0 : (order == 1 ? 2 : (order == 2 ? 3 : 0));
  int var_last, var_first;
  if (dtype == CHW_I32) {
    var_last = var_first = chw::kVarI32;
  } else if (norm == CHW_NORM_PER_LEVEL) {
    var_last = var_first = chw::kVarPerLevel;
  } else {
    var_first = chw::kVarPlain;
    var_last = norm == CHW_NORM_END ? chw::kVarEnd : chw::kVarPlain;
  }
  auto add = [&](int tier, int row_bits, int tile_bits) {
    for (const auto& x : c)
      if (x.tier == tier && x.row_bits == row_bits && x.tile_bits == tile_bits) return;
    c.push_back(chw::TuneChoice{tier, row_bits, tile_bits});
  };
  if (m <= 17) {
    if (m <= 16 && chw::lookup_tmem(m, var_last, om) != nullptr) add(kTierTmem, m, 0);
    if (m == 17 && om == 0 && chw::lookup_tmem_cross(m, var_last) != nullptr) add(kTierTmemCross, m, 0);
    // m = 15, 16: one SM holds the whole signal in tensor memory (92 % against 52-62 % for
    // the 2- and 4-CTA clusters and 41 % for the row-stack tier), so only the tensor-memory
    // kernel is timed; the others stay selectable by their flags
    for (int tb : {14, 13}) {
      if (m == 15 || m == 16) break;
      const Shape sh = row_shape(m, tb);
      if (sh.tb != tb && m != 17) continue;  // the tile preference does not apply
      if (chw::lookup_fused(0, m, sh.tb, sh.cb, var_last, om) != nullptr)
        add(sh.cb > 0 ? kTierCluster : kTierFused, m, sh.tb);
    }
  }
  if (m >= 17) {
    for (int a = 6; a <= 14; ++a) {
      const int b = m - a;
      if (b < 5 || b > 17) continue;
      for (int tb : {14, 13}) {
        const Shape s1 = row_shape(b, tb);
        const Shape s2 = om == 2 ? Shape{a <= 8 ? 13 : 14, 0} : col_shape(a, tb);
        const int om1 = om == 2 ? 4 : 1;
        const int clo = tmem_col_bits_tb(tb, a, b, om);
        const bool row_ok = tmem_row_pass_tb(tb, b, om1) ? chw::lookup_tmem(b, var_first, 1) != nullptr
                                                        : chw::lookup_fused(0, b, s1.tb, s1.cb, var_first, om1) != nullptr;
        const bool col_ok = clo != 0 ? chw::lookup_tmem_col(a + clo, clo, var_last) != nullptr
                                     : chw::lookup_fused(5, a, s2.tb, s2.cb, var_last, om) != nullptr;
        if (!row_ok || !col_ok) continue;
        const bool same = row_shape(b, 13).tb == row_shape(b, 14).tb && row_shape(b, 13).cb == row_shape(b, 14).cb &&
                          (om == 2 || (col_shape(a, 13).tb == col_shape(a, 14).tb && col_shape(a, 13).cb == col_shape(a, 14).cb));
        add(kTierTwoPass, b, same ? 14 : tb);
      }
    }
  }
  if (c.size() <= 1) c.clear();
  return c;
}

void apply_choice(chw_plan_s* p, const chw::TuneChoice& c) {
  p->tier = c.tier;
  p->row_bits = c.row_bits;
  p->tile_bits = c.tile_bits;
  p->passes = c.tier == kTierTwoPass ? 2 : 1;
}

bool autotune_requested(uint32_t flags) {
  if ((flags & CHW_FLAG_AUTOTUNE) != 0) return true;
  const char* e = std::getenv("CHW_AUTOTUNE");
  return e != nullptr && std::atoi(e) != 0;
}

// The cache file named by CHW_TUNE_CACHE, read once per process.
const char* tune_cache_path() {
  static std::once_flag once;
  static std::string path;
  std::call_once(once, [] {
    const char* e = std::getenv("CHW_TUNE_CACHE");
    if (e != nullptr && *e != 0) {
      path = e;
      chw::tune_cache_load(path.c_str());
    }
  });
  return path.empty() ? nullptr : path.c_str();
}

// Pick the plan's configuration by timing every candidate (CUDA events, default stream) on
// synthetic signals of the plan's shape: min(batch, 2^26 / 2^m) signals (at least one), so
// that a candidate's run covers more than the L2; two warm-up runs, then the mean of five.
// A cached choice for the same key is used instead of timing (if it is still a candidate).
chw_status_t autotune_plan(chw_plan_s* p) {
  const std::vector<chw::TuneChoice> cands = tune_candidates(p->m, p->dtype, p->norm, p->flags);
  if (cands.empty()) return CHW_OK;
  cudaDeviceProp prop{};
  CHW_CUDA(cudaGetDeviceProperties(&prop, p->device));
  const std::string key = chw::tune_key(prop.name, p->m, p->batch, p->dtype, p->norm, p->order);
  const char* path = tune_cache_path();
  chw::TuneChoice hit{};
  float hit_us = 0.f;
  if (chw::tune_cache_get(key, &hit, &hit_us)) {
    for (const auto& c : cands)
      if (c.tier == hit.tier && c.row_bits == hit.row_bits && c.tile_bits == hit.tile_bits) {
        apply_choice(p, c);
        p->tuned = 2;
        p->tune_us = hit_us;
        return CHW_OK;
      }
  }
  const int64_t n = int64_t{1} << p->m;
  int64_t tbatch = (int64_t{1} << 26) / n;
  if (tbatch < 1) tbatch = 1;
  if (tbatch > p->batch) tbatch = p->batch;
  const int64_t total = tbatch * n;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
  const int64_t slots = std::min<int64_t>(sms > 0 ? sms : 1, tbatch);
  const size_t bytes = static_cast<size_t>(total) * 4;
  const size_t ws_bytes = std::max({bytes, static_cast<size_t>(slots * n) * 4, cross_scratch_bytes(p->device)});
  void *x = nullptr, *y = nullptr, *ws = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto release = [&] {
    if (x) cudaFree(x);
    if (y) cudaFree(y);
    if (ws) cudaFree(ws);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (cudaMalloc(&x, bytes) != cudaSuccess || cudaMalloc(&y, bytes) != cudaSuccess ||
      cudaMalloc(&ws, ws_bytes) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    release();
    cudaGetLastError();
    return fail(CHW_ERR_OOM, "autotuner buffers of %zu bytes", 2 * bytes + ws_bytes);
  }
  cudaMemset(x, 0x3c, bytes);  // every word 0x3c3c3c3c: a normal fp32 (0.0115) or int32
  int best = -1;
  float best_ms = 0.f;
  for (size_t i = 0; i < cands.size(); ++i) {
    chw_plan_s t{};
    t.device = p->device;
    t.m = p->m;
    t.batch = tbatch;
    t.dtype = p->dtype;
    t.norm = p->norm;
    t.flags = p->flags;
    t.order = p->order;
    t.total = total;
    t.d_status = p->d_status;
    t.rowstack_slots = slots;
    apply_choice(&t, cands[i]);
    bool ok = true;
    for (int w = 0; w < 2 && ok; ++w)
      ok = run_transform(&t, x, y, tbatch, nullptr, nullptr, nullptr, nullptr, ws, nullptr) == CHW_OK;
    if (ok) {
      cudaEventRecord(e0, nullptr);
      for (int r = 0; r < 5 && ok; ++r)
        ok = run_transform(&t, x, y, tbatch, nullptr, nullptr, nullptr, nullptr, ws, nullptr) == CHW_OK;
      cudaEventRecord(e1, nullptr);
    }
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      release();
      return fail(CHW_ERR_CUDA, "autotuner: %s", cudaGetErrorString(cudaGetLastError()));
    }
    float ms = 0.f;
    int st = 0;
    cudaMemcpy(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    cudaMemset(p->d_status, 0, kStatusBytes);
    if (!ok || st != 0 || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      cudaGetLastError();
      continue;  // a candidate that fails is not chosen
    }
    ms /= 5.f;
    if (best < 0 || ms < best_ms) {
      best = static_cast<int>(i);
      best_ms = ms;
    }
  }
  release();
  g_err.clear();
  if (best < 0) return fail(CHW_ERR_CUDA, "autotuner: no candidate ran");
  apply_choice(p, cands[best]);
  p->tuned = 1;
  p->tune_us = best_ms * 1000.f;
  chw::tune_cache_put(key, cands[best], p->tune_us);
  if (path != nullptr) chw::tune_cache_save(path);
  return CHW_OK;
}

}  // namespace

namespace chw {

// Internal, for chw_forward_noalloc: the launches chw_forward makes for a two-pass plan of
// this shape (the same split and kernels), with the pass-1 intermediate in caller-given
// device memory `scratch` (batch * 2^m words) and device errors latched into `status`.
// Allocates nothing: the plan descriptor lives on the host stack and only carries
// arguments.
chw_status_t two_pass_into(int m, int64_t batch, chw_dtype_t dtype, chw_norm_t norm, const void* x, void* y,
                           void* scratch, int* status, cudaStream_t st) {
  chw_plan_s t{};
  CHW_CUDA(cudaGetDevice(&t.device));
  t.m = m;
  t.batch = batch;
  t.dtype = dtype;
  t.norm = norm;
  t.total = batch << m;
  t.tier = kTierTwoPass;
  t.passes = 2;
  t.row_bits = m - two_pass_col_bits(m);
  t.d_status = status;
  return run_transform(&t, x, y, batch, nullptr, nullptr, nullptr, nullptr, scratch, st);
}

// Internal: the reason chw_last_error_message() reports on this host thread.
chw_status_t set_error(chw_status_t s, const char* msg) { return fail(s, "%s", msg); }
void clear_error() { g_err.clear(); }

}  // namespace chw

extern "C" {

const char* chw_status_string(chw_status_t s) {
  switch (s) {
    case CHW_OK: return "CHW_OK";
    case CHW_ERR_INVALID_ARG: return "CHW_ERR_INVALID_ARG: invalid argument";
    case CHW_ERR_UNSUPPORTED: return "CHW_ERR_UNSUPPORTED: not implemented for these arguments";
    case CHW_ERR_ALIGNMENT: return "CHW_ERR_ALIGNMENT: pointer not 16-byte aligned";
    case CHW_ERR_OOM: return "CHW_ERR_OOM: device allocation failed";
    case CHW_ERR_CUDA: return "CHW_ERR_CUDA: CUDA runtime error";
    case CHW_ERR_TIMEOUT: return "CHW_ERR_TIMEOUT: a bounded device wait gave up";
    case CHW_ERR_DEVICE_CHECK: return "CHW_ERR_DEVICE_CHECK: device-side check failed";
  }
  return "unknown chw_status_t";
}

const char* chw_last_error_message(void) { return g_err.c_str(); }

chw_status_t chw_plan(chw_plan_t* out, int m, int64_t batch, chw_dtype_t dtype, chw_norm_t norm, uint32_t flags) {
  g_err.clear();
  if (out == nullptr) return fail(CHW_ERR_INVALID_ARG, "plan output pointer is NULL");
  *out = nullptr;
  chw_status_t r = check_plan_args(m, batch, dtype, norm);
  if (r != CHW_OK) return r;

  if ((flags & CHW_FLAG_TEST_CORRUPT) != 0) return fail(CHW_ERR_INVALID_ARG, "CHW_FLAG_TEST_CORRUPT is for ragged plans");
  auto* p = new chw_plan_s();
  p->m = m;
  p->batch = batch;
  p->dtype = dtype;
  p->norm = norm;
  p->flags = flags;
  p->total = batch * (int64_t{1} << m);
  p->row_bits = m;
  const bool nat = (flags & CHW_FLAG_ORDER_NATURAL) != 0, seq = (flags & CHW_FLAG_ORDER_SEQUENCY) != 0;
  if (nat && seq) {
    delete p;
    return fail(CHW_ERR_INVALID_ARG, "CHW_FLAG_ORDER_NATURAL and CHW_FLAG_ORDER_SEQUENCY exclude each other");
  }
  p->order = nat ? 1 : (seq ? 2 : 0);
  if (p->order != 0 && (flags & CHW_FLAG_ROWSTACK) != 0) {
    delete p;
    return fail(CHW_ERR_UNSUPPORTED, "ordered outputs are not available with CHW_FLAG_ROWSTACK");
  }

  if (p->order != 0 && is_lowp(dtype)) {
    if (m > 13) {
      delete p;
      return fail(CHW_ERR_UNSUPPORTED, "bf16/fp16 storage needs m <= 13 (one CTA per signal)");
    }
    p->tier = kTierSimple;  // the simple kernel stores any order
  } else if (nat && m >= 15 && m <= 16 && (flags & (CHW_FLAG_FORCE_SIMPLE | CHW_FLAG_FORCE_MULTIPASS |
                                                      CHW_FLAG_CLUSTER | CHW_FLAG_TEST_STALL)) == 0) {
    p->tier = kTierTmem;  // natural order from the tensor-memory kernel's staging
  } else if (nat && m >= 15 && (flags & CHW_FLAG_FORCE_SIMPLE) == 0) {
    // natural order: single-CTA rows, then columns written as stride-2^b runs
    if (m > 23) {
      delete p;
      return fail(CHW_ERR_UNSUPPORTED, "natural order takes m <= 23");
    }
    p->tier = kTierTwoPass;
    p->passes = 2;
    p->row_bits = m - (m >= 18 ? 9 : 6);
  } else if (is_lowp(dtype)) {
    if (m > 13) {
      delete p;
      return fail(CHW_ERR_UNSUPPORTED, "bf16/fp16 storage needs m <= 13 (one CTA per signal)");
    }
    p->tier = (m == 11 || m == 12) && (flags & CHW_FLAG_FORCE_SIMPLE) == 0 ? kTierLowp : kTierSimple;
  } else if ((flags & CHW_FLAG_FORCE_SIMPLE) != 0) {
    if (m > 13) {
      delete p;
      return fail(CHW_ERR_UNSUPPORTED, "the simple kernel takes m <= 13");
    }
    p->tier = kTierSimple;
  } else if ((flags & CHW_FLAG_FORCE_MULTIPASS) != 0 && m >= 11 && m <= 29) {
    p->tier = kTierTwoPass;
    p->passes = 2;
    p->row_bits = m - (m >= 23 ? (m - 17 > 6 ? m - 17 : 6) : 6);
  } else if (m == 17 && p->order == 0 && (flags & (CHW_FLAG_ROWSTACK | CHW_FLAG_CLUSTER | CHW_FLAG_TEST_STALL)) == 0) {
    // 2^17 words do not fit one SM: two SMs hold half a signal each in tensor memory and
    // exchange the last label bit over DSMEM (one HBM round trip); without that kernel the
    // two-pass split (a = 9), measured faster on GB300 than the 8-CTA cluster (3078 vs
    // 2722 GB/s on 2048 signals)
    if (chw::lookup_tmem_cross(17, fused_variant(p, true)) != nullptr) {
      p->tier = kTierTmemCross;
    } else {
      p->tier = kTierTwoPass;
      p->passes = 2;
      p->row_bits = 8;
    }
  } else if (m <= 17) {
    if (m < 5 && p->total % 32 != 0) {
      p->tier = kTierSimple;
    } else if (m >= 15) {
      const bool tmem = m <= 16 && p->order != 1 &&
                        (flags & (CHW_FLAG_ROWSTACK | CHW_FLAG_CLUSTER | CHW_FLAG_TEST_STALL)) == 0;
      p->tier = (flags & CHW_FLAG_ROWSTACK) != 0 ? kTierRowStack : (tmem ? kTierTmem : kTierCluster);
    } else {
      p->tier = kTierFused;
    }
  } else if (m <= 29 || (m == 30 && p->order == 0)) {
    p->tier = kTierTwoPass;
    p->passes = 2;
    const int a = two_pass_col_bits(m, p->order);
    p->row_bits = m - a;
  } else {
    delete p;
    return fail(CHW_ERR_UNSUPPORTED, "m=%d in sequency order needs three HBM passes, which this library does not implement", m);
  }

  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) {
    delete p;
    return fail(CHW_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  }
  e = cudaMalloc(&p->d_status, kStatusBytes);
  if (e != cudaSuccess) {
    delete p;
    return fail(CHW_ERR_CUDA, "cudaMalloc(status): %s", cudaGetErrorString(e));
  }
  cudaMemset(p->d_status, 0, kStatusBytes);
  if (autotune_requested(flags)) {
    r = autotune_plan(p);
    if (r != CHW_OK) {
      const std::string why = g_err;
      cudaFree(p->d_status);
      delete p;
      return fail(r, "%s", why.c_str());
    }
  }
  if (p->tier == kTierRowStack) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    p->rowstack_slots = sms > 0 ? sms : 1;
    if (p->rowstack_slots > batch) p->rowstack_slots = batch;
    p->workspace_bytes = static_cast<size_t>(p->rowstack_slots << m) * elem_bytes(dtype);
    e = cudaMalloc(&p->workspace, p->workspace_bytes);
    if (e != cudaSuccess) {
      const size_t bytes = p->workspace_bytes;
      cudaFree(p->d_status);
      delete p;
      cudaGetLastError();
      return fail(CHW_ERR_OOM, "workspace of %zu bytes: %s", bytes, cudaGetErrorString(e));
    }
  }
  if (p->tier == kTierTwoPass || p->tier == kTierTmemCross) {
    p->workspace_bytes = p->tier == kTierTmemCross ? cross_scratch_bytes(p->device)
                                                   : static_cast<size_t>(p->total) * elem_bytes(dtype);
    e = cudaMalloc(&p->workspace, p->workspace_bytes);
    if (e != cudaSuccess) {
      const size_t bytes = p->workspace_bytes;
      cudaFree(p->d_status);
      delete p;
      cudaGetLastError();
      return fail(CHW_ERR_OOM, "workspace of %zu bytes: %s", bytes, cudaGetErrorString(e));
    }
  }
  if (!is_lowp(dtype)) {
    p->haar_ws_bytes = static_cast<size_t>(chw::haar_scratch_words(m, batch)) * 4;
    if (p->haar_ws_bytes > 0 && cudaMalloc(&p->haar_ws, p->haar_ws_bytes) != cudaSuccess) {
      const size_t bytes = p->haar_ws_bytes;
      cudaGetLastError();
      chw_plan_destroy(p);
      return fail(CHW_ERR_OOM, "Haar scratch of %zu bytes", bytes);
    }
  }
  if ((flags & CHW_FLAG_HAAR_WALSH) != 0) {
    r = build_haar_walsh(p);
    if (r != CHW_OK) {
      const std::string why = g_err;
      chw_plan_destroy(p);
      return fail(r, "%s", why.c_str());
    }
  }
  *out = p;
  return CHW_OK;
}

chw_status_t chw_plan_destroy(chw_plan_t p) {
  if (p == nullptr) return CHW_OK;
  destroy_host_pipeline(p);
  if (p->workspace) cudaFree(p->workspace);
  if (p->d_status) cudaFree(p->d_status);
  if (p->ragged) chw::ragged_destroy(p->ragged);
  if (p->haar_ws) cudaFree(p->haar_ws);
  if (p->hw) chw::ragged_destroy(p->hw);
  for (chw_plan_s* b : p->hw_big)
    if (b) chw_plan_destroy(b);
  for (cudaStream_t h : p->hw_side)
    if (h) cudaStreamDestroy(h);
  for (cudaEvent_t h : p->hw_ev)
    if (h) cudaEventDestroy(h);
  delete p;
  return CHW_OK;
}

int chw_tune_candidates(int m, chw_dtype_t dtype, chw_norm_t norm, uint32_t flags, chw_tune_choice_t* out, int cap) {
  const std::vector<chw::TuneChoice> c = tune_candidates(m, dtype, norm, flags);
  for (int i = 0; out != nullptr && i < cap && i < static_cast<int>(c.size()); ++i)
    out[i] = chw_tune_choice_t{c[i].tier, c[i].row_bits, c[i].tile_bits};
  return static_cast<int>(c.size());
}

namespace {
int order_of(uint32_t flags) {
  return (flags & CHW_FLAG_ORDER_NATURAL) != 0 ? 1 : ((flags & CHW_FLAG_ORDER_SEQUENCY) != 0 ? 2 : 0);
}
}  // namespace

chw_status_t chw_tune_cache_put(const char* device, int m, int64_t batch, chw_dtype_t dtype, chw_norm_t norm,
                                uint32_t flags, const chw_tune_choice_t* choice, float us) {
  if (device == nullptr || choice == nullptr) return fail(CHW_ERR_INVALID_ARG, "NULL device name or choice");
  if (batch < 1 || m < 0 || m > CHW_MAX_M) return fail(CHW_ERR_INVALID_ARG, "bad m or batch");
  chw::tune_cache_put(chw::tune_key(device, m, batch, dtype, norm, order_of(flags)),
                      chw::TuneChoice{choice->tier, choice->row_bits, choice->tile_bits}, us);
  return CHW_OK;
}

chw_status_t chw_tune_cache_get(const char* device, int m, int64_t batch, chw_dtype_t dtype, chw_norm_t norm,
                                uint32_t flags, chw_tune_choice_t* choice, float* us) {
  if (device == nullptr || choice == nullptr) return fail(CHW_ERR_INVALID_ARG, "NULL device name or choice");
  if (batch < 1 || m < 0 || m > CHW_MAX_M) return fail(CHW_ERR_INVALID_ARG, "bad m or batch");
  chw::TuneChoice c{};
  if (!chw::tune_cache_get(chw::tune_key(device, m, batch, dtype, norm, order_of(flags)), &c, us))
    return fail(CHW_ERR_UNSUPPORTED, "no cached choice for this key");
  *choice = chw_tune_choice_t{c.tier, c.row_bits, c.tile_bits};
  return CHW_OK;
}

int chw_tune_cache_load(const char* path) { return chw::tune_cache_load(path); }

chw_status_t chw_tune_cache_save(const char* path) {
  if (path == nullptr) return fail(CHW_ERR_INVALID_ARG, "NULL path");
  if (!chw::tune_cache_save(path)) return fail(CHW_ERR_INVALID_ARG, "cannot write %s", path);
  return CHW_OK;
}

void chw_tune_cache_clear(void) { chw::tune_cache_clear(); }

chw_status_t chw_plan_get_info(chw_plan_t p, chw_plan_info_t* info) {
  if (p == nullptr || info == nullptr) return fail(CHW_ERR_INVALID_ARG, "NULL plan or info");
  std::memset(info, 0, sizeof(*info));
  info->m = p->ragged ? -1 : p->m;
  info->batch = p->batch;
  info->dtype = p->dtype;
  info->norm = p->norm;
  info->tier = p->tier;
  info->passes = p->passes;
  info->row_bits = p->row_bits;
  info->cluster = 1;
  info->kernels_per_call = p->passes;
  if (p->tier == kTierFused || p->tier == kTierCluster) info->cluster = 1 << row_shape(p->m, p->tile_bits).cb;
  if (p->tier == kTierTmemCross) info->cluster = 1 << (p->m - 16);
  if (p->tier == kTierTwoPass)
    info->cluster = tmem_row_pass(p, p->row_bits, p->order == 1 ? 4 : 1) ? 1 : 1 << row_shape(p->row_bits, p->tile_bits).cb;
  info->workspace_bytes = static_cast<int64_t>(p->workspace_bytes);
  info->total_elements = p->total;
  info->order = p->order;
  info->tile_bits = p->tile_bits;
  info->tuned = p->tuned;
  info->tune_us = p->tune_us;
  if (p->ragged) {
    info->kernels_per_call = chw::ragged_launches(p->ragged);  // all replayed by one graph launch
    info->workspace_bytes = static_cast<int64_t>(chw::ragged_workspace_bytes(p->ragged));
  }
  return CHW_OK;
}

static chw_status_t forward_common(chw_plan_t p, const void* x, void* y, const int32_t* exp_in, int32_t* exp_out,
                                   const int8_t* diag_in, const int8_t* diag_out, void* stream) {
  g_err.clear();
  if (p == nullptr) return fail(CHW_ERR_INVALID_ARG, "plan is NULL");
  if (p->ragged) return fail(CHW_ERR_INVALID_ARG, "ragged plans run through chw_forward_ragged");
  chw_status_t r = validate_data_ptr(x, "x");
  if (r != CHW_OK) return r;
  r = validate_data_ptr(y, "y");
  if (r != CHW_OK) return r;
  if (is_lowp(p->dtype)) {
    if (exp_in == nullptr || exp_out == nullptr) return fail(CHW_ERR_INVALID_ARG, "bf16/fp16 need exp_in and exp_out");
  } else if (exp_in != nullptr || exp_out != nullptr) {
    return fail(CHW_ERR_INVALID_ARG, "exp_in/exp_out are for bf16/fp16 only");
  }
  return run_transform(p, x, y, p->batch, exp_in, exp_out, diag_in, diag_out, p->workspace,
                       static_cast<cudaStream_t>(stream));
}

chw_status_t chw_forward(chw_plan_t p, const void* x, void* y, const int32_t* exp_in, int32_t* exp_out,
                         const int8_t* diag, void* stream) {
  return forward_common(p, x, y, exp_in, exp_out, nullptr, diag, stream);
}

chw_status_t chw_adjoint(chw_plan_t p, const void* y, void* x, const int32_t* exp_in, int32_t* exp_out,
                         const int8_t* diag, void* stream) {
  // H^T = H: the reversed cascade of Psi^T stages performs the forward butterflies with
  // inputs and outputs relabelled, so the same kernels run; D is applied to the input.
  return forward_common(p, y, x, exp_in, exp_out, diag, nullptr, stream);
}

chw_status_t chw_forward_host(chw_plan_t p, const void* x_host, void* y_host, const int32_t* exp_in_host,
                              int32_t* exp_out_host, const int8_t* diag_host) {
  g_err.clear();
  if (p == nullptr) return fail(CHW_ERR_INVALID_ARG, "plan is NULL");
  if (p->ragged) return fail(CHW_ERR_INVALID_ARG, "ragged plans run through chw_forward_ragged");
  if (x_host == nullptr || y_host == nullptr) return fail(CHW_ERR_INVALID_ARG, "x_host / y_host is NULL");
  const bool lowp = is_lowp(p->dtype);
  if (lowp && (exp_in_host == nullptr || exp_out_host == nullptr))
    return fail(CHW_ERR_INVALID_ARG, "bf16/fp16 need exp_in_host and exp_out_host");
  if (!lowp && (exp_in_host != nullptr || exp_out_host != nullptr))
    return fail(CHW_ERR_INVALID_ARG, "exp_in_host/exp_out_host are for bf16/fp16 only");
  const int64_t n = int64_t{1} << p->m;
  const size_t eb = elem_bytes(p->dtype);
  if (p->h_chunk == 0) {
    // chunks of about 64 MiB (at least one signal) cycle over three streams so that the
    // copy in, the transform and the copy out of consecutive chunks overlap
    int64_t chunk = (int64_t{64} << 20) / static_cast<int64_t>(n * eb);
    if (chunk < 1) chunk = 1;
    if (chunk > p->batch) chunk = p->batch;
    if (p->tier == kTierSimple || lowp) {
      // whole signals per chunk already
    } else if (p->m < 5) {
      while ((chunk * n) % 32 != 0 && chunk < p->batch) ++chunk;
    }
    p->h_chunk = chunk;
    const size_t bytes = static_cast<size_t>(chunk * n) * eb;
    for (int i = 0; i < 3; ++i) {
      if (cudaStreamCreateWithFlags(&p->h_stream[i], cudaStreamNonBlocking) != cudaSuccess ||
          cudaMalloc(&p->h_buf[i], bytes) != cudaSuccess ||
          (p->tier == kTierTwoPass && cudaMalloc(&p->h_ws[i], bytes) != cudaSuccess) ||
          (p->tier == kTierTmemCross && cudaMalloc(&p->h_ws[i], cross_scratch_bytes(p->device)) != cudaSuccess) ||
          (p->tier == kTierRowStack &&
           cudaMalloc(&p->h_ws[i], static_cast<size_t>(p->rowstack_slots << p->m) * eb) != cudaSuccess) ||
          (lowp && (cudaMalloc(&p->h_exp[i][0], chunk * sizeof(int32_t)) != cudaSuccess ||
                    cudaMalloc(&p->h_exp[i][1], chunk * sizeof(int32_t)) != cudaSuccess))) {
        cudaGetLastError();
        destroy_host_pipeline(p);
        return fail(CHW_ERR_OOM, "host pipeline buffers");
      }
    }
    if (cudaMalloc(&p->h_diag, static_cast<size_t>(n)) != cudaSuccess) {
      cudaGetLastError();
      destroy_host_pipeline(p);
      return fail(CHW_ERR_OOM, "host pipeline diag buffer");
    }
  }
  const int8_t* d_diag = nullptr;
  if (diag_host != nullptr) {
    CHW_CUDA(cudaMemcpy(p->h_diag, diag_host, static_cast<size_t>(n), cudaMemcpyHostToDevice));
    d_diag = p->h_diag;
  }
  const int64_t chunk = p->h_chunk;
  int i = 0;
  for (int64_t s0 = 0; s0 < p->batch; s0 += chunk, i = (i + 1) % 3) {
    const int64_t cnt = (p->batch - s0) < chunk ? (p->batch - s0) : chunk;
    const size_t off = static_cast<size_t>(s0 * n) * eb, bytes = static_cast<size_t>(cnt * n) * eb;
    cudaStream_t st = p->h_stream[i];
    CHW_CUDA(cudaMemcpyAsync(p->h_buf[i], static_cast<const uint8_t*>(x_host) + off, bytes, cudaMemcpyHostToDevice, st));
    if (lowp)
      CHW_CUDA(cudaMemcpyAsync(p->h_exp[i][0], exp_in_host + s0, cnt * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    const int64_t saved = p->batch;
    chw_status_t r;
    {
      // the transform of this chunk, in place in the staging buffer
      if (p->tier != kTierSimple && !lowp && p->m < 5 && (cnt * n) % 32 != 0) {
        const int tier = p->tier;
        p->tier = kTierSimple;
        r = run_transform(p, p->h_buf[i], p->h_buf[i], cnt, nullptr, nullptr, nullptr, d_diag, nullptr, st);
        p->tier = tier;
      } else {
        r = run_transform(p, p->h_buf[i], p->h_buf[i], cnt, lowp ? p->h_exp[i][0] : nullptr,
                          lowp ? p->h_exp[i][1] : nullptr, nullptr, d_diag, p->h_ws[i], st);
      }
    }
    (void)saved;
    if (r != CHW_OK) return r;
    CHW_CUDA(cudaMemcpyAsync(static_cast<uint8_t*>(y_host) + off, p->h_buf[i], bytes, cudaMemcpyDeviceToHost, st));
    if (lowp)
      CHW_CUDA(cudaMemcpyAsync(exp_out_host + s0, p->h_exp[i][1], cnt * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  }
  for (int k = 0; k < 3; ++k) CHW_CUDA(cudaStreamSynchronize(p->h_stream[k]));
  return CHW_OK;
}

chw_status_t chw_last_device_status(chw_plan_t p) {
  g_err.clear();
  if (p == nullptr) return fail(CHW_ERR_INVALID_ARG, "plan is NULL");
  CHW_CUDA(cudaDeviceSynchronize());
  int s = 0;
  int64_t index = 0;
  chw_status_t r = take_status(p->d_status, &s, &index);
  if (r != CHW_OK) return r;
  for (chw_plan_s* b : p->hw_big) {
    if (b == nullptr) continue;
    int sb = 0;
    int64_t ib = 0;
    r = take_status(b->d_status, &sb, &ib);
    if (r != CHW_OK) return r;
    if (s == 0) {
      s = sb;
      index = ib;
    }
  }
  if (s == CHW_ERR_DEVICE_CHECK)
    return fail(CHW_ERR_DEVICE_CHECK, "device check failed: element index %lld out of range",
                static_cast<long long>(index));
  if (s != 0) return fail(static_cast<chw_status_t>(s), "device reported %s", chw_status_string(static_cast<chw_status_t>(s)));
  return CHW_OK;
}

chw_status_t chw_haar(chw_plan_t p, const void* x, void* z, void* stream) {
  g_err.clear();
  chw_status_t r = check_haar_call(p, x, z, "x", "z");
  if (r != CHW_OK) return r;
  if (overlaps(x, z, static_cast<size_t>(p->total) * 4)) return fail(CHW_ERR_INVALID_ARG, "x and z overlap");
  CHW_CUDA(chw::haar_forward(fused_variant(p, true), p->m, p->batch, x, z, p->haar_ws, p->d_status,
                             static_cast<cudaStream_t>(stream)));
  return CHW_OK;
}

chw_status_t chw_haar_inverse(chw_plan_t p, const void* z, void* x, void* stream) {
  g_err.clear();
  chw_status_t r = check_haar_call(p, z, x, "z", "x");
  if (r != CHW_OK) return r;
  if (overlaps(x, z, static_cast<size_t>(p->total) * 4)) return fail(CHW_ERR_INVALID_ARG, "z and x overlap");
  CHW_CUDA(chw::haar_inverse(fused_variant(p, true), p->m, p->batch, z, x, p->haar_ws,
                             static_cast<cudaStream_t>(stream)));
  return CHW_OK;
}

chw_status_t chw_from_haar(chw_plan_t p, const void* z, void* y, void* stream) {
  g_err.clear();
  chw_status_t r = check_haar_call(p, z, y, "z", "y");
  if (r != CHW_OK) return r;
  if (p->hw == nullptr && !p->hw_ready) return fail(CHW_ERR_INVALID_ARG, "the plan was made without CHW_FLAG_HAAR_WALSH");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (p->hw_ready) return run_haar_walsh(p, z, y, st);
  std::string why;
  if (chw::ragged_run(p->hw, z, y, st, &why) != 0) return fail(CHW_ERR_CUDA, "Haar-Walsh scales: %s", why.c_str());
  for (int k = chw::kRaggedMaxM + 1; k < p->m; ++k) {
    chw_plan_s* b = p->hw_big[k];
    for (int64_t s = 0; s < p->batch; ++s) {
      const int64_t o = (s << p->m) + (int64_t{1} << k);
      r = run_transform(b, static_cast<const uint32_t*>(z) + o, static_cast<uint32_t*>(y) + o, 1, nullptr, nullptr,
                        nullptr, nullptr, b->workspace, st);
      if (r != CHW_OK) return r;
    }
  }
  return CHW_OK;
}

chw_status_t chw_forward_haar(chw_plan_t p, const void* x, void* y, void* z, void* stream) {
  g_err.clear();
  chw_status_t r = check_haar_call(p, x, y, "x", "y");
  if (r != CHW_OK) return r;
  r = validate_data_ptr(z, "z");
  if (r != CHW_OK) return r;
  const size_t bytes = static_cast<size_t>(p->total) * 4;
  if (overlaps(x, z, bytes) || overlaps(y, z, bytes)) return fail(CHW_ERR_INVALID_ARG, "z overlaps x or y");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  // One HBM round trip where the tier's kernels capture stage 0 (single-CTA row tiles of
  // whole signals, the tensor-memory tier): z leaves the same pass as y.
  const bool fused = p->m >= 1 && p->order == 0 &&
                     (p->tier == kTierTmem || (p->tier == kTierFused && row_shape(p->m, p->tile_bits).cb == 0));
  if (fused) {
    p->call_haar_z = z;
    r = run_transform(p, x, y, p->batch, nullptr, nullptr, nullptr, nullptr, p->workspace, st);
    p->call_haar_z = nullptr;
    return r;
  }
  // Otherwise z first (x may be y), then y, by the plan's own kernels.
  r = chw_haar(p, x, z, stream);
  if (r != CHW_OK) return r;
  return run_transform(p, x, y, p->batch, nullptr, nullptr, nullptr, nullptr, p->workspace, st);
}

}  // extern "C"

namespace {

// A ragged plan over signals at `offsets` (count + 1 entries, the last one = total).
chw_status_t make_ragged(chw_plan_t* out, const uint8_t* ms_host, const int64_t* offsets, int64_t count,
                         chw_dtype_t dtype, chw_norm_t norm, uint32_t flags) {
  auto* p = new chw_plan_s();
  p->m = -1;
  p->batch = count;
  p->dtype = dtype;
  p->norm = norm;
  p->flags = flags;
  p->tier = kTierRagged;
  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_status, kStatusBytes);
  if (e != cudaSuccess) {
    delete p;
    return fail(CHW_ERR_CUDA, "ragged plan: %s", cudaGetErrorString(e));
  }
  cudaMemset(p->d_status, 0, kStatusBytes);
  std::vector<int64_t> off(offsets, offsets + count + 1);
  if ((flags & CHW_FLAG_TEST_CORRUPT) != 0) {
    // test hook (checked plans only): the first signal with m >= 13 and the first with
    // m <= 12 get offsets past the end of x and y (32-aligned, so only the range is wrong)
    const int64_t past = ((off[count] + (int64_t{1} << 20)) + 31) & ~int64_t{31};
    bool big = false, small = false;
    for (int64_t i = 0; i < count; ++i) {
      if (!big && ms_host[i] >= 13) {
        off[i] = past;
        big = true;
      } else if (!small && ms_host[i] <= 12) {
        off[i] = past + (int64_t{1} << 21);
        small = true;
      }
    }
  }
  std::string why;
  p->ragged = chw::ragged_create_at(ms_host, off.data(), count, off[count],
                                    dtype == CHW_I32 ? chw::kVarI32 : fused_variant(p, true), p->d_status,
                                    autotune_requested(flags), &why, (flags & CHW_FLAG_CHECKED) != 0);
  if (p->ragged != nullptr && chw::ragged_tuned(p->ragged)) p->tuned = 1;
  if (p->ragged == nullptr) {
    cudaFree(p->d_status);
    delete p;
    return fail(CHW_ERR_OOM, "ragged plan: %s", why.c_str());
  }
  p->total = chw::ragged_total(p->ragged);
  p->passes = chw::ragged_passes(p->ragged);
  *out = p;
  return CHW_OK;
}

chw_status_t check_ragged_args(chw_plan_t* out, const uint8_t* ms_host, int64_t count, chw_dtype_t dtype,
                               chw_norm_t norm, uint32_t flags) {
  if (out == nullptr) return fail(CHW_ERR_INVALID_ARG, "plan output pointer is NULL");
  *out = nullptr;
  if (ms_host == nullptr || count < 1) return fail(CHW_ERR_INVALID_ARG, "ms_host is NULL or count < 1");
  if (count > (int64_t{1} << 31) - 1) return fail(CHW_ERR_INVALID_ARG, "count must be below 2^31");
  if (dtype != CHW_F32 && dtype != CHW_I32) return fail(CHW_ERR_UNSUPPORTED, "ragged plans take int32 or fp32");
  chw_status_t r = check_plan_args(0, 1, dtype, norm);
  if (r != CHW_OK) return r;
  if ((flags & CHW_FLAG_TEST_CORRUPT) != 0 && (flags & CHW_FLAG_CHECKED) == 0)
    return fail(CHW_ERR_INVALID_ARG, "CHW_FLAG_TEST_CORRUPT runs only with CHW_FLAG_CHECKED");
  for (int64_t i = 0; i < count; ++i)
    if (ms_host[i] > chw::kRaggedMaxM)
      return fail(CHW_ERR_INVALID_ARG, "ms[%lld]=%d outside 0..%d", static_cast<long long>(i), ms_host[i],
                  chw::kRaggedMaxM);
  return CHW_OK;
}

}  // namespace

extern "C" {

chw_status_t chw_plan_ragged(chw_plan_t* out, const uint8_t* ms_host, int64_t count, chw_dtype_t dtype,
                             chw_norm_t norm, uint32_t flags) {
  g_err.clear();
  chw_status_t r = check_ragged_args(out, ms_host, count, dtype, norm, flags);
  if (r != CHW_OK) return r;
  std::vector<int64_t> off(count + 1);
  chw::ragged_pack(ms_host, count, off.data());
  return make_ragged(out, ms_host, off.data(), count, dtype, norm, flags);
}

chw_status_t chw_plan_ragged_at(chw_plan_t* out, const uint8_t* ms_host, const int64_t* offsets_host, int64_t count,
                                int64_t total, chw_dtype_t dtype, chw_norm_t norm, uint32_t flags) {
  g_err.clear();
  chw_status_t r = check_ragged_args(out, ms_host, count, dtype, norm, flags);
  if (r != CHW_OK) return r;
  if (offsets_host == nullptr) return fail(CHW_ERR_INVALID_ARG, "offsets_host is NULL");
  if (total < 1 || total > (int64_t{1} << 40)) return fail(CHW_ERR_INVALID_ARG, "total outside 1..2^40");
  std::vector<int64_t> order(count);
  for (int64_t i = 0; i < count; ++i) {
    const int64_t o = offsets_host[i], n = int64_t{1} << ms_host[i];
    if (o < 0 || o > total - n)
      return fail(CHW_ERR_INVALID_ARG, "signal %lld at [%lld, %lld) is not inside [0, %lld)", static_cast<long long>(i),
                  static_cast<long long>(o), static_cast<long long>(o + n), static_cast<long long>(total));
    if (ms_host[i] >= 13 && o % 32 != 0)
      return fail(CHW_ERR_ALIGNMENT, "signal %lld (m=%d) must start on a 32-element boundary (offset %lld)",
                  static_cast<long long>(i), ms_host[i], static_cast<long long>(o));
    order[i] = i;
  }
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return offsets_host[a] < offsets_host[b]; });
  for (int64_t k = 1; k < count; ++k) {
    const int64_t a = order[k - 1], b = order[k];
    if (offsets_host[b] < offsets_host[a] + (int64_t{1} << ms_host[a]))
      return fail(CHW_ERR_INVALID_ARG, "signals %lld and %lld overlap", static_cast<long long>(a),
                  static_cast<long long>(b));
  }
  std::vector<int64_t> off(offsets_host, offsets_host + count);
  off.push_back(total);
  return make_ragged(out, ms_host, off.data(), count, dtype, norm, flags);
}

chw_status_t chw_ragged_offsets(chw_plan_t p, int64_t* offsets_host) {
  if (p == nullptr || p->ragged == nullptr || offsets_host == nullptr)
    return fail(CHW_ERR_INVALID_ARG, "not a ragged plan, or NULL output");
  chw::ragged_offsets(p->ragged, offsets_host);
  return CHW_OK;
}

chw_status_t chw_forward_ragged(chw_plan_t p, const void* x, void* y, void* stream) {
  g_err.clear();
  if (p == nullptr || p->ragged == nullptr) return fail(CHW_ERR_INVALID_ARG, "not a ragged plan");
  chw_status_t r = validate_data_ptr(x, "x");
  if (r != CHW_OK) return r;
  r = validate_data_ptr(y, "y");
  if (r != CHW_OK) return r;
  std::string why;
  const int rc = chw::ragged_run(p->ragged, x, y, static_cast<cudaStream_t>(stream), &why);
  if (rc != 0) return fail(CHW_ERR_CUDA, "ragged run: %s", why.c_str());
  return CHW_OK;
}

}  // extern "C"
