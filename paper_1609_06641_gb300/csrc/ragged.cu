// Host side of ragged plans: packing, grouping by length, graph capture (see ragged.cuh).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "ragged_kernel.cuh"

namespace chw {

// One translation unit per variant instantiates the short-signal kernel (generated by the build).
extern template cudaError_t launch_ragged_small<kVarPerLevel>(const RaggedArgs&, cudaStream_t);
extern template cudaError_t launch_ragged_small<kVarEnd>(const RaggedArgs&, cudaStream_t);
extern template cudaError_t launch_ragged_small<kVarPlain>(const RaggedArgs&, cudaStream_t);
extern template cudaError_t launch_ragged_small<kVarI32>(const RaggedArgs&, cudaStream_t);

// ------------------------------------------------------------------ host side
struct RaggedGroup {
  int m = 0;
  int64_t count = 0;
  int64_t* d_off = nullptr;  // the group's signal offsets (device)
  int opt = 0;               // the group's configuration (see group_options)
  bool aligned = false;      // every offset is a multiple of ragged_align(m)
};

struct RaggedPlan {
  int64_t count = 0;
  bool checked = false;
  std::vector<uint8_t> ms;
  std::vector<int64_t> off;  // count + 1 entries
  int64_t total = 0;
  int variant = 0;
  int* d_status = nullptr;
  // short signals: a work list for the persistent kernel
  int ntasks = 0;
  RaggedTask* d_tasks = nullptr;
  int32_t* d_head = nullptr;
  uint8_t* d_ms = nullptr;
  int64_t* d_off = nullptr;
  // longer signals: one batched launch (two per chunk for m >= 18) per length
  std::vector<RaggedGroup> groups;
  uint32_t* d_scratch = nullptr;
  int64_t scratch_words = 0;
  uint4* d_xscratch = nullptr;  // exchange slots of the m = 17 pair kernel
  int64_t xclusters = 0;
  int launches = 0;
  bool tuned = false;
  cudaStream_t cap = nullptr;
  cudaStream_t side = nullptr;  // second branch of the recorded graph
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaGraphExec_t exec = nullptr;
  const void* gx = nullptr;
  void* gy = nullptr;
};

namespace {

void free_plan(RaggedPlan* r) {
  if (r->exec) cudaGraphExecDestroy(r->exec);
  if (r->cap) cudaStreamDestroy(r->cap);
  if (r->side) cudaStreamDestroy(r->side);
  if (r->fork) cudaEventDestroy(r->fork);
  if (r->join) cudaEventDestroy(r->join);
  cudaFree(r->d_tasks);
  cudaFree(r->d_head);
  cudaFree(r->d_ms);
  cudaFree(r->d_off);
  for (RaggedGroup& g : r->groups) cudaFree(g.d_off);
  cudaFree(r->d_scratch);
  cudaFree(r->d_xscratch);
  delete r;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return enc;
}

bool encode_rows(CUtensorMap* map, const void* ptr, int64_t words) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {32, static_cast<cuuint64_t>(words / 32)};
  cuuint64_t strides[1] = {128};
  cuuint32_t box[2] = {32, 256};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void*>(ptr), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

float end_scale_host(int m) {  // fp32(2^{-m/2}), as the kernels compute it
  const float r = (m & 1) ? 0.70710678118654752440f : 1.0f;
  return std::ldexp(r, -(m / 2));
}

// Configurations of a length group (RaggedGroup::opt).
//   m = 13, 14   one: the batched single-CTA kernel.
//   m = 15, 16   0: clusters of 2^14-word tiles; 1: clusters of 2^13-word tiles; 2 (aligned
//                groups only, the built-in choice there): one signal per SM in tensor memory.
//   m = 17       0: 8-CTA cluster; 1: the two-pass split with a = 9; 2 (aligned groups only,
//                the built-in choice there): a pair of SMs per signal in tensor memory.
//   m = 18..20   the two-pass split with a = 9 (0), 8 (1) or 10 (2) column bits.
// The tensor-memory kernels store each signal's output by TMA as runs of 2^(m-8) words, so
// they need offsets that are multiples of that (ragged_align); the library's packing gives
// them, caller offsets may.
int group_options(int m, bool aligned) {
  if (m == 15 || m == 16 || m == 17) return aligned ? 3 : 2;
  if (m >= 18) return 3;
  return 1;
}

int default_option(int m, bool aligned) { return aligned && m >= 15 && m <= 17 ? 2 : 0; }

bool tmem_opt(int m, int opt) { return m >= 15 && m <= 17 && opt == 2; }

bool two_pass_opt(int m, int opt) { return m >= 18 || (m == 17 && opt == 1); }


// The output of a tensor-memory launch over the whole packed array: rows of 2^(m-8) words,
// boxes of 32 words x 256 rows (one signal), SWIZZLE_128B.  Rows past the last whole one
// hold no aligned signal's output.
bool encode_runs(CUtensorMap* map, void* ptr, int64_t words, int m) {
  auto enc = tensor_map_encoder();
  if (!enc || (words >> (m - 8)) < 256) return false;
  cuuint64_t dims[2] = {cuuint64_t{1} << (m - 8), static_cast<cuuint64_t>(words >> (m - 8))};
  cuuint64_t strides[1] = {cuuint64_t{4} << (m - 8)};
  cuuint32_t box[2] = {32, 256};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

int two_pass_a(int m, int opt) {
  if (m == 17) return 9;
  return opt == 1 ? 8 : (opt == 2 ? 10 : 9);
}

int64_t two_pass_chunk(int m) { return std::max<int64_t>(1, kRaggedScratchWords >> m); }

int group_launches(const RaggedGroup& g) {
  if (!two_pass_opt(g.m, g.opt)) return 1;
  return static_cast<int>(2 * ((g.count + two_pass_chunk(g.m) - 1) / two_pass_chunk(g.m)));
}

// Record (or issue) the launches of `count` signals of one length group on stream `st`.
cudaError_t launch_group(const RaggedPlan* r, const RaggedGroup& g, int64_t count, const CUtensorMap& tx,
                         const CUtensorMap& ts, void* y, cudaStream_t st) {
  const int m = g.m;
  if (tmem_opt(m, g.opt)) {
    // one signal per SM (m = 15, 16) or per pair of SMs (m = 17) in tensor memory, each
    // signal read and written at its own (aligned) offset
    if (!g.aligned) return cudaErrorInvalidValue;
    TmemLaunchFn fn = m == 17 ? lookup_tmem_cross(17, r->variant) : lookup_tmem(m, r->variant, 0);
    CUtensorMap tout;
    if (!fn || !encode_runs(&tout, y, r->total, m)) return cudaErrorInvalidValue;
    FusedArgs a{};
    a.status = r->d_status;
    a.checked = r->checked;
    a.in_total = r->total;
    a.out = y;
    a.out_total = r->total;
    a.end_scale = end_scale_host(m);
    a.diag_mask = (int64_t{1} << m) - 1;
    a.in_off = g.d_off;
    a.out_off = g.d_off;
    a.sig_shift = 0;
    if (m == 17) {
      if (r->d_xscratch == nullptr) return cudaErrorInvalidValue;
      a.xscratch = r->d_xscratch;
      a.xclusters = r->xclusters;
    }
    return fn(&tx, &tout, a, count, st);
  }
  if (!two_pass_opt(m, g.opt)) {
    const int tb = m == 13 ? 13 : ((m == 15 || m == 16) && g.opt == 1 ? 13 : 14);
    const int cb = m - tb > 0 ? m - tb : 0;
    FusedLaunchFn fn = lookup_fused(0, m, tb, cb, r->variant, 0);
    if (!fn) return cudaErrorInvalidValue;
    FusedArgs a{};
    a.status = r->d_status;
    a.checked = r->checked;
    a.in_total = r->total;
    a.out = y;
    a.out_total = r->total;
    a.end_scale = end_scale_host(m);
    a.in_off = g.d_off;
    a.out_off = g.d_off;
    a.sig_shift = 0;
    return fn(&tx, a, count, st);
  }
  // Two passes: pass 1 on rows of 2^b (2^(13-b) rows per 2^13-word tile, 2^(m-13) tiles per
  // signal) into column-blocked scratch; pass 2 on 2^a x 32 column tiles (2^(tb+cb) words,
  // 2^(m-tb-cb) per signal) written back at the signal's offset.
  const int A = two_pass_a(m, g.opt), b = m - A;
  const int tb2 = A <= 8 ? 13 : 14, cb2 = A <= 9 ? 0 : A - 9, ub2 = tb2 + cb2;
  const int v1 = r->variant == kVarEnd ? static_cast<int>(kVarPlain) : r->variant;
  FusedLaunchFn f1 = lookup_fused(0, b, 13, 0, v1, 1);
  FusedLaunchFn f2 = lookup_fused(5, A, tb2, cb2, r->variant, 0);
  if (!f1 || !f2) return cudaErrorInvalidValue;
  const int64_t chunk = two_pass_chunk(m);
  for (int64_t s0 = 0; s0 < count; s0 += chunk) {
    const int64_t cnt = std::min(chunk, count - s0);
    FusedArgs p1{};
    p1.status = r->d_status;
    p1.checked = r->checked;
    p1.in_total = r->total;
    p1.out = r->d_scratch;
    p1.out_total = cnt << m;
    p1.end_scale = 1.0f;
    p1.colblock_a = A;
    p1.in_off = g.d_off + s0;
    p1.sig_shift = m - 13;
    cudaError_t e = f1(&tx, p1, cnt << (m - 13), st);
    if (e != cudaSuccess) return e;
    FusedArgs p2{};
    p2.status = r->d_status;
    p2.checked = r->checked;
    p2.in_total = cnt << m;
    p2.out = y;
    p2.out_total = r->total;
    p2.end_scale = end_scale_host(m);
    p2.out_off = g.d_off + s0;
    p2.sig_shift = m - ub2;
    e = f2(&ts, p2, cnt << (m - ub2), st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Time every configuration of every group with more than one, on up to 2^26 words of the
// group's signals (offsets into temporary arrays of the plan's size, CUDA events, one
// warm-up and the mean of three runs), and keep each group's fastest.  Skipped (built-in
// choices kept) when the temporary arrays cannot be allocated.
void tune_groups(RaggedPlan* r) {
  void *x = nullptr, *y = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const size_t bytes = static_cast<size_t>(r->total) * 4;
  if (cudaMalloc(&x, bytes) != cudaSuccess || cudaMalloc(&y, bytes) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
  } else {
    cudaMemset(x, 0x3c, bytes);
    CUtensorMap tx, ts;
    const void* sp = r->d_scratch != nullptr ? static_cast<const void*>(r->d_scratch) : x;
    const int64_t sw = r->d_scratch != nullptr ? r->scratch_words : r->total;
    if (encode_rows(&tx, x, r->total) && encode_rows(&ts, sp, sw)) {
      for (RaggedGroup& g : r->groups) {
        const int nopt = group_options(g.m, g.aligned);
        if (nopt < 2) continue;
        const int64_t cnt = std::min<int64_t>(g.count, std::max<int64_t>(1, (int64_t{1} << 26) >> g.m));
        int best = 0;
        float best_ms = -1.f;
        for (int opt = 0; opt < nopt; ++opt) {
          g.opt = opt;
          bool ok = launch_group(r, g, cnt, tx, ts, y, r->cap) == cudaSuccess;
          cudaEventRecord(e0, r->cap);
          for (int k = 0; k < 3 && ok; ++k) ok = launch_group(r, g, cnt, tx, ts, y, r->cap) == cudaSuccess;
          cudaEventRecord(e1, r->cap);
          float ms = 0.f;
          int st = 0;
          ok = ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
          cudaMemcpy(&st, r->d_status, sizeof(int), cudaMemcpyDeviceToHost);
          cudaMemset(r->d_status, 0, sizeof(int));
          cudaGetLastError();
          if (ok && st == 0 && (best_ms < 0.f || ms < best_ms)) {
            best = opt;
            best_ms = ms;
          }
        }
        g.opt = best;
      }
      r->tuned = true;
    }
  }
  if (x) cudaFree(x);
  if (y) cudaFree(y);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
}

}  // namespace

int64_t ragged_align(int m) { return m >= 15 && m <= 17 ? int64_t{1} << (m - 8) : 32; }

void ragged_pack(const uint8_t* ms, int64_t count, int64_t* off) {
  int64_t o = 0;
  for (int64_t i = 0; i < count; ++i) {
    const int64_t al = ragged_align(ms[i]);  // 128 bytes, or a whole output run (m = 15..17)
    o = (o + al - 1) & ~(al - 1);
    off[i] = o;
    o += int64_t{1} << ms[i];
    o = (o + 31) & ~int64_t{31};
  }
  off[count] = o;
}

RaggedPlan* ragged_create(const uint8_t* ms, int64_t count, int variant, int* d_status, bool tune, std::string* why) {
  std::vector<int64_t> off(count + 1);
  ragged_pack(ms, count, off.data());
  return ragged_create_at(ms, off.data(), count, off[count], variant, d_status, tune, why);
}

RaggedPlan* ragged_create_at(const uint8_t* ms, const int64_t* offsets, int64_t count, int64_t total, int variant,
                             int* d_status, bool tune, std::string* why, bool checked) {
  auto* r = new RaggedPlan();
  r->count = count;
  r->checked = checked;
  r->ms.assign(ms, ms + count);
  r->off.assign(offsets, offsets + count);
  r->off.push_back(total);
  r->variant = variant;
  r->d_status = d_status;
  r->total = total;

  // ---- short signals: runs of consecutive short signals, about 128 KiB each
  std::vector<RaggedTask> tasks;
  for (int64_t i = 0; i < count;) {
    if (ms[i] > kRaggedSmallMaxM) {
      ++i;
      continue;
    }
    RaggedTask t{};
    t.index = static_cast<int32_t>(i);
    int64_t words = 0;
    while (i < count && ms[i] <= kRaggedSmallMaxM && words < kSmallGroupWords) {
      words += int64_t{1} << ms[i];
      ++i;
      ++t.count;
    }
    tasks.push_back(t);
  }
  r->ntasks = static_cast<int>(tasks.size());
  if (r->ntasks > 0) r->launches += 1;

  // ---- longer signals: one group per length
  cudaError_t e = cudaSuccess;
  for (int m = kRaggedSmallMaxM + 1; m <= kRaggedMaxM && e == cudaSuccess; ++m) {
    std::vector<int64_t> go;
    for (int64_t i = 0; i < count; ++i)
      if (ms[i] == m) go.push_back(offsets[i]);
    if (go.empty()) continue;
    RaggedGroup g;
    g.m = m;
    g.count = static_cast<int64_t>(go.size());
    g.aligned = std::all_of(go.begin(), go.end(), [&](int64_t o) { return o % ragged_align(m) == 0; }) &&
                (total >> (m - 8)) >= 256;
    g.opt = default_option(m, g.aligned);
    if (m == 17 && g.aligned && r->d_xscratch == nullptr && e == cudaSuccess) {
      int dev = 0;
      cudaGetDevice(&dev);
      r->xclusters = tmem_cross_clusters(dev);
      e = cudaMalloc(&r->d_xscratch, static_cast<size_t>(r->xclusters) << 17);
    }
    e = cudaMalloc(&g.d_off, go.size() * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMemcpy(g.d_off, go.data(), go.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    r->groups.push_back(g);
    if (m >= (tune ? 17 : 18)) r->scratch_words = kRaggedScratchWords;  // two-pass configurations
  }
  if (e == cudaSuccess && r->ntasks > 0) {
    e = cudaMalloc(&r->d_tasks, tasks.size() * sizeof(RaggedTask));
    if (e == cudaSuccess)
      e = cudaMemcpy(r->d_tasks, tasks.data(), tasks.size() * sizeof(RaggedTask), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&r->d_head, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&r->d_ms, count);
    if (e == cudaSuccess) e = cudaMemcpy(r->d_ms, ms, count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&r->d_off, (count + 1) * sizeof(int64_t));
    if (e == cudaSuccess)
      e = cudaMemcpy(r->d_off, r->off.data(), (count + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess && r->scratch_words > 0) e = cudaMalloc(&r->d_scratch, r->scratch_words * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&r->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&r->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->join, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    *why = cudaGetErrorString(e);
    cudaGetLastError();
    free_plan(r);
    return nullptr;
  }
  if (tune && !r->groups.empty()) tune_groups(r);
  bool scratch = false;
  for (const RaggedGroup& g : r->groups) {
    r->launches += group_launches(g);
    scratch |= two_pass_opt(g.m, g.opt);
  }
  if (!scratch && r->d_scratch != nullptr) {  // no two-pass group after all
    cudaFree(r->d_scratch);
    r->d_scratch = nullptr;
    r->scratch_words = 0;
  }
  return r;
}

void ragged_destroy(RaggedPlan* r) { free_plan(r); }
int64_t ragged_total(const RaggedPlan* r) { return r->total; }
int ragged_passes(const RaggedPlan* r) { return r->scratch_words > 0 ? 2 : 1; }
int ragged_launches(const RaggedPlan* r) { return r->launches; }
bool ragged_tuned(const RaggedPlan* r) { return r->tuned; }
size_t ragged_workspace_bytes(const RaggedPlan* r) { return static_cast<size_t>(r->scratch_words) * sizeof(uint32_t); }
void ragged_offsets(const RaggedPlan* r, int64_t* out) { std::memcpy(out, r->off.data(), (r->count + 1) * sizeof(int64_t)); }

int ragged_run(RaggedPlan* r, const void* x, void* y, cudaStream_t st, std::string* why) {
  if (r->exec == nullptr || r->gx != x || r->gy != y) {
    if (r->exec) {
      cudaGraphExecDestroy(r->exec);
      r->exec = nullptr;
    }
    // Tensor maps need whole 32-word rows; without a batched launch (short signals only) the
    // map is never used and one row stands in for arrays shorter than 32 words.
    const bool tma = !r->groups.empty();
    CUtensorMap tx, ts;
    if (!encode_rows(&tx, x, tma ? r->total : 32) ||
        !encode_rows(&ts, r->d_scratch ? static_cast<const void*>(r->d_scratch) : x,
                     r->d_scratch ? r->scratch_words : (tma ? r->total : 32))) {
      *why = "cuTensorMapEncodeTiled failed";
      return 1;
    }
    RaggedArgs a{};
    a.tasks = r->d_tasks;
    a.ntasks = r->ntasks;
    a.queue_head = r->d_head;
    a.ms = r->d_ms;
    a.off = r->d_off;
    a.x = static_cast<const uint32_t*>(x);
    a.y = static_cast<uint32_t*>(y);
    a.total = r->total;
    a.checked = r->checked;
    a.status = r->d_status;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(r->cap, cudaStreamCaptureModeThreadLocal);
    cudaError_t le = cudaSuccess;
    if (e == cudaSuccess) {
      // Two branches: the two-pass groups, which share one scratch, one after another on
      // the capture stream; the short signals and the one-pass groups on the side stream.
      // Every launch writes its own signals only, so the branches may overlap on the GPU
      // (each branch's kernels fill the SMs the other's tails leave idle).
      if (cudaEventRecord(r->fork, r->cap) != cudaSuccess || cudaStreamWaitEvent(r->side, r->fork, 0) != cudaSuccess)
        le = cudaErrorUnknown;
      if (le == cudaSuccess && r->ntasks > 0) {
        cudaMemsetAsync(r->d_head, 0, sizeof(int32_t), r->side);
        switch (r->variant) {
          case kVarPerLevel: le = launch_ragged_small<kVarPerLevel>(a, r->side); break;
          case kVarEnd: le = launch_ragged_small<kVarEnd>(a, r->side); break;
          case kVarPlain: le = launch_ragged_small<kVarPlain>(a, r->side); break;
          default: le = launch_ragged_small<kVarI32>(a, r->side); break;
        }
      }
      for (const RaggedGroup& grp : r->groups)
        if (le == cudaSuccess && !two_pass_opt(grp.m, grp.opt)) le = launch_group(r, grp, grp.count, tx, ts, y, r->side);
      for (const RaggedGroup& grp : r->groups)
        if (le == cudaSuccess && two_pass_opt(grp.m, grp.opt)) le = launch_group(r, grp, grp.count, tx, ts, y, r->cap);
      if (cudaEventRecord(r->join, r->side) != cudaSuccess || cudaStreamWaitEvent(r->cap, r->join, 0) != cudaSuccess)
        if (le == cudaSuccess) le = cudaErrorUnknown;
      e = cudaStreamEndCapture(r->cap, &g);
      if (e == cudaSuccess && le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&r->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      *why = cudaGetErrorString(e);
      cudaGetLastError();
      return 1;
    }
    r->gx = x;
    r->gy = y;
  }
  const cudaError_t e = cudaGraphLaunch(r->exec, st);
  if (e != cudaSuccess) {
    *why = cudaGetErrorString(e);
    return 1;
  }
  return 0;
}

}  // namespace chw
