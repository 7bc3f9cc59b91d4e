// Host side of ragged plans: packing, task table, graph capture (see ragged.cuh).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "ragged_kernel.cuh"

namespace chw {

// One translation unit per variant instantiates the kernel (generated by the build).
extern template cudaError_t launch_ragged<kVarPerLevel>(const CUtensorMap&, const CUtensorMap&, const RaggedArgs&, cudaStream_t);
extern template cudaError_t launch_ragged<kVarEnd>(const CUtensorMap&, const CUtensorMap&, const RaggedArgs&, cudaStream_t);
extern template cudaError_t launch_ragged<kVarPlain>(const CUtensorMap&, const CUtensorMap&, const RaggedArgs&, cudaStream_t);
extern template cudaError_t launch_ragged<kVarI32>(const CUtensorMap&, const CUtensorMap&, const RaggedArgs&, cudaStream_t);

// ------------------------------------------------------------------ host side
struct RaggedPlan {
  int64_t count = 0;
  std::vector<uint8_t> ms;
  std::vector<int64_t> off;  // count + 1 entries
  int64_t total = 0;
  int64_t map_words = 0;  // extent of the input tensor map
  int variant = 0;
  int* d_status = nullptr;
  int ntasks = 0;
  int nctr = 0;
  int nbig = 0;
  RaggedTask* d_tasks = nullptr;
  int32_t* d_ctrs = nullptr;  // [0] queue head, [1..] dependency counters
  uint8_t* d_ms = nullptr;
  int64_t* d_off = nullptr;
  uint32_t* d_ring = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  const void* gx = nullptr;
  void* gy = nullptr;
};

namespace {

void free_plan(RaggedPlan* r) {
  if (r->exec) cudaGraphExecDestroy(r->exec);
  if (r->cap) cudaStreamDestroy(r->cap);
  cudaFree(r->d_tasks);
  cudaFree(r->d_ctrs);
  cudaFree(r->d_ms);
  cudaFree(r->d_off);
  cudaFree(r->d_ring);
  delete r;
}

bool encode_rows(CUtensorMap* map, const void* ptr, int64_t words) {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  if (!enc) return false;
  cuuint64_t dims[2] = {32, static_cast<cuuint64_t>(words / 32)};
  cuuint64_t strides[1] = {128};
  cuuint32_t box[2] = {32, 256};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void*>(ptr), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

RaggedPlan* ragged_create(const uint8_t* ms, int64_t count, int variant, int* d_status, std::string* why) {
  std::vector<int64_t> off(count + 1);
  int64_t o = 0;
  for (int64_t i = 0; i < count; ++i) {
    off[i] = o;
    o += int64_t{1} << ms[i];
    o = (o + 31) & ~int64_t{31};  // every signal starts on a 128-byte boundary
  }
  off[count] = o;
  return ragged_create_at(ms, off.data(), count, o, variant, d_status, why);
}

RaggedPlan* ragged_create_at(const uint8_t* ms, const int64_t* offsets, int64_t count, int64_t total, int variant,
                             int* d_status, std::string* why) {
  auto* r = new RaggedPlan();
  r->count = count;
  r->ms.assign(ms, ms + count);
  r->off.assign(offsets, offsets + count);
  r->off.push_back(total);
  r->variant = variant;
  r->d_status = d_status;
  r->total = total;

  // ---- task table
  std::vector<RaggedTask> tasks;
  std::vector<int64_t> big;
  for (int64_t i = 0; i < count; ++i)
    if (ms[i] > kRaggedTileBits) big.push_back(i);
  std::stable_sort(big.begin(), big.end(), [&](int64_t a, int64_t b) { return ms[a] > ms[b]; });
  r->nbig = static_cast<int>(big.size());
  auto parts = [&](int64_t sig) { return 1 << (ms[sig] - kRaggedTileBits); };
  auto emit_rows = [&](int k) {
    const int64_t s = big[k];
    for (int j = 0; j < parts(s); ++j) {
      RaggedTask t{};
      t.kind = kTaskRow;
      t.m = ms[s];
      t.off = r->off[s];
      t.index = j;
      t.slot = k % kRingSlots;
      t.wait_on = k >= kRingSlots ? 1 + 2 * (k - kRingSlots) + 1 : -1;
      t.wait_val = k >= kRingSlots ? parts(big[k - kRingSlots]) : 0;
      t.done_ctr = 1 + 2 * k;
      tasks.push_back(t);
    }
  };
  auto emit_cols = [&](int k) {
    const int64_t s = big[k];
    for (int j = 0; j < parts(s); ++j) {
      RaggedTask t{};
      t.kind = kTaskCol;
      t.m = ms[s];
      t.off = r->off[s];
      t.index = j;
      t.slot = k % kRingSlots;
      t.wait_on = 1 + 2 * k;
      t.wait_val = parts(s);
      t.done_ctr = 1 + 2 * k + 1;
      tasks.push_back(t);
    }
  };
  for (int k = 0; k < r->nbig; ++k) {
    emit_rows(k);
    if (k >= 1) emit_cols(k - 1);
  }
  if (r->nbig > 0) emit_cols(r->nbig - 1);
  for (int64_t i = 0; i < count; ++i) {
    if (ms[i] != kRaggedTileBits) continue;
    RaggedTask t{};
    t.kind = kTaskTile;
    t.m = ms[i];
    t.off = r->off[i];
    t.wait_on = -1;
    t.done_ctr = -1;
    tasks.push_back(t);
  }
  for (int64_t i = 0; i < count;) {
    if (ms[i] >= kRaggedTileBits) {
      ++i;
      continue;
    }
    RaggedTask t{};
    t.kind = kTaskSmall;
    t.index = static_cast<int32_t>(i);
    t.wait_on = -1;
    t.done_ctr = -1;
    int64_t words = 0;
    while (i < count && ms[i] < kRaggedTileBits && words < kSmallGroupWords) {
      words += int64_t{1} << ms[i];
      ++i;
      ++t.count;
    }
    tasks.push_back(t);
  }
  r->ntasks = static_cast<int>(tasks.size());
  r->nctr = 1 + 2 * r->nbig;
  // TILE/ROW/COL tasks read x through a tensor map of whole 32-word rows; without them the
  // map is never used and one row stands in for arrays shorter than 32 words.
  bool tma = false;
  for (const RaggedTask& t : tasks) tma |= t.kind != kTaskSmall;
  r->map_words = tma ? r->total : 32;

  cudaError_t e = cudaMalloc(&r->d_tasks, std::max<size_t>(1, tasks.size()) * sizeof(RaggedTask));
  if (e == cudaSuccess && !tasks.empty())
    e = cudaMemcpy(r->d_tasks, tasks.data(), tasks.size() * sizeof(RaggedTask), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&r->d_ctrs, r->nctr * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&r->d_ms, count);
  if (e == cudaSuccess) e = cudaMemcpy(r->d_ms, ms, count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&r->d_off, (count + 1) * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMemcpy(r->d_off, r->off.data(), (count + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && r->nbig > 0) e = cudaMalloc(&r->d_ring, kRingSlots * kRingSlotWords * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&r->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    *why = cudaGetErrorString(e);
    cudaGetLastError();
    free_plan(r);
    return nullptr;
  }
  return r;
}

void ragged_destroy(RaggedPlan* r) { free_plan(r); }
int64_t ragged_total(const RaggedPlan* r) { return r->total; }
int ragged_passes(const RaggedPlan* r) { return r->nbig > 0 ? 2 : 1; }
size_t ragged_workspace_bytes(const RaggedPlan* r) {
  return r->nbig > 0 ? kRingSlots * kRingSlotWords * sizeof(uint32_t) : 0;
}
void ragged_offsets(const RaggedPlan* r, int64_t* out) { std::memcpy(out, r->off.data(), (r->count + 1) * sizeof(int64_t)); }

int ragged_run(RaggedPlan* r, const void* x, void* y, cudaStream_t st, std::string* why) {
  if (r->exec == nullptr || r->gx != x || r->gy != y) {
    if (r->exec) {
      cudaGraphExecDestroy(r->exec);
      r->exec = nullptr;
    }
    CUtensorMap tx, tr;
    if (!encode_rows(&tx, x, r->map_words) ||
        !encode_rows(&tr, r->d_ring ? static_cast<const void*>(r->d_ring) : x,
                     r->d_ring ? kRingSlots * kRingSlotWords : r->map_words)) {
      *why = "cuTensorMapEncodeTiled failed";
      return 1;
    }
    RaggedArgs a{};
    a.tasks = r->d_tasks;
    a.ntasks = r->ntasks;
    a.queue_head = r->d_ctrs;
    a.ctr = r->d_ctrs;
    a.ms = r->d_ms;
    a.off = r->d_off;
    a.x = static_cast<const uint32_t*>(x);
    a.y = static_cast<uint32_t*>(y);
    a.ring = r->d_ring;
    a.total = r->total;
    a.status = r->d_status;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(r->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaMemsetAsync(r->d_ctrs, 0, r->nctr * sizeof(int32_t), r->cap);
      switch (r->variant) {
        case kVarPerLevel: launch_ragged<kVarPerLevel>(tx, tr, a, r->cap); break;
        case kVarEnd: launch_ragged<kVarEnd>(tx, tr, a, r->cap); break;
        case kVarPlain: launch_ragged<kVarPlain>(tx, tr, a, r->cap); break;
        default: launch_ragged<kVarI32>(tx, tr, a, r->cap); break;
      }
      e = cudaStreamEndCapture(r->cap, &g);
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
