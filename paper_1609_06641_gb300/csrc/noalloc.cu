// chw_forward_noalloc: the two-pass transform with its intermediate in a fixed, statically
// allocated device array instead of a plan-owned cudaMalloc workspace.
//
// Some callers cannot allocate device memory at the point where they need the transform:
// code running while a CUDA graph is being captured (cudaMalloc is not capturable), code
// whose process has handed all device memory to another allocator, and latency-sensitive
// callers that cannot afford cudaMalloc's implicit synchronisation.  For them this entry
// point takes the sizes directly (no plan object, whose creation allocates) and keeps the
// pass-1 intermediate in `g_noalloc_scratch` below, a file-scope array that every GPU
// which loads this library holds until the process exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/chw.h"
#include "launch.cuh"

namespace {

// 2^22 words (16 MiB) of pass-1 intermediate, plus 256 bytes of header (the device status
// word the kernels report bounded-wait timeouts into, cleared on every call).
constexpr int64_t kNoallocWords = int64_t{1} << 22;
constexpr int64_t kHeaderWords = 64;

__device__ __align__(256) uint32_t g_noalloc_scratch[kHeaderWords + kNoallocWords];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
uint32_t* g_scratch_ptr[kMaxDevices] = {};

thread_local char g_noalloc_err[256];

chw_status_t noalloc_fail(chw_status_t s, const char* msg) {
  std::snprintf(g_noalloc_err, sizeof(g_noalloc_err), "%s", msg);
  return s;
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

bool rows_map(CUtensorMap* map, const void* ptr, int64_t words, int tb) {
  auto enc = encoder();
  if (!enc) return false;
  const int boxr = (1 << (tb - 5)) < 256 ? (1 << (tb - 5)) : 256;
  cuuint64_t dims[2] = {32, static_cast<cuuint64_t>(words / 32)};
  cuuint64_t strides[1] = {128};
  cuuint32_t box[2] = {32, static_cast<cuuint32_t>(boxr)};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void*>(ptr), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

extern "C" chw_status_t chw_forward_noalloc(int m, int64_t batch, chw_dtype_t dtype, chw_norm_t norm, const void* x,
                                            void* y, void* stream) {
  g_noalloc_err[0] = '\0';
  if (m < 18 || m > 22) return noalloc_fail(CHW_ERR_UNSUPPORTED, "chw_forward_noalloc takes 18 <= m <= 22");
  if (batch < 1) return noalloc_fail(CHW_ERR_INVALID_ARG, "batch must be >= 1");
  if (batch > (kNoallocWords >> m))
    return noalloc_fail(CHW_ERR_INVALID_ARG,
                        "batch * 2^m exceeds the static scratch of 2^22 elements (16 MiB) of chw_forward_noalloc");
  if (dtype != CHW_F32 && dtype != CHW_I32) return noalloc_fail(CHW_ERR_UNSUPPORTED, "int32 or fp32 only");
  if (norm < CHW_NORM_NONE || norm > CHW_NORM_END) return noalloc_fail(CHW_ERR_INVALID_ARG, "unknown norm");
  if (dtype == CHW_I32 && norm != CHW_NORM_NONE) return noalloc_fail(CHW_ERR_INVALID_ARG, "int32 is unnormalised only");
  if (x == nullptr || y == nullptr) return noalloc_fail(CHW_ERR_INVALID_ARG, "x or y is NULL");
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) % 16 != 0)
    return noalloc_fail(CHW_ERR_ALIGNMENT, "x and y must be 16-byte aligned");

  // Set-up, once per device, with that device current: the device address of the array.
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(CHW_ERR_CUDA, "no current CUDA device");
  uint32_t* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_scratch_ptr[dev] == nullptr) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return noalloc_fail(CHW_ERR_CUDA, cudaGetErrorString(e));
      g_scratch_ptr[dev] = static_cast<uint32_t*>(p);
    }
    scratch = g_scratch_ptr[dev];
  }
  int* status = reinterpret_cast<int*>(scratch);
  uint32_t* inter = scratch + kHeaderWords;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  // The same split as a two-pass plan: a = max(6, m - 17) column bits, b = m - a row bits.
  const int a = (m - 17) > 6 ? (m - 17) : 6;
  const int b = m - a;
  const int64_t total = batch << m;
  const bool end = dtype == CHW_F32 && norm == CHW_NORM_END;
  int var1, var2;
  if (dtype == CHW_I32) {
    var1 = var2 = chw::kVarI32;
  } else if (norm == CHW_NORM_PER_LEVEL) {
    var1 = var2 = chw::kVarPerLevel;
  } else {
    var1 = chw::kVarPlain;
    var2 = end ? chw::kVarEnd : chw::kVarPlain;
  }
  const int tb1 = b <= 13 ? 13 : 14, cb1 = b <= 14 ? 0 : b - 14;
  const int tb2 = a <= 8 ? 13 : 14, cb2 = a <= 9 ? 0 : a - 9;
  chw::FusedLaunchFn f1 = chw::lookup_fused(0, b, tb1, cb1, var1, 1);
  chw::FusedLaunchFn f2 = chw::lookup_fused(5, a, tb2, cb2, var2, 0);
  if (!f1 || !f2) return noalloc_fail(CHW_ERR_UNSUPPORTED, "no two-pass kernels for this m");
  CUtensorMap m1, m2;
  if (!rows_map(&m1, x, total, tb1) || !rows_map(&m2, inter, total, tb2))
    return noalloc_fail(CHW_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  // The array keeps the previous call's contents: the status word must start at zero (the
  // intermediate is fully overwritten by pass 1).
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return noalloc_fail(CHW_ERR_CUDA, "status reset failed");

  chw::FusedArgs p1{};
  p1.out = inter;
  p1.out_total = total;
  p1.end_scale = 1.0f;
  p1.diag_mask = (int64_t{1} << m) - 1;
  p1.status = status;
  p1.colblock_a = a;
  const int64_t u1 = cb1 > 0 ? total >> (tb1 + cb1) : (total + (int64_t{1} << tb1) - 1) >> tb1;
  cudaError_t e = f1(&m1, p1, u1, st);
  if (e != cudaSuccess) return noalloc_fail(CHW_ERR_CUDA, cudaGetErrorString(e));

  chw::FusedArgs p2{};
  p2.out = y;
  p2.out_total = total;
  {
    const float r = (m & 1) ? 0.70710678118654752440f : 1.0f;
    p2.end_scale = std::ldexp(r, -(m / 2));
  }
  p2.diag_mask = (int64_t{1} << m) - 1;
  p2.status = status;
  const int64_t u2 = cb2 > 0 ? total >> (tb2 + cb2) : (total + (int64_t{1} << tb2) - 1) >> tb2;
  e = f2(&m2, p2, u2, st);
  if (e != cudaSuccess) return noalloc_fail(CHW_ERR_CUDA, cudaGetErrorString(e));
  return CHW_OK;
}
