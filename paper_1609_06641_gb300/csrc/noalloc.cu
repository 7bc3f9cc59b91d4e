// chw_forward_noalloc: the two-pass transform with its intermediate in a fixed, statically
// allocated device array instead of a plan-owned cudaMalloc workspace.
//
// Some callers cannot allocate device memory at the point where they need the transform:
// processes whose device memory has been handed in full to another allocator (a caching
// pool that reserved it all), code that must not take cudaMalloc's implicit device-wide
// synchronisation (latency-critical loops), and code that runs where the CUDA runtime's
// allocator may not be called.  For them this entry point takes the sizes directly (no
// plan object, whose creation allocates) and keeps the pass-1 intermediate in
// `g_noalloc_scratch` below, a file-scope array that every GPU which loads this library
// holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/chw.h"

namespace chw {
chw_status_t two_pass_into(int m, int64_t batch, chw_dtype_t dtype, chw_norm_t norm, const void* x, void* y,
                           void* scratch, int* status, cudaStream_t st);
chw_status_t set_error(chw_status_t s, const char* msg);
void clear_error();
}  // namespace chw

namespace {

// 2^22 words (16 MiB) of pass-1 intermediate, plus 256 bytes of header (the device status
// word the kernels report bounded-wait timeouts into, cleared on every call).
constexpr int64_t kNoallocWords = int64_t{1} << 22;
constexpr int64_t kHeaderWords = 64;

__device__ __align__(256) uint32_t g_noalloc_scratch[kHeaderWords + kNoallocWords];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
uint32_t* g_scratch_ptr[kMaxDevices] = {};

// The device address of the array on the current device, looked up once per device with
// that device current (host code may not use the symbol itself as a device address).
chw_status_t scratch_on_current_device(uint32_t** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return chw::set_error(CHW_ERR_CUDA, "no current CUDA device");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return chw::set_error(CHW_ERR_CUDA, cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<uint32_t*>(p);
  }
  *out = g_scratch_ptr[dev];
  return CHW_OK;
}

}  // namespace

extern "C" chw_status_t chw_forward_noalloc(int m, int64_t batch, chw_dtype_t dtype, chw_norm_t norm, const void* x,
                                            void* y, void* stream) {
  chw::clear_error();
  if (m < 18 || m > 22) return chw::set_error(CHW_ERR_UNSUPPORTED, "chw_forward_noalloc takes 18 <= m <= 22");
  if (dtype != CHW_F32 && dtype != CHW_I32) return chw::set_error(CHW_ERR_UNSUPPORTED, "int32 or fp32 only");
  if (batch < 1) return chw::set_error(CHW_ERR_INVALID_ARG, "batch must be >= 1");
  if (batch > (kNoallocWords >> m))
    return chw::set_error(CHW_ERR_INVALID_ARG,
                          "batch * 2^m exceeds the static scratch of 2^22 elements (16 MiB) of chw_forward_noalloc");
  if (norm < CHW_NORM_NONE || norm > CHW_NORM_END) return chw::set_error(CHW_ERR_INVALID_ARG, "unknown norm");
  if (dtype == CHW_I32 && norm != CHW_NORM_NONE)
    return chw::set_error(CHW_ERR_INVALID_ARG, "int32 is unnormalised only (CHW_NORM_NONE)");
  if (x == nullptr || y == nullptr) return chw::set_error(CHW_ERR_INVALID_ARG, "x or y is NULL");
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) % 16 != 0)
    return chw::set_error(CHW_ERR_ALIGNMENT, "x and y must be 16-byte aligned");

  uint32_t* scratch = nullptr;
  chw_status_t r = scratch_on_current_device(&scratch);
  if (r != CHW_OK) return r;
  int* status = reinterpret_cast<int*>(scratch);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // The array keeps the previous call's contents: the status word must start at zero (the
  // intermediate is fully overwritten by pass 1 before pass 2 reads it).
  const cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e != cudaSuccess) return chw::set_error(CHW_ERR_CUDA, cudaGetErrorString(e));
  // The launches of a two-pass plan of the same shape (same split, same kernels).
  return chw::two_pass_into(m, batch, dtype, norm, x, y, scratch + kHeaderWords, status, st);
}

extern "C" chw_status_t chw_noalloc_device_status(void) {
  chw::clear_error();
  uint32_t* scratch = nullptr;
  chw_status_t r = scratch_on_current_device(&scratch);
  if (r != CHW_OK) return r;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return chw::set_error(CHW_ERR_CUDA, cudaGetErrorString(e));
  int s = 0;
  e = cudaMemcpy(&s, scratch, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(scratch, 0, sizeof(int));
  if (e != cudaSuccess) return chw::set_error(CHW_ERR_CUDA, cudaGetErrorString(e));
  if (s != 0) return chw::set_error(static_cast<chw_status_t>(s), "a chw_forward_noalloc launch latched a device error");
  return CHW_OK;
}
