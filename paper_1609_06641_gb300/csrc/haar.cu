// Launchers of the Haar analysis and synthesis passes (see haar.cuh).
#include <cudaTypedefs.h>

#include "haar.cuh"
#include "launch.cuh"

namespace chw {

namespace {

// `words` 4-byte words at `ptr` as rows of 32 words, boxes of 256 rows (one 2^13 row of
// the Haar passes), SWIZZLE_128B.
bool haar_rows_map(CUtensorMap* map, const void* ptr, int64_t words) {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
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

template <class BF, bool END>
cudaError_t fwd_rows(const HaarFwdArgs& a, cudaStream_t st) {
  CUtensorMap map;
  if (!haar_rows_map(&map, a.in, a.rows << kHaarRowBits)) return cudaErrorInvalidValue;
  haar_fwd_row_kernel<BF, END><<<static_cast<unsigned>(a.rows), kHaarThreads, 0, st>>>(map, a);
  return cudaGetLastError();
}

template <class BF, bool END>
cudaError_t inv_rows(const HaarInvArgs& a, cudaStream_t st) {
  CUtensorMap map;
  if (!haar_rows_map(&map, a.out, a.rows << kHaarRowBits)) return cudaErrorInvalidValue;
  haar_inv_row_kernel<BF, END><<<static_cast<unsigned>(a.rows), kHaarThreads, 0, st>>>(map, a);
  return cudaGetLastError();
}

template <class BF, bool END>
cudaError_t fwd_pass(const HaarFwdArgs& a, cudaStream_t st) {
  if (a.tc == kHaarRowBits) return fwd_rows<BF, END>(a, st);
  const int64_t per_cta = int64_t{1} << (kHaarRowBits - a.tc);
  const int64_t grid = (a.rows + per_cta - 1) / per_cta;
  haar_fwd_kernel<BF, END><<<static_cast<unsigned>(grid), kHaarThreads, 0, st>>>(a);
  return cudaGetLastError();
}

template <class BF, bool END>
cudaError_t inv_pass(const HaarInvArgs& a, cudaStream_t st) {
  if (a.tc == kHaarRowBits) return inv_rows<BF, END>(a, st);
  const int64_t per_cta = int64_t{1} << (kHaarRowBits - a.tc);
  const int64_t grid = (a.rows + per_cta - 1) / per_cta;
  haar_inv_kernel<BF, END><<<static_cast<unsigned>(grid), kHaarThreads, 0, st>>>(a);
  return cudaGetLastError();
}

// Passes of a 2^m transform: pass p covers levels 13p+1 .. 13p+tc_p.
int haar_passes(int m) { return m == 0 ? 1 : (m + kHaarRowBits - 1) / kHaarRowBits; }

}  // namespace

// Words of scratch the Haar passes need for `batch` signals of 2^m elements: the row
// approximations between passes (2^{m-13} per signal, then 2^{m-26}).
int64_t haar_scratch_words(int m, int64_t batch) {
  int64_t w = 0;
  for (int p = 1; p < haar_passes(m); ++p) w += batch << (m - kHaarRowBits * p);
  return w;
}

// z = Psi_m x for `batch` signals (variant: kVarPerLevel, kVarEnd, kVarPlain, kVarI32).
cudaError_t haar_forward(int var, int m, int64_t batch, const void* x, void* z, uint32_t* scratch, int* status,
                         cudaStream_t st) {
  const int P = haar_passes(m);
  uint32_t* approx[4] = {};
  int64_t off = 0;
  for (int p = 1; p < P; ++p) {
    approx[p] = scratch + off;
    off += batch << (m - kHaarRowBits * p);
  }
  for (int p = 0; p < P; ++p) {
    HaarFwdArgs a{};
    a.mlen = m - kHaarRowBits * p;
    a.tc = a.mlen < kHaarRowBits ? a.mlen : kHaarRowBits;
    a.lev0 = kHaarRowBits * p;
    a.mtotal = m;
    a.in = p == 0 ? static_cast<const uint32_t*>(x) : approx[p];
    a.out = static_cast<uint32_t*>(z);
    a.out_stride = int64_t{1} << m;
    a.approx = p + 1 < P ? approx[p + 1] : nullptr;
    a.rows = batch << (a.mlen - a.tc);
    a.status = status;
    cudaError_t e = cudaSuccess;
    switch (var) {
      case kVarPerLevel: e = fwd_pass<BfF32PerLevel, false>(a, st); break;
      case kVarEnd: e = fwd_pass<BfF32Plain, true>(a, st); break;
      case kVarPlain: e = fwd_pass<BfF32Plain, false>(a, st); break;
      default: e = fwd_pass<BfI32, false>(a, st); break;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// x = Psi_m^T z, coarse pass first.
cudaError_t haar_inverse(int var, int m, int64_t batch, const void* z, void* x, uint32_t* scratch, cudaStream_t st) {
  const int P = haar_passes(m);
  uint32_t* approx[4] = {};
  int64_t off = 0;
  for (int p = 1; p < P; ++p) {
    approx[p] = scratch + off;
    off += batch << (m - kHaarRowBits * p);
  }
  for (int p = P - 1; p >= 0; --p) {
    HaarInvArgs a{};
    a.mlen = m - kHaarRowBits * p;
    a.tc = a.mlen < kHaarRowBits ? a.mlen : kHaarRowBits;
    a.lev0 = kHaarRowBits * p;
    a.mtotal = m;
    a.z = static_cast<const uint32_t*>(z);
    a.z_stride = int64_t{1} << m;
    a.approx = p + 1 < P ? approx[p + 1] : nullptr;
    a.out = p == 0 ? static_cast<uint32_t*>(x) : approx[p];
    a.rows = batch << (a.mlen - a.tc);
    cudaError_t e = cudaSuccess;
    switch (var) {
      case kVarPerLevel: e = inv_pass<BfF32PerLevel, false>(a, st); break;
      case kVarEnd: e = inv_pass<BfF32Plain, true>(a, st); break;
      case kVarPlain: e = inv_pass<BfF32Plain, false>(a, st); break;
      default: e = inv_pass<BfI32, false>(a, st); break;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace chw
