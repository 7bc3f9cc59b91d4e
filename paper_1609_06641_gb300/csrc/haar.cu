// Launchers of the Haar analysis and synthesis passes (see haar.cuh).
#include "haar.cuh"
#include "launch.cuh"

namespace chw {

namespace {

template <class BF, bool END>
cudaError_t fwd_pass(const HaarFwdArgs& a, cudaStream_t st) {
  const int64_t per_cta = int64_t{1} << (kHaarRowBits - a.tc);
  const int64_t grid = (a.rows + per_cta - 1) / per_cta;
  haar_fwd_kernel<BF, END><<<static_cast<unsigned>(grid), kHaarThreads, 0, st>>>(a);
  return cudaGetLastError();
}

template <class BF, bool END>
cudaError_t inv_pass(const HaarInvArgs& a, cudaStream_t st) {
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
cudaError_t haar_forward(int var, int m, int64_t batch, const void* x, void* z, uint32_t* scratch, cudaStream_t st) {
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
