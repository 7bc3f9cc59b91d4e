// Launchers of the tensor-memory kernel's column tiles (tmem.cuh with CLO > 0): the second
// pass of the two-pass split y = H_b X^T H_a for column transforms of a = 10..14 bits,
// column blocks of 2^CLO columns x 2^a rows (2^15 or 2^16 words, one SM each), every
// butterfly variant.
#include "tmem_launch.cuh"

namespace chw {

namespace {

template <int M, int CLO>
TmemLaunchFn col_variant(int var) {
  switch (var) {
    case kVarPerLevel: return &launch_tmem_kernel<M, BfF32PerLevel, false, 0, CLO>;
    case kVarEnd: return &launch_tmem_kernel<M, BfF32Plain, true, 0, CLO>;
    case kVarPlain: return &launch_tmem_kernel<M, BfF32Plain, false, 0, CLO>;
    case kVarI32: return &launch_tmem_kernel<M, BfI32, false, 0, CLO>;
    default: return nullptr;
  }
}

}  // namespace

TmemLaunchFn lookup_tmem_col(int m, int clo, int var) {
  if (m == 15 && clo == 5) return col_variant<15, 5>(var);
  if (m != 16) return nullptr;
  switch (clo) {
    case 5: return col_variant<16, 5>(var);
    case 4: return col_variant<16, 4>(var);
    case 3: return col_variant<16, 3>(var);
    case 2: return col_variant<16, 2>(var);
    default: return nullptr;
  }
}

}  // namespace chw
