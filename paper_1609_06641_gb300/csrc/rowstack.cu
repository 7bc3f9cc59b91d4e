// Instantiations of the row-stack kernel (2^15..2^17-element signals) and their lookup.
#include "rowstack.cuh"

namespace chw {

using RowstackLaunchFn = cudaError_t (*)(const CUtensorMap*, const FusedArgs&, uint32_t*, int64_t, int64_t,
                                         cudaStream_t);

RowstackLaunchFn lookup_rowstack(int m, int var) {
#define CHW_ROWSTACK(M_)                                                        \
  if (m == M_) {                                                                \
    switch (var) {                                                              \
      case kVarPerLevel: return &launch_rowstack<M_, BfF32PerLevel, false>;     \
      case kVarEnd: return &launch_rowstack<M_, BfF32Plain, true>;              \
      case kVarPlain: return &launch_rowstack<M_, BfF32Plain, false>;           \
      case kVarI32: return &launch_rowstack<M_, BfI32, false>;                  \
      default: return nullptr;                                                  \
    }                                                                           \
  }
  CHW_ROWSTACK(15)
  CHW_ROWSTACK(16)
  CHW_ROWSTACK(17)
#undef CHW_ROWSTACK
  return nullptr;
}

}  // namespace chw
