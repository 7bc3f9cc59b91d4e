// The column-blocked scratch of a two-pass split y = H_b X^T H_a (Theorem 1 applied to the
// 2^a x 2^M matrix of a signal), as the 5-D tensor view through which the tensor-memory
// row kernel writes it with TMA stores.  Host code: the plan encodes this view, and the
// host-side layout check walks it against the kernel's staging.
#pragma once

#include <cuda.h>

#include <cstdint>

namespace chw {

struct ColblockView {
  cuuint64_t dims[5];     // {2^c words, row r, block g mod 2^(M-8-c), run g >> (M-8-c), signal}
  cuuint64_t strides[4];  // bytes, of dims 1..4
  cuuint32_t box[5];      // {2^c words, 1 row, 2^(5-c) blocks, 256 runs, 1 signal}
  CUtensorMapSwizzle swizzle;
};

// `total` words of rows of 2^M words, 2^a rows per signal, blocks of 2^c columns (c = 2..5):
// element k of row r of signal s at s 2^(a+M) + (k >> c) 2^(a+c) + 2^c r + (k mod 2^c).
// A box row is 2^c words (16..128 bytes); shared memory holds it densely only when the
// swizzle span equals that width (a narrower row would take a whole span), so the swizzle
// is 128, 64 or 32 bytes for c = 5, 4, 3 and none for c = 2: one box is 256 runs of 128
// bytes, 32 KB.
constexpr ColblockView colblock_view(int64_t total, int M, int a, int c) {
  const cuuint64_t w = 4;
  ColblockView v{};
  v.dims[0] = cuuint64_t{1} << c;
  v.dims[1] = cuuint64_t{1} << a;
  v.dims[2] = cuuint64_t{1} << (M - 8 - c);
  v.dims[3] = 256;
  v.dims[4] = static_cast<cuuint64_t>(total >> (a + M));
  v.strides[0] = w << c;
  v.strides[1] = w << (a + c);
  v.strides[2] = w << (a + M - 8);
  v.strides[3] = w << (a + M);
  v.box[0] = 1u << c;
  v.box[1] = 1;
  v.box[2] = 1u << (5 - c);
  v.box[3] = 256;
  v.box[4] = 1;
  v.swizzle = c == 5   ? CU_TENSOR_MAP_SWIZZLE_128B
              : c == 4 ? CU_TENSOR_MAP_SWIZZLE_64B
              : c == 3 ? CU_TENSOR_MAP_SWIZZLE_32B
                       : CU_TENSOR_MAP_SWIZZLE_NONE;
  return v;
}

}  // namespace chw
