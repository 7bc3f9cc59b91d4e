// Ragged batches: many signals of uneven length 2^{m_i} (0 <= m_i <= 20), transformed by
// one CUDA graph launch.  The plan sorts the signals by length once and records, for each
// length present, the launch that suits it:
//   m <= 12   one persistent kernel over a work list of runs of consecutive short signals
//             (plain shared-memory cascade per signal);
//   m = 13,14 the batched single-CTA fused kernel, one unit per signal, reading and
//             writing every signal at its own offset (offset table on the device);
//   m = 15-17 the batched cluster kernel, likewise;
//   m = 18-20 the two-pass split y = H_b X^T H_a with a = 9: the first pass reads the
//             signals at their offsets into plan-owned scratch, the second writes them
//             back at their offsets, in chunks of signals that fit the scratch.
// A tuned plan times each length's alternatives when it is made (tile size for 2^15, 2^16;
// cluster or two passes for 2^17; a = 8, 9 or 10 for 2^18..2^20) and keeps the fastest.
// The graph is recorded per pair of x/y pointers and replayed by every call with them.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "launch.cuh"

namespace chw {

constexpr int kRaggedMaxM = 20;
constexpr int kRaggedSmallMaxM = 12;       // longer signals go to the batched launches
constexpr int kSmallGroupWords = 1 << 15;  // a small-signal task covers up to 128 KiB
constexpr int64_t kRaggedScratchWords = int64_t{1} << 26;  // two-pass scratch (256 MiB)

struct RaggedTask {
  int32_t index;  // first signal of the run
  int32_t count;  // signals in the run
};

struct RaggedArgs {
  const RaggedTask* tasks;
  int32_t ntasks;
  int32_t* queue_head;  // zeroed before each run
  const uint8_t* ms;
  const int64_t* off;
  const uint32_t* x;
  uint32_t* y;
  int64_t total;  // elements of x and y (checked mode: each signal must lie inside)
  int checked;    // CHW_FLAG_CHECKED
  int* status;
};

struct RaggedPlan;
// `tune`: time each length group's configurations (tile size, cluster or two passes, the
// two-pass split) on temporary arrays of the plan's size and keep the fastest.
RaggedPlan* ragged_create(const uint8_t* ms, int64_t count, int variant, int* d_status, bool tune, std::string* why);
// The library's packing of `count` signals: offsets[i] (count + 1 entries, the last one the
// total), each signal starting on a 32-element (128-byte) boundary.
// Start alignment (elements) of a signal of 2^m words in the library's packing: a whole
// output run of the tensor-memory kernels, 2^(m-8), for m = 15..17; 32 (128 bytes) else.
int64_t ragged_align(int m);
void ragged_pack(const uint8_t* ms, int64_t count, int64_t* offsets);
// The same over caller-chosen offsets (elements of x and y; `total` = their length): signals
// with m >= 13 must start on a 32-element boundary, shorter ones anywhere.  `checked`: the
// kernels range-check every offset they use (CHW_FLAG_CHECKED).
RaggedPlan* ragged_create_at(const uint8_t* ms, const int64_t* offsets, int64_t count, int64_t total, int variant,
                             int* d_status, bool tune, std::string* why, bool checked = false);
void ragged_destroy(RaggedPlan* r);
int64_t ragged_total(const RaggedPlan* r);
int ragged_passes(const RaggedPlan* r);
int ragged_launches(const RaggedPlan* r);
bool ragged_tuned(const RaggedPlan* r);
size_t ragged_workspace_bytes(const RaggedPlan* r);
void ragged_offsets(const RaggedPlan* r, int64_t* out);
int ragged_run(RaggedPlan* r, const void* x, void* y, cudaStream_t st, std::string* why);

}  // namespace chw
