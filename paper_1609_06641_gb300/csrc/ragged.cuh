// Ragged batches: many signals of uneven length 2^{m_i} (0 <= m_i <= 20) in one
// persistent launch over a device work queue, replayed from a CUDA graph.
//
// Tasks (built once per plan on the host, in this order of priority):
//   ROW   first pass of a signal with m >= 15: one 2^14-word row (row transform, H_14)
//         into a ring slot of scratch, column-blocked (see fused.cuh, OUTMODE 1);
//   COL   second pass of such a signal: one 2^14-word tile of 32-column blocks
//         (column transform over the 2^(m-14) rows), written to y;
//   TILE  a signal with m = 14: one fused tile;
//   SMALL a run of consecutive signals with m <= 13: plain shared-memory cascade.
// A COL task waits until every ROW task of its signal has finished; a ROW task of the k-th
// two-pass signal reuses ring slot k mod kRingSlots and waits until the COL tasks of signal
// k - kRingSlots are done.  Tasks only wait on tasks earlier in the queue, which running
// CTAs have already taken, so the schedule always progresses; every wait is bounded and
// reports CHW_ERR_TIMEOUT through the status word if it gives up.  The small ring keeps
// the intermediate in L2 most of the time.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "launch.cuh"

namespace chw {

constexpr int kRaggedMaxM = 20;
constexpr int kRaggedTileBits = 14;
constexpr int kRingSlots = 16;
constexpr int64_t kRingSlotWords = int64_t{1} << kRaggedMaxM;
constexpr int kSmallGroupWords = 1 << 15;  // a SMALL task covers up to 128 KiB of signals

enum RaggedTaskKind : int32_t { kTaskSmall = 0, kTaskTile = 1, kTaskRow = 2, kTaskCol = 3 };

struct RaggedTask {
  int32_t kind;
  int32_t m;
  int64_t off;       // element offset of the signal (SMALL: of its first signal)
  int32_t index;     // ROW: row, COL: tile, SMALL: first signal
  int32_t count;     // SMALL: number of signals
  int32_t slot;      // ROW/COL: ring slot
  int32_t wait_on;   // counter index to wait on, or -1
  int32_t wait_val;  // value the counter must reach
  int32_t done_ctr;  // counter index to increment when done, or -1
};

struct RaggedArgs {
  const RaggedTask* tasks;
  int32_t ntasks;
  int32_t* queue_head;  // zeroed before each run
  int32_t* ctr;         // zeroed before each run
  const uint8_t* ms;
  const int64_t* off;
  const uint32_t* x;
  uint32_t* y;
  uint32_t* ring;
  int64_t total;
  int* status;
};

struct RaggedPlan;
RaggedPlan* ragged_create(const uint8_t* ms, int64_t count, int variant, int* d_status, std::string* why);
// The same over caller-chosen offsets (elements of x and y; `total` = their length): signals
// with m >= 14 must start on a 32-element boundary, shorter ones anywhere.
RaggedPlan* ragged_create_at(const uint8_t* ms, const int64_t* offsets, int64_t count, int64_t total, int variant,
                             int* d_status, std::string* why);
void ragged_destroy(RaggedPlan* r);
int64_t ragged_total(const RaggedPlan* r);
int ragged_passes(const RaggedPlan* r);
size_t ragged_workspace_bytes(const RaggedPlan* r);
void ragged_offsets(const RaggedPlan* r, int64_t* out);
int ragged_run(RaggedPlan* r, const void* x, void* y, cudaStream_t st, std::string* why);

}  // namespace chw
