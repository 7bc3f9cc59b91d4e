// Autotuner cache: the fastest measured configuration per (device, m, batch bucket, dtype,
// norm, order), kept per process and optionally in a text file.
#pragma once

#include <cstdint>
#include <string>

namespace chw {

struct TuneChoice {
  int tier;       // plan tier (api.cu): fused, cluster, two-pass, row-stack, tensor memory
  int row_bits;   // two-pass: bits of the first (row) pass; otherwise m
  int tile_bits;  // CTA tile of the fused and cluster kernels: 13 or 14; 0 where none applies
};

// Batch bucket of the cache key: floor(log2(batch)).
int tune_batch_bucket(int64_t batch);

// Cache key of a configuration (device name with spaces replaced).
std::string tune_key(const char* device, int m, int64_t batch, int dtype, int norm, int order);

// The process cache.  get returns false when the key has no entry.
bool tune_cache_get(const std::string& key, TuneChoice* out, float* us);
void tune_cache_put(const std::string& key, const TuneChoice& c, float us);
void tune_cache_clear();

// Text file of the cache, one entry per line:
//   chw-tune-v1 <key> tier=<t> row_bits=<b> tile_bits=<tb> us=<microseconds>
// load merges the file's well-formed lines into the process cache (others are skipped) and
// returns the number of entries read, or -1 if the file cannot be opened; save writes
// every entry and returns false on an I/O error.
int tune_cache_load(const char* path);
bool tune_cache_save(const char* path);

}  // namespace chw
