// Autotuner cache (see tune.h).  Host code only.
#include "tune.h"

#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>

namespace chw {

namespace {

struct Entry {
  TuneChoice c;
  float us;
};

std::mutex g_mu;
std::map<std::string, Entry>& cache() {
  static std::map<std::string, Entry> m;
  return m;
}

}  // namespace

int tune_batch_bucket(int64_t batch) {
  int b = 0;
  while (batch > 1) {
    batch >>= 1;
    ++b;
  }
  return b;
}

std::string tune_key(const char* device, int m, int64_t batch, int dtype, int norm, int order) {
  std::string dev = device != nullptr ? device : "unknown";
  for (char& ch : dev)
    if (ch == ' ' || ch == '\t' || ch == '\n' || ch == '=') ch = '_';
  if (dev.empty()) dev = "unknown";
  char buf[160];
  std::snprintf(buf, sizeof(buf), "%s:m%d:bb%d:dt%d:nm%d:or%d", dev.c_str(), m, tune_batch_bucket(batch), dtype,
                norm, order);
  return buf;
}

bool tune_cache_get(const std::string& key, TuneChoice* out, float* us) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = cache().find(key);
  if (it == cache().end()) return false;
  if (out) *out = it->second.c;
  if (us) *us = it->second.us;
  return true;
}

void tune_cache_put(const std::string& key, const TuneChoice& c, float us) {
  std::lock_guard<std::mutex> lk(g_mu);
  cache()[key] = Entry{c, us};
}

void tune_cache_clear() {
  std::lock_guard<std::mutex> lk(g_mu);
  cache().clear();
}

int tune_cache_load(const char* path) {
  if (path == nullptr) return -1;
  FILE* f = std::fopen(path, "r");
  if (!f) return -1;
  int n = 0;
  char line[512];
  while (std::fgets(line, sizeof(line), f)) {
    char key[256];
    TuneChoice c{};
    float us = 0.f;
    if (std::sscanf(line, "chw-tune-v1 %255s tier=%d row_bits=%d tile_bits=%d us=%f", key, &c.tier, &c.row_bits,
                    &c.tile_bits, &us) != 5)
      continue;
    if (c.tier < 0 || c.row_bits < 0 || c.row_bits > 30 || (c.tile_bits != 0 && c.tile_bits != 13 && c.tile_bits != 14))
      continue;
    tune_cache_put(key, c, us);
    ++n;
  }
  std::fclose(f);
  return n;
}

bool tune_cache_save(const char* path) {
  if (path == nullptr) return false;
  std::map<std::string, Entry> snap;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    snap = cache();
  }
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return false;
  bool ok = true;
  for (const auto& kv : snap)
    ok &= std::fprintf(f, "chw-tune-v1 %s tier=%d row_bits=%d tile_bits=%d us=%.3f\n", kv.first.c_str(),
                       kv.second.c.tier, kv.second.c.row_bits, kv.second.c.tile_bits, kv.second.us) > 0;
  ok &= std::fclose(f) == 0;
  if (!ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return false;
  }
  return true;
}

}  // namespace chw
