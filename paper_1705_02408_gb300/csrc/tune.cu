// Launch-shape table (host only): keys (dimension, floor(log2 V)), dimension 0
// for batches that mix dimensions.  Read on every batched build and search.
#include <map>
#include <mutex>
#include <utility>

#include "internal.h"

namespace mpap {

namespace {

std::mutex g_mu;
std::map<std::pair<int, uint32_t>, mpap_tuning>& table() {
  static std::map<std::pair<int, uint32_t>, mpap_tuning> t;
  return t;
}

uint32_t bucket_of(uint32_t V) {
  uint32_t b = 0;
  while (V > 1) {
    V >>= 1;
    ++b;
  }
  return b;
}

}  // namespace

mpap_tuning default_tuning() {
  mpap_tuning t;
  t.edge_warps = 8;
  t.wave_blocks_per_sm = 8;
  t.plan_lanes_from = 8;
  t.front_cap = 64;
  t.grid_merge_from = 2048;
  return t;
}

bool tuning_valid(const mpap_tuning& t) {
  return (t.edge_warps == 4 || t.edge_warps == 8) && t.wave_blocks_per_sm >= 1 && t.wave_blocks_per_sm <= 64 &&
         t.plan_lanes_from >= 1 && t.plan_lanes_from <= 64 && t.front_cap >= 1 &&
         t.grid_merge_from >= 33 && t.grid_merge_from <= (1u << 30);
}

mpap_tuning tuning_for(int dim, uint32_t V) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = table().find({dim, bucket_of(V)});
  return it == table().end() ? default_tuning() : it->second;
}

int32_t tuning_set(int dim, uint32_t V, const mpap_tuning& t) {
  if (!tuning_valid(t) || (dim != 0 && dim != 2 && dim != 3 && dim != 6)) {
    set_error("tuning: invalid shape or dimension");
    return MPAP_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  table()[{dim, bucket_of(V)}] = t;
  return MPAP_OK;
}

void tuning_clear() {
  std::lock_guard<std::mutex> lk(g_mu);
  table().clear();
}

int32_t tuning_export(uint32_t cap, int32_t* dims, uint32_t* buckets, mpap_tuning* t, uint32_t* n) {
  std::lock_guard<std::mutex> lk(g_mu);
  const uint32_t total = (uint32_t)table().size();
  *n = total;
  uint32_t i = 0;
  for (const auto& kv : table()) {
    if (i >= cap) break;
    if (dims) dims[i] = kv.first.first;
    if (buckets) buckets[i] = kv.first.second;
    if (t) t[i] = kv.second;
    ++i;
  }
  if (total > cap) {
    set_error("tuning_export: %u entries, cap %u", total, cap);
    return MPAP_ERR_INVALID_ARG;
  }
  return MPAP_OK;
}

}  // namespace mpap
