// Kernel launch accounting and optional per-kernel timing.
//
// Every kernel launch of the library goes through a LaunchScope, which counts
// the launch and, when timing is enabled, brackets it with two CUDA events on
// the launching stream.  mpap_profile_read() waits for the recorded events and
// returns per-kernel launch counts and total device milliseconds.
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "profile.h"

namespace mpap {

namespace {

struct Pending {
  const char* name;
  cudaEvent_t a, b;
};

struct Agg {
  uint64_t launches = 0;
  double ms = 0.0;
};

struct Profiler {
  std::mutex mu;
  std::atomic<bool> on{false};
  std::atomic<uint64_t> launches{0};
  std::vector<cudaEvent_t> pool;
  std::vector<Pending> pending;
  std::map<std::string, Agg> agg;

  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void drain() {
    for (auto& p : pending) {
      cudaEventSynchronize(p.b);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, p.a, p.b);
      Agg& a = agg[p.name];
      a.launches += 1;
      a.ms += ms;
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
};

Profiler& prof() {
  static Profiler* p = new Profiler();
  return *p;
}

}  // namespace

LaunchScope::LaunchScope(cudaStream_t st, const char* name) : st_(st), name_(name) {
  Profiler& p = prof();
  p.launches.fetch_add(1, std::memory_order_relaxed);
  if (p.on.load(std::memory_order_relaxed)) {
    std::lock_guard<std::mutex> g(p.mu);
    a_ = p.get();
    b_ = p.get();
    cudaEventRecord(a_, st_);
  }
}

LaunchScope::~LaunchScope() {
  if (a_) {
    Profiler& p = prof();
    cudaEventRecord(b_, st_);
    std::lock_guard<std::mutex> g(p.mu);
    p.pending.push_back(Pending{name_, a_, b_});
  }
}

// Kernels launched inside CUDA graphs (the device-side wavefront loop) report
// their launch counts and device-timed durations here.
void profile_add(const char* name, uint64_t launches, double ms) {
  Profiler& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  Agg& a = p.agg[name];
  a.launches += launches;
  a.ms += ms;
}

bool profile_enabled() { return prof().on.load(std::memory_order_relaxed); }

void launch_count_add(uint64_t n) { prof().launches.fetch_add(n, std::memory_order_relaxed); }

}  // namespace mpap

extern "C" {

int32_t mpap_profile_enable(int32_t on) {
  mpap::prof().on.store(on != 0);
  return MPAP_OK;
}

int32_t mpap_profile_reset(void) {
  auto& p = mpap::prof();
  std::lock_guard<std::mutex> g(p.mu);
  p.drain();
  p.agg.clear();
  p.launches.store(0);
  return MPAP_OK;
}

uint64_t mpap_launch_count(void) { return mpap::prof().launches.load(); }

int32_t mpap_profile_read(uint32_t cap, char* names, uint64_t* launches, double* total_ms, uint32_t* n) {
  auto& p = mpap::prof();
  std::lock_guard<std::mutex> g(p.mu);
  p.drain();
  uint32_t i = 0;
  for (auto& kv : p.agg) {
    if (i < cap) {
      if (names) {
        std::strncpy(names + 64 * (size_t)i, kv.first.c_str(), 63);
        names[64 * (size_t)i + 63] = 0;
      }
      if (launches) launches[i] = kv.second.launches;
      if (total_ms) total_ms[i] = kv.second.ms;
    }
    ++i;
  }
  if (n) *n = i;
  return i <= cap ? MPAP_OK : MPAP_ERR_INVALID_ARG;
}

}  // extern "C"
