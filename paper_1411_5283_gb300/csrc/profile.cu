// Optional per-kernel timing: when enabled, every kernel launch of the
// library is bracketed by a pair of CUDA events recorded on its own stream.
// bsort_profile_read() waits for the events and folds them into per-kernel
// totals (launch count, summed device time).
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace bsort {

namespace {

struct Pending {
  const char* name;
  cudaEvent_t a, b;
};

struct Total {
  std::string name;
  uint64_t launches = 0;
  double ms = 0.0;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free;
std::vector<Total> g_totals;
const char* g_open_name = nullptr;
cudaEvent_t g_open_event = nullptr;

cudaEvent_t take_event() {
  if (!g_free.empty()) {
    cudaEvent_t e = g_free.back();
    g_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

}  // namespace

bool profiling() { return g_on; }

void prof_begin(const char* name, cudaStream_t s) {
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_mu);
  g_open_name = name;
  g_open_event = take_event();
  cudaEventRecord(g_open_event, s);
}

void prof_end(cudaStream_t s) {
  if (!g_on || !g_open_event) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = take_event();
  cudaEventRecord(b, s);
  g_pending.push_back({g_open_name, g_open_event, b});
  g_open_event = nullptr;
}

}  // namespace bsort

using namespace bsort;

extern "C" {

bsort_status bsort_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = on != 0;
  return BSORT_OK;
}

bsort_status bsort_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& p : g_pending) {
    cudaEventSynchronize(p.b);
    g_free.push_back(p.a);
    g_free.push_back(p.b);
  }
  g_pending.clear();
  g_totals.clear();
  return BSORT_OK;
}

uint32_t bsort_profile_read(char* names, size_t names_bytes, uint64_t* launches, double* ms,
                            uint32_t max_entries) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& p : g_pending) {
    cudaEventSynchronize(p.b);
    float t = 0.f;
    cudaEventElapsedTime(&t, p.a, p.b);
    Total* tot = nullptr;
    for (auto& x : g_totals)
      if (x.name == p.name) tot = &x;
    if (!tot) {
      g_totals.push_back(Total{p.name});
      tot = &g_totals.back();
    }
    tot->launches += 1;
    tot->ms += t;
    g_free.push_back(p.a);
    g_free.push_back(p.b);
  }
  g_pending.clear();
  const uint32_t n = static_cast<uint32_t>(g_totals.size());
  size_t used = 0;
  for (uint32_t i = 0; i < n && i < max_entries; ++i) {
    if (launches) launches[i] = g_totals[i].launches;
    if (ms) ms[i] = g_totals[i].ms;
    if (names) {
      const std::string& nm = g_totals[i].name;
      if (used + nm.size() + 1 <= names_bytes) {
        std::memcpy(names + used, nm.c_str(), nm.size() + 1);
        used += nm.size() + 1;
      }
    }
  }
  return n;
}

}  // extern "C"
