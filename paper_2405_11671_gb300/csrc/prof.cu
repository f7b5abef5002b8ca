// prof.cu -- launch counting and optional per-kernel device timing.
//
// Every kernel launch of the library increments a process-wide counter
// (byo_kernel_launches).  When profiling is on, the main kernels of each call
// are bracketed by CUDA events recorded on the caller's stream; byo_profile_read
// resolves them (synchronising) into per-kernel launch counts and total device
// milliseconds.  This is the library's tracing facility; it adds two event
// records per bracketed launch and nothing when off.
#include <string.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "byo_internal.cuh"
#include "prof.cuh"

namespace byo {

namespace {
std::atomic<uint64_t> g_launches{0};
std::atomic<bool> g_on{false};
std::mutex g_mu;
struct Pending {
  std::string name;
  cudaEvent_t a, b;
};
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free;
struct Stat {
  std::string name;
  uint64_t launches;
  double ms;
};
std::vector<Stat> g_stats;

cudaEvent_t take_event() {
  if (!g_free.empty()) {
    cudaEvent_t e = g_free.back();
    g_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}
}  // namespace

void note_launch(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
bool profiling_on() { return g_on.load(std::memory_order_relaxed); }

ProfScope::ProfScope(const char* name, cudaStream_t s) : name_(name), s_(s), a_(nullptr) {
  if (!g_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  a_ = take_event();
  if (a_) cudaEventRecord(static_cast<cudaEvent_t>(a_), s_);
}

ProfScope::~ProfScope() {
  if (!a_) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = take_event();
  if (!b) {
    g_free.push_back(static_cast<cudaEvent_t>(a_));
    return;
  }
  cudaEventRecord(b, s_);
  g_pending.push_back(Pending{name_, static_cast<cudaEvent_t>(a_), b});
}

}  // namespace byo

using namespace byo;

extern "C" {

uint64_t byo_kernel_launches(void) { return g_launches.load(); }

byo_status byo_profile_enable(int on) {
  g_on.store(on != 0);
  return BYO_OK;
}

byo_status byo_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& p : g_pending) {
    cudaEventSynchronize(p.b);
    g_free.push_back(p.a);
    g_free.push_back(p.b);
  }
  g_pending.clear();
  g_stats.clear();
  return BYO_OK;
}

byo_status byo_profile_read(byo_kernel_stat* host_stats, uint32_t cap, uint32_t* host_count) {
  clear_error();
  if (!host_count || (cap && !host_stats)) {
    set_error("byo_profile_read: NULL output");
    return BYO_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& p : g_pending) {
    cudaError_t e = cudaEventSynchronize(p.b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.a, p.b);
    if (e != cudaSuccess) return cuda_status(e, "byo_profile_read");
    bool found = false;
    for (auto& s : g_stats) {
      if (s.name == p.name) {
        s.launches += 1;
        s.ms += ms;
        found = true;
        break;
      }
    }
    if (!found) g_stats.push_back(Stat{p.name, 1, (double)ms});
    g_free.push_back(p.a);
    g_free.push_back(p.b);
  }
  g_pending.clear();
  *host_count = (uint32_t)g_stats.size();
  uint32_t c = g_stats.size() < cap ? (uint32_t)g_stats.size() : cap;
  for (uint32_t i = 0; i < c; ++i) {
    memset(host_stats[i].name, 0, sizeof(host_stats[i].name));
    strncpy(host_stats[i].name, g_stats[i].name.c_str(), sizeof(host_stats[i].name) - 1);
    host_stats[i].launches = g_stats[i].launches;
    host_stats[i].total_ms = g_stats[i].ms;
  }
  return BYO_OK;
}

}  // extern "C"
