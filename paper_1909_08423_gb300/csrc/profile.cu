// Launch counting and opt-in CUDA-event timing of one kernel class.
//
// Every launch site calls pn_note_launch(name, stream) right after the
// launch.  The counter feeds pn_launch_count(); when timing is enabled for
// `name`, a pair of events brackets that launch on its own stream (the
// start event is recorded by pn_prof_begin before the launch).
#include <string.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "pn_internal.cuh"

namespace {
std::atomic<unsigned long long> g_launches{0};
std::mutex g_mu;
std::string g_target;
bool g_on = false;
struct Rec {
  cudaEvent_t a, b;
};
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
cudaEvent_t g_pending = nullptr;

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

void pn_prof_begin(const char* name, cudaStream_t st) {
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_target != name) return;
  g_pending = take_event();
  cudaEventRecord(g_pending, st);
}

void pn_note_launch(const char* name, cudaStream_t st) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_target != name || !g_pending) return;
  cudaEvent_t b = take_event();
  cudaEventRecord(b, st);
  g_recs.push_back({g_pending, b});
  g_pending = nullptr;
}

extern "C" unsigned long long pn_launch_count(void) { return g_launches.load(); }

extern "C" int pn_profile_kernel(const char* name) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& r : g_recs) {
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  g_on = name && name[0];
  g_target = g_on ? name : "";
  return PN_OK;
}

extern "C" int pn_profile_read(int64_t* count, double* total_ms) {
  std::lock_guard<std::mutex> lk(g_mu);
  double tot = 0;
  for (auto& r : g_recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) {
      pn_set_error("profile: event synchronize failed");
      return PN_EDEVICE;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, r.a, r.b);
    tot += ms;
  }
  if (count) *count = (int64_t)g_recs.size();
  if (total_ms) *total_ms = tot;
  return PN_OK;
}
