// Launch counting, opt-in CUDA-event timing of one kernel class, and the
// unit-peak microbenchmarks used as roofline denominators.
//
// Every launch site calls pn_note_launch(name, stream) right after the
// launch.  The counter feeds pn_launch_count(); when timing is enabled for
// `name`, a pair of events brackets that launch on its own stream (the
// start event is recorded by pn_prof_begin before the launch), and launch
// sites that know their algorithmic work report it through pn_prof_work.
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
double g_work = 0;
double g_bytes = 0;

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

void pn_prof_work(const char* name, double work) {
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_target == name) g_work += work;
}

void pn_prof_bytes(const char* name, double bytes) {
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_target == name) g_bytes += bytes;
}

extern "C" unsigned long long pn_launch_count(void) { return g_launches.load(); }

extern "C" int pn_profile_kernel(const char* name) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& r : g_recs) {
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  g_work = 0;
  g_bytes = 0;
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

extern "C" int pn_profile_work(double* work) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (work) *work = g_work;
  return PN_OK;
}

extern "C" int pn_profile_bytes(double* bytes) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (bytes) *bytes = g_bytes;
  return PN_OK;
}

// ------------------------------------------------------ unit peaks
// Eight independent multiply-add chains per thread keep every FMA lane busy
// (a dependent chain would expose the pipeline latency); the operands come
// from the arguments so that nothing folds at compile time, and the result
// is stored only under a condition that never holds.
namespace {
template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* out, int iters, T b, T c) {
  T a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = (T)(threadIdx.x + i) * c;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  if (s == (T)-1.2345) out[blockIdx.x] = s;
}
}  // namespace

extern "C" int pn_measure_peak(int kind, double* tflops, void* stream) {
  if ((kind != 0 && kind != 1) || !tflops) {
    pn_set_error("pn_measure_peak: kind 0 (float32 FMA) or 1 (float64 FMA) and an output");
    return PN_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  PN_CUDA(cudaGetDevice(&dev));
  PN_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256;
  const int iters = kind == 0 ? 400000 : 8000;
  void* out = nullptr;
  PN_CUDA(cudaMallocAsync(&out, (size_t)blocks * 8, st));
  cudaEvent_t a, b;
  PN_CUDA(cudaEventCreate(&a));
  PN_CUDA(cudaEventCreate(&b));
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    PN_CUDA(cudaEventRecord(a, st));
    if (kind == 0)
      PN_LAUNCH("k_fma_peak", st, (k_fma_peak<float><<<blocks, threads, 0, st>>>((float*)out, iters, 0.9999999f, 1e-7f)));
    else
      PN_LAUNCH("k_fma_peak", st, (k_fma_peak<double><<<blocks, threads, 0, st>>>((double*)out, iters, 0.9999999, 1e-7)));
    PN_CUDA(cudaEventRecord(b, st));
    PN_CUDA(cudaEventSynchronize(b));
    float ms = 0;
    PN_CUDA(cudaEventElapsedTime(&ms, a, b));
    if (rep > 0) best = ms < best ? ms : best;  // the first launch warms the clocks
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  PN_CUDA(cudaFreeAsync(out, st));
  PN_CUDA(cudaStreamSynchronize(st));
  *tflops = 2.0 * 8.0 * (double)iters * blocks * threads / (best * 1e-3) / 1e12;
  return PN_OK;
}
