// ln|psi| for callers that must not allocate device memory at call time.
//
// Some callers cannot call cudaMalloc (or anything that allocates) when they
// evaluate: a host thread recording a CUDA graph (allocation is not allowed
// during stream capture), a real-time or latency-bound loop that must not
// block on the allocator, or a process that reserves all of its device memory
// up front and may not grow afterwards.  pn_eval_logpsi_static serves them:
// it runs the same value pass as pn_eval_logpsi, but its intermediates live
// in one fixed file-scope device array instead of the handle's workspace, and
// the call itself allocates nothing.  The system handle must have been made
// earlier by pn_init_system, which does allocate.
#include <mutex>

#include "pn_internal.cuh"

// Fixed scratch: 16 MiB on every GPU that loads the library, held until the
// process exits.
#define PN_STATIC_SCRATCH_BYTES (16u << 20)
static __device__ __align__(256) unsigned char pn_static_scratch[PN_STATIC_SCRATCH_BYTES];

namespace {

// The array's name in host code is only a stand-in, not a device address:
// its address on each device comes from cudaGetSymbolAddress, looked up once
// per device with that device current.
constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

int scratch_on_current_device(void** out) {
  int dev = -1;
  PN_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    pn_set_error("static scratch: device ordinal %d beyond %d", dev, kMaxDevices);
    return PN_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, pn_static_scratch);
    if (e != cudaSuccess || !p) {
      pn_set_error("static scratch: cudaGetSymbolAddress failed on device %d: %s", dev, cudaGetErrorString(e));
      return PN_EDEVICE;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return PN_OK;
}

template <typename R>
int eval_static(pn_system_s* s, const double* r, int W, double* logabs, double* sign, int* status, cudaStream_t st) {
  const DevSys& ds = s->ds;
  const size_t need = pn_work_bytes(ds, W, 1, (int)sizeof(R));
  if (need > PN_STATIC_SCRATCH_BYTES) {
    int cap = 0;
    while (pn_work_bytes(ds, cap + 1, 1, (int)sizeof(R)) <= PN_STATIC_SCRATCH_BYTES) ++cap;
    pn_set_error("static scratch holds %d walkers of this system (%u bytes); %d requested", cap,
                 (unsigned)PN_STATIC_SCRATCH_BYTES, W);
    return PN_EINVAL;
  }
  void* base = nullptr;
  if (int e = scratch_on_current_device(&base)) return e;
  Work<R> w = pn_carve_work<R>(ds, W, 1, base);
  const DevNet<R> net = pn_devnet<R>(s);
  // Nothing in the value pass reads scratch before writing it, so the array
  // needs no clearing between calls.
  if (int e = pn_forward_chunk<R>(ds, net, w, r, W, 0, st)) return e;
  PN_CUDA(cudaMemcpyAsync(logabs, w.out_logabs, (size_t)W * 8, cudaMemcpyDeviceToDevice, st));
  if (sign) PN_CUDA(cudaMemcpyAsync(sign, w.out_sign, (size_t)W * 8, cudaMemcpyDeviceToDevice, st));
  if (status) PN_CUDA(cudaMemcpyAsync(status, w.out_status, (size_t)W * 4, cudaMemcpyDeviceToDevice, st));
  return PN_OK;
}

}  // namespace

extern "C" int pn_eval_logpsi_static(pn_system_t s, const double* r, int W, double* logabs, double* sign, int* status,
                                     void* stream) {
  if (!s || W < 0 || (W > 0 && (!r || !logabs))) {
    pn_set_error("bad arguments");
    return PN_EINVAL;
  }
  if (W == 0) return PN_OK;
  if (!pn_is_device_ptr(r) || !pn_is_device_ptr(logabs) || (sign && !pn_is_device_ptr(sign)) ||
      (status && !pn_is_device_ptr(status))) {
    pn_set_error("pn_eval_logpsi_static takes device buffers only (host buffers would need staging memory)");
    return PN_EINVAL;
  }
  int cur = -1;
  PN_CUDA(cudaGetDevice(&cur));
  if (cur != s->device) {
    pn_set_error("pn_eval_logpsi_static: make the handle's device (%d) current first", s->device);
    return PN_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  return s->precision == PN_FP64 ? eval_static<double>(s, r, W, logabs, sign, status, st)
                                 : eval_static<float>(s, r, W, logabs, sign, status, st);
}
