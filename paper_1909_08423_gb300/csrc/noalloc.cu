// ln|psi| for callers that must not allocate device memory at call time.
//
// Some callers cannot call cudaMalloc (or anything that allocates) when they
// evaluate: a real-time or latency-bound loop that must not block on the
// allocator, or a process that reserves all of its device memory up front
// and may not grow afterwards.  pn_eval_logpsi_static serves them:
// it runs the same value pass as pn_eval_logpsi, but its intermediates live
// in one fixed file-scope device array instead of the handle's workspace, and
// the call itself allocates nothing.  The system handle must have been made
// earlier by pn_init_system, which does allocate.
#include <algorithm>
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

// The value pass's intermediates only (the handle's workspace also holds
// position staging, energies, gradients and proposal buffers that this call
// never touches): bytes for W walkers, and the carve with the unused
// buffers left null.
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

template <typename R>
size_t value_bytes(const DevSys& s, size_t W) {
  const size_t N = s.N, e = sizeof(R);
  const size_t ldH = std::max(s.Zd, s.D), ldZ = std::max(3 * s.Zd, s.D);
  return align256(W * s.Ppair * 4 * 8) + align256(W * N * s.n_orb * 5 * 8) + align256(W * s.Ppair * 3 * s.K * e) +
         align256(W * s.Ppair * 3 * s.Zd * e) + align256(W * N * s.D * e) + align256(W * N * ldH * e) +
         align256(W * N * ldZ * e) + 3 * align256(W * s.D * e) + align256(W * N * s.n_orb * e) + align256(W * e) +
         align256(W * s.n_det * 2 * (3 + 3 * N) * 8) + 2 * align256(W * 8) + align256(W * 4);
}

template <typename R>
Work<R> value_carve(const DevSys& s, int Wc, void* base) {
  Work<R> w{};
  char* p = (char*)base;
  const size_t W = Wc, N = s.N, e = sizeof(R);
  const size_t ldH = std::max(s.Zd, s.D), ldZ = std::max(3 * s.Zd, s.D);
  auto take = [&](size_t bytes) { char* q = p; p += align256(bytes); return (void*)q; };
  w.Wc = Wc;
  w.T = 1;
  w.geo = (double*)take(W * s.Ppair * 4 * 8);
  w.phi = (double*)take(W * N * s.n_orb * 5 * 8);
  w.efeat = (R*)take(W * s.Ppair * 3 * s.K * e);
  w.wjet = (R*)take(W * s.Ppair * 3 * s.Zd * e);
  w.X = (R*)take(W * N * s.D * e);
  w.H = (R*)take(W * N * ldH * e);
  w.Zb = (R*)take(W * N * ldZ * e);
  w.Xs = (R*)take(W * s.D * e);
  w.As = (R*)take(W * s.D * e);
  w.Bs = (R*)take(W * s.D * e);
  w.F = (R*)take(W * N * s.n_orb * e);
  w.Jj = (R*)take(W * e);
  w.det = (double*)take(W * s.n_det * 2 * (3 + 3 * N) * 8);
  w.out_logabs = (double*)take(W * 8);
  w.out_sign = (double*)take(W * 8);
  w.out_status = (int*)take(W * 4);
  w.ldH = (int)ldH;
  w.ldZ = (int)ldZ;
  w.end = p;
  return w;
}

template <typename R>
int eval_static(pn_system_s* s, const double* r, int W, double* logabs, double* sign, int* status, cudaStream_t st) {
  const DevSys& ds = s->ds;
  const size_t need = value_bytes<R>(ds, W);
  if (need > PN_STATIC_SCRATCH_BYTES) {
    int cap = 0;
    while (value_bytes<R>(ds, cap + 1) <= PN_STATIC_SCRATCH_BYTES) ++cap;
    pn_set_error("static scratch holds %d walkers of this system (%u bytes); %d requested", cap,
                 (unsigned)PN_STATIC_SCRATCH_BYTES, W);
    return PN_EINVAL;
  }
  void* base = nullptr;
  if (int e = scratch_on_current_device(&base)) return e;
  Work<R> w = value_carve<R>(ds, W, base);
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
