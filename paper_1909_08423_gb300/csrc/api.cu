// C ABI entry points for evaluation, sampling and clipping.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>

#include "kernels.cuh"
#include "pn_internal.cuh"

namespace {

inline unsigned nblk(size_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <typename R>
Work<R>& work_of(pn_system_s* s);
template <>
Work<double>& work_of<double>(pn_system_s* s) { return s->w64; }
template <>
Work<float>& work_of<float>(pn_system_s* s) { return s->w32; }

// ---------------------------------------------------------------- sampling
// r' = r + sigma xi for every coordinate of walker w (walker id walker0 + w).
__global__ void k_propose(const double* __restrict__ r, double* __restrict__ rp, int Wn, int N, unsigned walker0,
                          unsigned long long seed, unsigned long long step, double sigma) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= Wn) return;
  const int n3 = 3 * N;
  for (int j = 0; j * 4 < n3; ++j) {
    double z[4];
    pn_normals4(seed, walker0 + w, step, j, z);
    for (int k = 0; k < 4; ++k) {
      const int m = 4 * j + k;
      if (m < n3) rp[(size_t)w * n3 + m] = r[(size_t)w * n3 + m] + sigma * z[k];
    }
  }
}

// accept iff u < exp(2 (lp' - lp)); u is word 0 of block ceil(3N/4).
__global__ void k_accept(double* __restrict__ r, double* __restrict__ lp, const double* __restrict__ rp,
                         const double* __restrict__ lpp, int Wn, int N, unsigned walker0, unsigned long long seed,
                         unsigned long long step, unsigned long long* n_acc) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= Wn) return;
  const int n3 = 3 * N;
  unsigned c[4] = {(unsigned)((n3 + 3) / 4), walker0 + w, (unsigned)(step & 0xffffffffull), (unsigned)(step >> 32)};
  pn_philox(c, (unsigned)(seed & 0xffffffffull), (unsigned)(seed >> 32));
  const double u = pn_u01(c[0]);
  const bool acc = u < exp(2.0 * (lpp[w] - lp[w]));
  if (acc) {
    for (int m = 0; m < n3; ++m) r[(size_t)w * n3 + m] = rp[(size_t)w * n3 + m];
    lp[w] = lpp[w];
    atomicAdd(n_acc, 1ull);
  }
}

// ---------------------------------------------------------- Langevin moves
// Drift displacement of electron e: c = tau * grad_e ln|psi|, shortened to
// the distance from r_e to the nearest nucleus when longer, so that the
// drift cannot carry the electron past a nucleus.
__device__ inline void langevin_drift(const DevSys& s, const double* re, const double* ge, double tau, double c[3]) {
  double dmin = INFINITY;
  for (int I = 0; I < s.M; ++I) {
    const double a = re[0] - s.R[3 * I], b = re[1] - s.R[3 * I + 1], d = re[2] - s.R[3 * I + 2];
    dmin = fmin(dmin, sqrt(a * a + b * b + d * d));
  }
  for (int x = 0; x < 3; ++x) c[x] = tau * ge[x];
  const double len = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
  if (len > dmin) {
    const double f = dmin / len;
    for (int x = 0; x < 3; ++x) c[x] *= f;
  }
}

// r' = r + c(r) + sqrt(tau) xi (normals from the same Philox layout as the
// Gaussian proposal); keeps |xi|^2 / 2, the forward term of the proposal
// density ratio.
__global__ void k_langevin_propose(DevSys s, const double* __restrict__ r, const double* __restrict__ drift,
                                   double* __restrict__ rp, double* __restrict__ half_xi2, int Wn, unsigned walker0,
                                   unsigned long long seed, unsigned long long step, double tau) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= Wn) return;
  const int N = s.N, n3 = 3 * N;
  const double st = sqrt(tau);
  double x2 = 0;
  for (int e = 0; e < N; ++e) {
    double c[3];
    langevin_drift(s, r + (size_t)w * n3 + 3 * e, drift + (size_t)w * n3 + 3 * e, tau, c);
    for (int x = 0; x < 3; ++x) rp[(size_t)w * n3 + 3 * e + x] = r[(size_t)w * n3 + 3 * e + x] + c[x];
  }
  for (int j = 0; j * 4 < n3; ++j) {
    double z[4];
    pn_normals4(seed, walker0 + w, step, j, z);
    for (int k = 0; k < 4; ++k) {
      const int m = 4 * j + k;
      if (m < n3) {
        rp[(size_t)w * n3 + m] += st * z[k];
        x2 += z[k] * z[k];
      }
    }
  }
  half_xi2[w] = 0.5 * x2;
}

// Metropolis-Hastings test u < |psi'/psi|^2 T(r' -> r) / T(r -> r') with
// T(x -> y) = exp(-|y - x - c(x)|^2 / (2 tau)); u is word 0 of block
// ceil(3N/4) as for the Gaussian proposal.  On accept r, ln|psi| and the
// drift take the proposal's values.
__global__ void k_langevin_accept(DevSys s, double* __restrict__ r, double* __restrict__ lp,
                                  double* __restrict__ drift, const double* __restrict__ rp,
                                  const double* __restrict__ lpp, const double* __restrict__ gp,
                                  const double* __restrict__ half_xi2, int Wn, unsigned walker0,
                                  unsigned long long seed, unsigned long long step, double tau,
                                  unsigned long long* n_acc) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= Wn) return;
  const int N = s.N, n3 = 3 * N;
  double back2 = 0;
  for (int e = 0; e < N; ++e) {
    double c[3];
    langevin_drift(s, rp + (size_t)w * n3 + 3 * e, gp + (size_t)w * n3 + 3 * e, tau, c);
    for (int x = 0; x < 3; ++x) {
      const double b = r[(size_t)w * n3 + 3 * e + x] - rp[(size_t)w * n3 + 3 * e + x] - c[x];
      back2 += b * b;
    }
  }
  const double log_ratio = 2.0 * (lpp[w] - lp[w]) + half_xi2[w] - back2 / (2.0 * tau);
  unsigned cc[4] = {(unsigned)((n3 + 3) / 4), walker0 + w, (unsigned)(step & 0xffffffffull), (unsigned)(step >> 32)};
  pn_philox(cc, (unsigned)(seed & 0xffffffffull), (unsigned)(seed >> 32));
  const double u = pn_u01(cc[0]);
  if (u < exp(log_ratio)) {
    for (int m = 0; m < n3; ++m) {
      r[(size_t)w * n3 + m] = rp[(size_t)w * n3 + m];
      drift[(size_t)w * n3 + m] = gp[(size_t)w * n3 + m];
    }
    lp[w] = lpp[w];
    atomicAdd(n_acc, 1ull);
  }
}

// Configurations of a line scan: every point is the base configuration r0
// [N][3] with electron e moved to r0[e] + (t0 + (k0 + k) dt) dir.
__global__ void k_line_positions(const double* __restrict__ r0, int N, int e, double dx, double dy, double dz, double t0,
                                 double dt, int k0, int n, double* __restrict__ r) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double tk = t0 + (double)(k0 + k) * dt;
  for (int m = 0; m < 3 * N; ++m) r[(size_t)k * 3 * N + m] = r0[m];
  r[(size_t)k * 3 * N + 3 * e] = r0[3 * e] + tk * dx;
  r[(size_t)k * 3 * N + 3 * e + 1] = r0[3 * e + 1] + tk * dy;
  r[(size_t)k * 3 * N + 3 * e + 2] = r0[3 * e + 2] + tk * dz;
}

// electron e at R[nuc(e)] + normal, normals at step 2^64 - 1.
__global__ void k_init_walkers(DevSys s, const int* __restrict__ nuc, double* __restrict__ r, int W,
                               unsigned long long seed) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  const int n3 = 3 * s.N;
  const unsigned long long step = ~0ull;
  for (int j = 0; j * 4 < n3; ++j) {
    double z[4];
    pn_normals4(seed, (unsigned)w, step, j, z);
    for (int k = 0; k < 4; ++k) {
      const int m = 4 * j + k;
      if (m < n3) r[(size_t)w * n3 + m] = s.R[3 * nuc[m / 3] + m % 3] + z[k];
    }
  }
}

// ------------------------------------------------------------------ guard
// Walkers of a mixed chunk whose two evaluations differ by more than tau
// (or give a non-finite difference) go to the list; singular walkers are
// left alone (their E_loc is undefined in any precision).
__global__ void k_guard_flag(const double* __restrict__ e1, const double* __restrict__ e2,
                             const int* __restrict__ status, int Wn, double tau, int* __restrict__ list,
                             int* __restrict__ count) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= Wn) return;
  if (status[w] == PN_WALKER_SINGULAR) return;
  if (!(fabs(e1[w] - e2[w]) <= tau)) list[atomicAdd(count, 1)] = w;
}

// Positions of flagged walkers k0 .. k0 + n - 1 into the float64 workspace.
__global__ void k_guard_gather(const double* __restrict__ r, const int* __restrict__ list, int k0, int n, int N,
                               double* __restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n * 3 * N) return;
  const int k = q / (3 * N), m = q - k * 3 * N;
  out[q] = r[(size_t)list[k0 + k] * 3 * N + m];
}

// Float64 results of the flagged walkers back into the outputs (the
// chunk's workspace, or the caller's arrays at global indices; null
// destinations are skipped).
__global__ void k_guard_scatter(const int* __restrict__ list, int k0, int n, int N, const double* __restrict__ e64,
                                const double* __restrict__ l64, const double* __restrict__ s64,
                                const int* __restrict__ st64, const double* __restrict__ g64, double* __restrict__ e,
                                double* __restrict__ l, double* __restrict__ sg, int* __restrict__ st,
                                double* __restrict__ g, int64_t* __restrict__ n_total) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int w = list[k0 + k];
  if (e) e[w] = e64[k];
  if (l) l[w] = l64[k];
  if (sg) sg[w] = s64[k];
  if (st) st[w] = st64[k];
  if (g)
    for (int m = 0; m < 3 * N; ++m) g[(size_t)w * 3 * N + m] = g64[(size_t)k * 3 * N + m];
  if (k == 0) atomicAdd((unsigned long long*)n_total, (unsigned long long)n);
}

// The chunk's flagged walkers (local indices) appended to the pending list
// as global indices.
__global__ void k_guard_append(const int* __restrict__ list, int n, int c0, int* __restrict__ pend) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) pend[k] = c0 + list[k];
}

// Value-pass components for step-by-step checks.
template <typename R>
__global__ void k_components(DevSys s, const double* __restrict__ phi, const R* __restrict__ F,
                             const R* __restrict__ Jj, const double* __restrict__ det, int Wn, double* __restrict__ ophi,
                             double* __restrict__ oJ, double* __restrict__ of, double* __restrict__ old) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= Wn) return;
  const int N = s.N, no = s.n_orb, stride = 3 + 3 * N;
  for (int k = 0; k < N * no; ++k) {
    if (ophi) ophi[(size_t)w * N * no + k] = phi[((size_t)w * N * no + k) * 5];
    if (of) of[(size_t)w * N * no + k] = 1.0 + (double)F[(size_t)w * N * no + k];
  }
  if (oJ) oJ[w] = (double)Jj[w];
  if (old)
    for (int p = 0; p < s.n_det; ++p) {
      const double* d = det + ((size_t)w * s.n_det + p) * 2 * stride;
      old[(size_t)w * s.n_det + p] = d[0] + d[stride];
    }
}

// ---------------------------------------------------------------- clipping
// One block: bitonic sort of the batch in shared memory for the median,
// mean absolute deviation, logarithmic clipping, then the loss weights.
// The sort runs on order-preserving 64-bit integer keys of the doubles
// (sign bit set for non-negatives, all bits flipped for negatives), so that
// its compares stay off the float64 pipe; padding takes the largest key.
__device__ inline unsigned long long clip_key(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ inline double clip_unkey(unsigned long long k) {
  return __longlong_as_double((long long)((k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k));
}
__global__ void k_clip(const double* __restrict__ E, int W, double q, double* __restrict__ out,
                       double* __restrict__ cot) {
  extern __shared__ unsigned long long skey[];
  __shared__ double red[32];
  int n = 1;
  while (n < W) n <<= 1;
  for (int i = threadIdx.x; i < n; i += blockDim.x) skey[i] = i < W ? clip_key(E[i]) : ~0ull;
  __syncthreads();
  for (int k = 2; k <= n; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const bool up = (i & k) == 0;
          const unsigned long long a = skey[i], b = skey[l];
          if ((a > b) == up) { skey[i] = b; skey[l] = a; }
        }
      }
      __syncthreads();
    }
  const double m = 0.5 * (clip_unkey(skey[(W - 1) / 2]) + clip_unkey(skey[W / 2]));
  auto block_sum = [&](double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    return t;
  };
  double a = 0;
  for (int i = threadIdx.x; i < W; i += blockDim.x) a += fabs(E[i] - m);
  const double dev = block_sum(a) / W;
  const double Lq = q * dev;
  double sum = 0;
  for (int i = threadIdx.x; i < W; i += blockDim.x) {
    const double x = E[i] - m;
    double v = E[i];
    if (fabs(x) > Lq) v = m + copysign(Lq * (1.0 + log(fabs(x) / Lq)), x);
    out[i] = v;
    sum += v;
  }
  const double mean = block_sum(sum) / W;
  if (cot)
    for (int i = threadIdx.x; i < W; i += blockDim.x) cot[i] = 2.0 * (out[i] - mean) / W;
}

// Batches beyond one block's shared memory: the keys are sorted in global
// memory by a bitonic network (one launch per compare distance), then one
// block forms the statistics from the sorted keys.
__global__ void k_clip_keys(const double* __restrict__ E, int W, int n, unsigned long long* __restrict__ key) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) key[i] = i < W ? clip_key(E[i]) : ~0ull;
}

__global__ void k_bitonic_step(unsigned long long* __restrict__ key, int n, int j, int k) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int l = i ^ j;
  if (l > i) {
    const bool up = (i & k) == 0;
    const unsigned long long a = key[i], b = key[l];
    if ((a > b) == up) { key[i] = b; key[l] = a; }
  }
}

__global__ void k_clip_stats(const unsigned long long* __restrict__ key, const double* __restrict__ E, int W, double q,
                             double* __restrict__ out, double* __restrict__ cot) {
  __shared__ double red[32];
  const double m = 0.5 * (clip_unkey(key[(W - 1) / 2]) + clip_unkey(key[W / 2]));
  auto block_sum = [&](double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    return t;
  };
  double a = 0;
  for (int i = threadIdx.x; i < W; i += blockDim.x) a += fabs(E[i] - m);
  const double Lq = q * block_sum(a) / W;
  double sum = 0;
  for (int i = threadIdx.x; i < W; i += blockDim.x) {
    const double x = E[i] - m;
    double v = E[i];
    if (fabs(x) > Lq) v = m + copysign(Lq * (1.0 + log(fabs(x) / Lq)), x);
    out[i] = v;
    sum += v;
  }
  const double mean = block_sum(sum) / W;
  if (cot)
    for (int i = threadIdx.x; i < W; i += blockDim.x) cot[i] = 2.0 * (out[i] - mean) / W;
}

bool is_host(const void* p) { return p && !pn_is_device_ptr(p); }

int set_device(pn_system_s* s) {
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != s->device) PN_CUDA(cudaSetDevice(s->device));
  return PN_OK;
}

template <typename R>
int eval_impl(pn_system_s* s, const double* r, int W, int jet, double* eloc, double* logabs, double* sign, int* status,
              cudaStream_t st) {
  const Guard* g = (s->guard_mem && s->guard.tau > 0) ? &s->guard : nullptr;
  return pn_run_eval<R>(s->ds, pn_devnet<R>(s), work_of<R>(s), s->Wc, r, W, jet, eloc, logabs, sign, status, st, g);
}

template <typename R>
int components_impl(pn_system_s* s, const double* r, int W, double* phi, double* J, double* f, double* ld,
                    cudaStream_t st) {
  Work<R>& w = work_of<R>(s);
  const DevNet<R> net = pn_devnet<R>(s);
  const DevSys& ds = s->ds;
  const int N = ds.N, no = ds.n_orb;
  const bool rdev = pn_is_device_ptr(r);
  const bool host_out = is_host(phi) || is_host(J) || is_host(f) || is_host(ld);
  // call-scoped staging for the gathered outputs (a diagnostic entry point)
  double* tmp = nullptr;
  const size_t per_w = (size_t)2 * N * no + 1 + ds.n_det;
  PN_CUDA(cudaMallocAsync((void**)&tmp, (size_t)s->Wc * per_w * 8, st));
  for (int c0 = 0; c0 < W; c0 += s->Wc) {
    const int Wn = std::min(s->Wc, W - c0);
    const double* rc = r + (size_t)c0 * N * 3;
    if (!rdev) {
      PN_CUDA(cudaMemcpyAsync(w.r, rc, (size_t)Wn * N * 3 * 8, cudaMemcpyHostToDevice, st));
      rc = w.r;
    }
    if (int e = pn_forward_chunk<R>(ds, net, w, rc, Wn, 0, st)) return e;
    double* tphi = tmp;
    double* tf = tphi + (size_t)Wn * N * no;
    double* tJ = tf + (size_t)Wn * N * no;
    double* tld = tJ + Wn;
    PN_LAUNCH("k_components", st, k_components<R><<<nblk(Wn, 64), 64, 0, st>>>(ds, w.phi, w.F, w.Jj, w.det, Wn, tphi, tJ, tf, tld));
    if (phi) PN_CUDA(cudaMemcpyAsync(phi + (size_t)c0 * N * no, tphi, (size_t)Wn * N * no * 8, cudaMemcpyDefault, st));
    if (f) PN_CUDA(cudaMemcpyAsync(f + (size_t)c0 * N * no, tf, (size_t)Wn * N * no * 8, cudaMemcpyDefault, st));
    if (J) PN_CUDA(cudaMemcpyAsync(J + c0, tJ, (size_t)Wn * 8, cudaMemcpyDefault, st));
    if (ld) PN_CUDA(cudaMemcpyAsync(ld + (size_t)c0 * ds.n_det, tld, (size_t)Wn * ds.n_det * 8, cudaMemcpyDefault, st));
    // the staging area is reused by the next chunk
    PN_CUDA(cudaStreamSynchronize(st));
  }
  (void)host_out;
  PN_CUDA(cudaFreeAsync(tmp, st));
  PN_CUDA(cudaStreamSynchronize(st));
  return PN_OK;
}

template <typename R>
int metropolis_impl(pn_system_s* s, double* r, double* logabs, int W, int n_steps, double sigma,
                    unsigned long long seed, unsigned long long step0, int64_t* n_accept, cudaStream_t st) {
  return pn_run_metropolis<R>(s->ds, pn_devnet<R>(s), work_of<R>(s), s->Wc, r, logabs, W, n_steps, sigma, seed, step0,
                              n_accept, st);
}

}  // namespace

// ------------------------------------------------------ drivers with explicit workspace
// The guard of a mixed jet chunk (see Guard), first half: the second
// evaluation and the flags.  Reads the flag count back to the host (one
// synchronisation) and returns it.
static int guard_flag_chunk(const DevSys& ds, const DevNet<float>& net, Work<float>& w, const Guard& g, int Wn,
                            int* nflag, cudaStream_t st) {
  if (int e = pn_probe_heads_chunk(ds, net, w, Wn, g.e_probe, st)) return e;
  PN_CUDA(cudaMemsetAsync(g.count, 0, sizeof(int), st));
  PN_LAUNCH("k_guard_flag", st, k_guard_flag<<<nblk(Wn, 128), 128, 0, st>>>(w.out_eloc, g.e_probe, w.out_status, Wn,
                                                                            g.tau, g.list, g.count));
  PN_CUDA(cudaMemcpyAsync(nflag, g.count, sizeof(int), cudaMemcpyDeviceToHost, st));
  PN_CUDA(cudaStreamSynchronize(st));
  return PN_OK;
}

// Second half: the float64 re-evaluation of the walkers list[0 .. n) (their
// positions in r) in pieces of g.cap, the results scattered to the given
// outputs at the same indices (any may be null).  The re-evaluation's
// linear maps run as float32 pairs (about 44 bits, at float32 issue rates);
// everything else in float64.
static int guard_reevaluate(const DevSys& ds, const Guard& g, const int* list, int n_all, const double* r, double* eloc,
                            double* logabs, double* sign, int* status, double* grad, cudaStream_t st) {
  const int N = ds.N;
  Work<double> w64 = g.w64;
  DevSys d64 = ds;
  d64.lin_f32x2 = 1;
  for (int k0 = 0; k0 < n_all; k0 += g.cap) {
    const int n = std::min(g.cap, n_all - k0);
    PN_LAUNCH("k_guard_gather", st, k_guard_gather<<<nblk((size_t)n * 3 * N, 128), 128, 0, st>>>(r, list, k0, n, N,
                                                                                                  w64.r));
    if (int e = pn_forward_chunk<double>(d64, g.net64, w64, w64.r, n, 1, st)) return e;
    PN_LAUNCH("k_guard_scatter", st,
              k_guard_scatter<<<nblk(n, 64), 64, 0, st>>>(list, k0, n, N, w64.out_eloc, w64.out_logabs, w64.out_sign,
                                                           w64.out_status, w64.out_grad, eloc, logabs, sign, status,
                                                           grad, g.n_total));
  }
  return PN_OK;
}

template <typename R>
int pn_run_eval(const DevSys& ds, const DevNet<R>& net, Work<R>& w, int Wc, const double* r, int W, int jet,
                double* eloc, double* logabs, double* sign, int* status, cudaStream_t st, const Guard* g) {
  const int N = ds.N;
  const bool rdev = pn_is_device_ptr(r);
  const bool sync = !rdev || is_host(eloc) || is_host(logabs) || is_host(sign) || is_host(status);
  const bool guarded = sizeof(R) == 4 && jet && g && g->tau > 0;
  // With the positions and every output on the device, the guard's flagged
  // walkers of successive chunks are collected (global indices, up to g.cap)
  // and re-evaluated together, writing the caller's arrays: larger float64
  // batches than one chunk's.  Otherwise each chunk's are re-evaluated into
  // its workspace before its outputs are copied.
  const bool batch = guarded && !sync;
  int pending = 0;
  for (int c0 = 0; c0 < W; c0 += Wc) {
    const int Wn = std::min(Wc, W - c0);
    const double* rc = r + (size_t)c0 * N * 3;
    if (!rdev) {
      PN_CUDA(cudaMemcpyAsync(w.r, rc, (size_t)Wn * N * 3 * 8, cudaMemcpyHostToDevice, st));
      rc = w.r;
    }
    if (int e = pn_forward_chunk<R>(ds, net, w, rc, Wn, jet, st)) return e;
    if constexpr (sizeof(R) == 4) {
      if (guarded) {
        int nflag = 0;
        if (int e = guard_flag_chunk(ds, net, w, *g, Wn, &nflag, st)) return e;
        if (!batch || nflag > g->cap) {
          if (int e = guard_reevaluate(ds, *g, g->list, nflag, rc, w.out_eloc, w.out_logabs, w.out_sign, w.out_status,
                                       w.out_grad, st))
            return e;
        } else if (nflag > 0) {
          if (pending + nflag > g->cap) {
            if (int e = guard_reevaluate(ds, *g, g->pend, pending, r, eloc, logabs, sign, status, nullptr, st)) return e;
            pending = 0;
          }
          PN_LAUNCH("k_guard_gather", st, k_guard_append<<<nblk(nflag, 128), 128, 0, st>>>(g->list, nflag, c0,
                                                                                          g->pend + pending));
          pending += nflag;
        }
      }
    }
    if (eloc && jet) PN_CUDA(cudaMemcpyAsync(eloc + c0, w.out_eloc, Wn * 8, cudaMemcpyDefault, st));
    if (logabs) PN_CUDA(cudaMemcpyAsync(logabs + c0, w.out_logabs, Wn * 8, cudaMemcpyDefault, st));
    if (sign) PN_CUDA(cudaMemcpyAsync(sign + c0, w.out_sign, Wn * 8, cudaMemcpyDefault, st));
    if (status) PN_CUDA(cudaMemcpyAsync(status + c0, w.out_status, Wn * 4, cudaMemcpyDefault, st));
  }
  if constexpr (sizeof(R) == 4) {
    if (pending > 0)
      if (int e = guard_reevaluate(ds, *g, g->pend, pending, r, eloc, logabs, sign, status, nullptr, st)) return e;
  }
  if (sync) PN_CUDA(cudaStreamSynchronize(st));
  return PN_OK;
}
template int pn_run_eval<double>(const DevSys&, const DevNet<double>&, Work<double>&, int, const double*, int, int,
                                 double*, double*, double*, int*, cudaStream_t, const Guard*);
template int pn_run_eval<float>(const DevSys&, const DevNet<float>&, Work<float>&, int, const double*, int, int,
                                double*, double*, double*, int*, cudaStream_t, const Guard*);

template <typename R>
int pn_run_metropolis(const DevSys& ds, const DevNet<R>& net, Work<R>& w, int Wc, double* r, double* logabs, int W,
                      int n_steps, double sigma, unsigned long long seed, unsigned long long step0, int64_t* n_accept,
                      cudaStream_t st) {
  const int N = ds.N;
  const bool rdev = pn_is_device_ptr(r), ldev = pn_is_device_ptr(logabs);
  PN_CUDA(cudaMemsetAsync(w.n_acc, 0, 8, st));
  for (int c0 = 0; c0 < W; c0 += Wc) {
    const int Wn = std::min(Wc, W - c0);
    double* rc = r + (size_t)c0 * N * 3;
    double* lc = logabs + c0;
    if (!rdev) {
      PN_CUDA(cudaMemcpyAsync(w.r, rc, (size_t)Wn * N * 3 * 8, cudaMemcpyHostToDevice, st));
      rc = w.r;
    }
    if (!ldev) {
      PN_CUDA(cudaMemcpyAsync(w.lp_prop, lc, (size_t)Wn * 8, cudaMemcpyHostToDevice, st));
      lc = w.lp_prop;
    }
    int fused = PN_ENOTREADY;
    if constexpr (sizeof(R) == 4) {
      if (ds.fused_sampler == 4)
        fused = pn_run_metropolis_tc(ds, net, rc, lc, Wn, (unsigned)c0, n_steps, sigma, seed, step0, w.n_acc, st);
    }
    // where the tensor-core sampler does not fit, embeddings wider than 64
    // run faster through the staged value pass than through the fused
    // CUDA-core kernels (N2 shape, 16384 walkers: 26 vs 35 ms per step)
    const bool wide = ds.fused_sampler == 4 && ds.D > 64;
    if (fused == PN_ENOTREADY && ds.fused_sampler && !wide)
      fused = pn_run_metropolis_fused<R>(ds, net, rc, lc, Wn, (unsigned)c0, n_steps, sigma, seed, step0, w.n_acc, st);
    if (fused != PN_OK && fused != PN_ENOTREADY) return fused;
    for (int k = 0; fused != PN_OK && k < n_steps; ++k) {
      const unsigned long long step = step0 + (unsigned long long)k;
      PN_LAUNCH("k_propose", st, k_propose<<<nblk(Wn, 128), 128, 0, st>>>(rc, w.r_prop, Wn, N, (unsigned)c0, seed, step, sigma));
      if (int e = pn_forward_chunk<R>(ds, net, w, w.r_prop, Wn, 0, st)) return e;
      PN_LAUNCH("k_accept", st, k_accept<<<nblk(Wn, 128), 128, 0, st>>>(rc, lc, w.r_prop, w.out_logabs, Wn, N, (unsigned)c0, seed, step, w.n_acc));
    }
    if (!rdev) PN_CUDA(cudaMemcpyAsync(r + (size_t)c0 * N * 3, rc, (size_t)Wn * N * 3 * 8, cudaMemcpyDeviceToHost, st));
    if (!ldev) PN_CUDA(cudaMemcpyAsync(logabs + c0, lc, (size_t)Wn * 8, cudaMemcpyDeviceToHost, st));
  }
  if (n_accept) PN_CUDA(cudaMemcpyAsync(n_accept, w.n_acc, 8, cudaMemcpyDefault, st));
  if (!rdev || !ldev || is_host(n_accept)) PN_CUDA(cudaStreamSynchronize(st));
  return PN_OK;
}
template int pn_run_metropolis<double>(const DevSys&, const DevNet<double>&, Work<double>&, int, double*, double*, int,
                                       int, double, unsigned long long, unsigned long long, int64_t*, cudaStream_t);
template int pn_run_metropolis<float>(const DevSys&, const DevNet<float>&, Work<float>&, int, double*, double*, int,
                                      int, double, unsigned long long, unsigned long long, int64_t*, cudaStream_t);

// ln|psi| and grad_r ln|psi| (the Langevin drift) of a workspace chunk:
// by reverse mode on the system's tape when rev is given, else by the jet
// pass (which also forms E_loc).  Results land in w.out_logabs, w.out_grad.
template <typename R>
static int drift_of_chunk(pn_system_s* rev, const DevSys& ds, const DevNet<R>& net, Work<R>& w, const double* r,
                          int Wn, cudaStream_t st) {
  if (rev) return pn_drift_reverse<R>(rev, r, Wn, w.out_logabs, w.out_grad, st);
  return pn_forward_chunk<R>(ds, net, w, r, Wn, 1, st);
}

template <typename R>
int pn_run_drift(pn_system_s* rev, const DevSys& ds, const DevNet<R>& net, Work<R>& w, int Wc, const double* r, int W,
                 double* logabs, double* drift, cudaStream_t st) {
  const int N = ds.N;
  const bool rdev = pn_is_device_ptr(r);
  for (int c0 = 0; c0 < W; c0 += Wc) {
    const int Wn = std::min(Wc, W - c0);
    const double* rc = r + (size_t)c0 * N * 3;
    if (!rdev) {
      PN_CUDA(cudaMemcpyAsync(w.r, rc, (size_t)Wn * N * 3 * 8, cudaMemcpyHostToDevice, st));
      rc = w.r;
    }
    if (int e = drift_of_chunk<R>(rev, ds, net, w, rc, Wn, st)) return e;
    if (logabs) PN_CUDA(cudaMemcpyAsync(logabs + c0, w.out_logabs, Wn * 8, cudaMemcpyDefault, st));
    PN_CUDA(cudaMemcpyAsync(drift + (size_t)c0 * N * 3, w.out_grad, (size_t)Wn * N * 3 * 8, cudaMemcpyDefault, st));
  }
  if (!rdev || is_host(logabs) || is_host(drift)) PN_CUDA(cudaStreamSynchronize(st));
  return PN_OK;
}
template int pn_run_drift<double>(pn_system_s*, const DevSys&, const DevNet<double>&, Work<double>&, int, const double*,
                                  int, double*, double*, cudaStream_t);
template int pn_run_drift<float>(pn_system_s*, const DevSys&, const DevNet<float>&, Work<float>&, int, const double*, int,
                                 double*, double*, cudaStream_t);

// Langevin Metropolis-Hastings steps, staged per workspace chunk: propose,
// ln|psi'| and its gradient at the proposals (reverse mode when rev is
// given, else the jet pass), accept.  r, logabs and drift are device
// buffers, updated in place.
template <typename R>
int pn_run_langevin(pn_system_s* rev, const DevSys& ds, const DevNet<R>& net, Work<R>& w, int Wc, double* r, double* logabs,
                    double* drift, int W, int n_steps, double tau, unsigned long long seed, unsigned long long step0,
                    int64_t* n_accept, cudaStream_t st) {
  const int N = ds.N;
  PN_CUDA(cudaMemsetAsync(w.n_acc, 0, 8, st));
  for (int c0 = 0; c0 < W; c0 += Wc) {
    const int Wn = std::min(Wc, W - c0);
    double* rc = r + (size_t)c0 * N * 3;
    double* lc = logabs + c0;
    double* dc = drift + (size_t)c0 * N * 3;
    for (int k = 0; k < n_steps; ++k) {
      const unsigned long long step = step0 + (unsigned long long)k;
      PN_LAUNCH("k_langevin_propose", st,
                k_langevin_propose<<<nblk(Wn, 128), 128, 0, st>>>(ds, rc, dc, w.r_prop, w.lp_prop, Wn, (unsigned)c0,
                                                                  seed, step, tau));
      if (int e = drift_of_chunk<R>(rev, ds, net, w, w.r_prop, Wn, st)) return e;
      PN_LAUNCH("k_langevin_accept", st,
                k_langevin_accept<<<nblk(Wn, 128), 128, 0, st>>>(ds, rc, lc, dc, w.r_prop, w.out_logabs, w.out_grad,
                                                                 w.lp_prop, Wn, (unsigned)c0, seed, step, tau,
                                                                 w.n_acc));
    }
  }
  if (n_accept) PN_CUDA(cudaMemcpyAsync(n_accept, w.n_acc, 8, cudaMemcpyDefault, st));
  if (is_host(n_accept)) PN_CUDA(cudaStreamSynchronize(st));
  return PN_OK;
}
template int pn_run_langevin<double>(pn_system_s*, const DevSys&, const DevNet<double>&, Work<double>&, int, double*, double*,
                                     double*, int, int, double, unsigned long long, unsigned long long, int64_t*,
                                     cudaStream_t);
template int pn_run_langevin<float>(pn_system_s*, const DevSys&, const DevNet<float>&, Work<float>&, int, double*, double*, double*,
                                    int, int, double, unsigned long long, unsigned long long, int64_t*, cudaStream_t);

// E_loc, ln|psi| and sign along a line: npts points t0 .. t1 (inclusive) of
// electron e's position r0[e] + t dir, in workspace chunks.  r0 is staged in
// the workspace's proposal buffer, so nothing is allocated.
template <typename R>
int pn_run_line_scan(const DevSys& ds, const DevNet<R>& net, Work<R>& w, int Wc, const double* r0, int e,
                     const double dir[3], double t0, double t1, int npts, double* eloc, double* logabs, double* sign,
                     int* status, cudaStream_t st) {
  const int N = ds.N;
  PN_CUDA(cudaMemcpyAsync(w.r_prop, r0, (size_t)N * 3 * 8, cudaMemcpyDefault, st));
  const double dt = npts > 1 ? (t1 - t0) / (double)(npts - 1) : 0.0;
  for (int c0 = 0; c0 < npts; c0 += Wc) {
    const int Wn = std::min(Wc, npts - c0);
    PN_LAUNCH("k_line_positions", st,
              k_line_positions<<<nblk(Wn, 128), 128, 0, st>>>(w.r_prop, N, e, dir[0], dir[1], dir[2], t0, dt, c0, Wn,
                                                              w.r));
    if (int er = pn_forward_chunk<R>(ds, net, w, w.r, Wn, 1, st)) return er;
    if (eloc) PN_CUDA(cudaMemcpyAsync(eloc + c0, w.out_eloc, Wn * 8, cudaMemcpyDefault, st));
    if (logabs) PN_CUDA(cudaMemcpyAsync(logabs + c0, w.out_logabs, Wn * 8, cudaMemcpyDefault, st));
    if (sign) PN_CUDA(cudaMemcpyAsync(sign + c0, w.out_sign, Wn * 8, cudaMemcpyDefault, st));
    if (status) PN_CUDA(cudaMemcpyAsync(status + c0, w.out_status, Wn * 4, cudaMemcpyDefault, st));
  }
  if (is_host(eloc) || is_host(logabs) || is_host(sign) || is_host(status) || !pn_is_device_ptr(r0))
    PN_CUDA(cudaStreamSynchronize(st));
  return PN_OK;
}
template int pn_run_line_scan<double>(const DevSys&, const DevNet<double>&, Work<double>&, int, const double*, int,
                                      const double[3], double, double, int, double*, double*, double*, int*,
                                      cudaStream_t);
template int pn_run_line_scan<float>(const DevSys&, const DevNet<float>&, Work<float>&, int, const double*, int,
                                     const double[3], double, double, int, double*, double*, double*, int*,
                                     cudaStream_t);

int pn_run_init_walkers(const DevSys& ds, double* r, int W, unsigned long long seed, cudaStream_t st) {
  PN_LAUNCH("k_init_walkers", st, k_init_walkers<<<nblk(W, 128), 128, 0, st>>>(ds, ds.nuc, r, W, seed));
  return PN_OK;
}

// ------------------------------------------------------------------- C ABI
#define PN_SYS_CHECK(s)                                   \
  do {                                                    \
    if (!(s)) { pn_set_error("null system"); return PN_EINVAL; } \
    if (int e_ = set_device(s)) return e_;                \
  } while (0)

extern "C" int pn_eval_logpsi(pn_system_t s, const double* r, int W, double* logabs, double* sign, int* status,
                              void* stream) {
  PN_SYS_CHECK(s);
  if (W < 0 || (W > 0 && (!r || !logabs))) { pn_set_error("bad arguments"); return PN_EINVAL; }
  if (W == 0) return PN_OK;
  cudaStream_t st = (cudaStream_t)stream;
  return s->precision == PN_FP64 ? eval_impl<double>(s, r, W, 0, nullptr, logabs, sign, status, st)
                                 : eval_impl<float>(s, r, W, 0, nullptr, logabs, sign, status, st);
}

extern "C" int pn_eval_local_energy(pn_system_t s, const double* r, int W, double* eloc, double* logabs, double* sign,
                                    int* status, void* stream) {
  PN_SYS_CHECK(s);
  if (W < 0 || (W > 0 && (!r || !eloc))) { pn_set_error("bad arguments"); return PN_EINVAL; }
  if (W == 0) return PN_OK;
  cudaStream_t st = (cudaStream_t)stream;
  return s->precision == PN_FP64 ? eval_impl<double>(s, r, W, 1, eloc, logabs, sign, status, st)
                                 : eval_impl<float>(s, r, W, 1, eloc, logabs, sign, status, st);
}

extern "C" int pn_eval_components(pn_system_t s, const double* r, int W, double* phi, double* J, double* f, double* ld,
                                  void* stream) {
  PN_SYS_CHECK(s);
  if (W < 0 || (W > 0 && !r)) { pn_set_error("bad arguments"); return PN_EINVAL; }
  if (W == 0) return PN_OK;
  cudaStream_t st = (cudaStream_t)stream;
  return s->precision == PN_FP64 ? components_impl<double>(s, r, W, phi, J, f, ld, st)
                                 : components_impl<float>(s, r, W, phi, J, f, ld, st);
}

extern "C" int pn_metropolis_step(pn_system_t s, double* r, double* logabs, int W, int n_steps, double sigma,
                                  uint64_t seed, uint64_t step0, int64_t* n_accept, void* stream) {
  PN_SYS_CHECK(s);
  if (W < 0 || n_steps < 0 || !(sigma > 0) || (W > 0 && (!r || !logabs))) {
    pn_set_error("bad arguments");
    return PN_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (W == 0 || n_steps == 0) {
    if (n_accept) {
      int64_t z = 0;
      PN_CUDA(cudaMemcpyAsync(n_accept, &z, 8, cudaMemcpyDefault, st));
      PN_CUDA(cudaStreamSynchronize(st));
    }
    return PN_OK;
  }
  return s->precision == PN_FP64 ? metropolis_impl<double>(s, r, logabs, W, n_steps, sigma, seed, step0, n_accept, st)
                                 : metropolis_impl<float>(s, r, logabs, W, n_steps, sigma, seed, step0, n_accept, st);
}

extern "C" int pn_eval_drift(pn_system_t s, const double* r, int W, double* logabs, double* drift, void* stream) {
  PN_SYS_CHECK(s);
  if (W < 0 || (W > 0 && (!r || !drift))) {
    pn_set_error("bad arguments");
    return PN_EINVAL;
  }
  if (W == 0) return PN_OK;
  cudaStream_t st = (cudaStream_t)stream;
  pn_system_s* rev = s->drift_mode ? s : nullptr;
  return s->precision == PN_FP64
             ? pn_run_drift<double>(rev, s->ds, pn_devnet<double>(s), work_of<double>(s), s->Wc, r, W, logabs, drift, st)
             : pn_run_drift<float>(rev, s->ds, pn_devnet<float>(s), work_of<float>(s), s->Wc, r, W, logabs, drift, st);
}

extern "C" int pn_langevin_step(pn_system_t s, double* r, double* logabs, double* drift, int W, int n_steps,
                                double tau, uint64_t seed, uint64_t step0, int64_t* n_accept, void* stream) {
  PN_SYS_CHECK(s);
  if (W < 0 || n_steps < 0 || !(tau > 0) || (W > 0 && (!r || !logabs || !drift))) {
    pn_set_error("bad arguments");
    return PN_EINVAL;
  }
  if (W > 0 && (!pn_is_device_ptr(r) || !pn_is_device_ptr(logabs) || !pn_is_device_ptr(drift))) {
    pn_set_error("pn_langevin_step takes device buffers for r, logabs and drift");
    return PN_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (W == 0 || n_steps == 0) {
    if (n_accept) {
      int64_t z = 0;
      PN_CUDA(cudaMemcpyAsync(n_accept, &z, 8, cudaMemcpyDefault, st));
      PN_CUDA(cudaStreamSynchronize(st));
    }
    return PN_OK;
  }
  pn_system_s* rev = s->drift_mode ? s : nullptr;
  return s->precision == PN_FP64
             ? pn_run_langevin<double>(rev, s->ds, pn_devnet<double>(s), work_of<double>(s), s->Wc, r, logabs, drift, W,
                                       n_steps, tau, seed, step0, n_accept, st)
             : pn_run_langevin<float>(rev, s->ds, pn_devnet<float>(s), work_of<float>(s), s->Wc, r, logabs, drift, W,
                                      n_steps, tau, seed, step0, n_accept, st);
}

extern "C" int pn_eval_line_scan(pn_system_t s, const double* r0, int electron, const double* dir, double t0,
                                 double t1, int npts, double* eloc, double* logabs, double* sign, int* status,
                                 void* stream) {
  PN_SYS_CHECK(s);
  if (npts < 0 || (npts > 0 && (!r0 || !dir || !eloc)) || electron < 0 || electron >= s->ds.N ||
      !std::isfinite(t0) || !std::isfinite(t1)) {
    pn_set_error("bad arguments");
    return PN_EINVAL;
  }
  if (npts == 0) return PN_OK;
  double d[3] = {dir[0], dir[1], dir[2]};  // dir is a host array
  cudaStream_t st = (cudaStream_t)stream;
  return s->precision == PN_FP64
             ? pn_run_line_scan<double>(s->ds, pn_devnet<double>(s), work_of<double>(s), s->Wc, r0, electron, d, t0,
                                        t1, npts, eloc, logabs, sign, status, st)
             : pn_run_line_scan<float>(s->ds, pn_devnet<float>(s), work_of<float>(s), s->Wc, r0, electron, d, t0, t1,
                                       npts, eloc, logabs, sign, status, st);
}

extern "C" int pn_init_walkers(pn_system_t s, double* r, int W, uint64_t seed, void* stream) {
  PN_SYS_CHECK(s);
  if (W < 0 || (W > 0 && !r)) { pn_set_error("bad arguments"); return PN_EINVAL; }
  if (W == 0) return PN_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const DevSys& ds = s->ds;
  const bool rdev = pn_is_device_ptr(r);
  double* rd = r;
  if (!rdev) PN_CUDA(cudaMallocAsync((void**)&rd, (size_t)W * ds.N * 3 * 8, st));
  if (int e = pn_run_init_walkers(ds, rd, W, seed, st)) return e;
  if (!rdev) {
    PN_CUDA(cudaMemcpyAsync(r, rd, (size_t)W * ds.N * 3 * 8, cudaMemcpyDeviceToHost, st));
    PN_CUDA(cudaFreeAsync(rd, st));
  }
  PN_CUDA(cudaStreamSynchronize(st));
  return PN_OK;
}

extern "C" int pn_set_option(pn_system_t s, int option, int value) {
  if (!s) { pn_set_error("null system"); return PN_EINVAL; }
  switch (option) {
    case PN_OPT_FUSED_SAMPLER:
      if (value < 0 || value > 4) { pn_set_error("fused sampler option takes 0..4"); return PN_EINVAL; }
      s->ds.fused_sampler = value;
      return PN_OK;
    case PN_OPT_DRIFT:
      if (value < 0 || value > 1) { pn_set_error("drift option takes 0 (jet pass) or 1 (reverse mode)"); return PN_EINVAL; }
      s->drift_mode = value;
      return PN_OK;
    case PN_OPT_GUARD:
      if (value < 0) { pn_set_error("guard option takes tau in micro-hartree, 0 = off"); return PN_EINVAL; }
      if (value > 0 && !s->guard_mem) { pn_set_error("the local-energy guard exists for PN_MIXED handles only"); return PN_EINVAL; }
      s->guard.tau = value * 1e-6;
      return PN_OK;
    case PN_OPT_GUARD_PROBE:
      if (value < 0 || value > 2) { pn_set_error("guard probe option takes 0, 1 or 2"); return PN_EINVAL; }
      s->ds.guard_probe = value;
      return PN_OK;
    case PN_OPT_DET_TABLE:
      if (value < 0 || value > 2) { pn_set_error("determinant option takes 0..2"); return PN_EINVAL; }
      s->ds.no_table = value == 1 ? 0 : (value == 0 ? 1 : 2);
      return PN_OK;
    case PN_OPT_TENSOR_CORES:
      if (value < 0 || value > 7) { pn_set_error("tensor-core option takes a mask 0..7"); return PN_EINVAL; }
      s->ds.tensor_cores = value;
      return PN_OK;
    default:
      pn_set_error("unknown option %d", option);
      return PN_EINVAL;
  }
}

extern "C" int pn_device_status(pn_system_t s) {
  if (!s) { pn_set_error("null system"); return PN_EINVAL; }
  PN_CUDA(cudaDeviceSynchronize());
  int h = 0;
  PN_CUDA(cudaMemcpy(&h, s->ds.dev_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    const int zero = 0;
    PN_CUDA(cudaMemcpy(s->ds.dev_err, &zero, sizeof(int), cudaMemcpyHostToDevice));
    pn_set_error("a bounded device wait expired (tensor-core completion)");
    return PN_ETIMEOUT;
  }
  return PN_OK;
}

extern "C" int pn_clip_local_energy(const double* eloc, int W, double q, double* out, double* cot, void* stream) {
  if (W <= 0 || W > (1 << 26) || !eloc || !out || !(q > 0)) {
    pn_set_error("clip: need 0 < W <= 2^26, q > 0 and buffers");
    return PN_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const bool host = is_host(eloc) || is_host(out) || is_host(cot);
  const double* e = eloc;
  double *o = out, *c = cot, *tmp = nullptr;
  if (host) {
    PN_CUDA(cudaMallocAsync((void**)&tmp, (size_t)W * 3 * 8, st));
    PN_CUDA(cudaMemcpyAsync(tmp, eloc, (size_t)W * 8, cudaMemcpyDefault, st));
    e = tmp;
    o = tmp + W;
    c = cot ? tmp + 2 * W : nullptr;
  }
  int n = 1;
  while (n < W) n <<= 1;
  if (W <= 16384) {
    const size_t smem = (size_t)n * 8;
    PN_CUDA(pn_allow_max_smem(k_clip));
    PN_LAUNCH("k_clip", st, k_clip<<<1, 1024, smem, st>>>(e, W, q, o, c));
  } else {
    unsigned long long* key = nullptr;
    PN_CUDA(cudaMallocAsync((void**)&key, (size_t)n * 8, st));
    PN_LAUNCH("k_clip", st, k_clip_keys<<<nblk(n, 256), 256, 0, st>>>(e, W, n, key));
    for (int k = 2; k <= n; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1)
        PN_LAUNCH("k_clip", st, k_bitonic_step<<<nblk(n, 256), 256, 0, st>>>(key, n, j, k));
    PN_LAUNCH("k_clip", st, k_clip_stats<<<1, 1024, 0, st>>>(key, e, W, q, o, c));
    PN_CUDA(cudaFreeAsync(key, st));
  }
  if (host) {
    PN_CUDA(cudaMemcpyAsync(out, o, (size_t)W * 8, cudaMemcpyDefault, st));
    if (cot) PN_CUDA(cudaMemcpyAsync(cot, c, (size_t)W * 8, cudaMemcpyDefault, st));
    PN_CUDA(cudaFreeAsync(tmp, st));
    PN_CUDA(cudaStreamSynchronize(st));
  }
  return PN_OK;
}

extern "C" int pn_guard_count(pn_system_t s, int64_t* n) {
  if (!s || !n) { pn_set_error("bad arguments"); return PN_EINVAL; }
  *n = 0;
  if (!s->guard_mem) return PN_OK;
  if (int e = set_device(s)) return e;
  PN_CUDA(cudaDeviceSynchronize());
  PN_CUDA(cudaMemcpy(n, s->guard.n_total, 8, cudaMemcpyDeviceToHost));
  PN_CUDA(cudaMemset(s->guard.n_total, 0, 8));
  return PN_OK;
}
