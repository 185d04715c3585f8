// Serving loop: continuous batching of local-energy and sampling jobs for
// molecules of different sizes.
//
// A scheduler thread admits queued jobs as soon as a slot is free and the
// job's device footprint fits the remaining memory budget (jobs further back
// may be admitted past one that does not fit yet).  Each slot has its own
// CUDA stream and its own host thread: the slot thread takes the job's
// workspace from the stream-ordered allocator on the slot's stream, enqueues
// all of the job's work there, and waits for it, so jobs on different slots
// overlap on the GPU and a wait inside one job (the mixed local-energy
// guard reads one count per chunk) holds up no other slot.  A job's result
// depends only on its own inputs, seed and chunk size -- not on which other
// jobs run beside it -- so a result is the same alone and in a mix.  Each
// job's first and last device work is bracketed by CUDA events, reported
// relative to the server's creation, so that overlap is observable.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "pn_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

// Per-job statistics of the local energies: finite walkers' sum and sum of
// squares, and the count of the others.  One block.
__global__ void k_job_stats(const double* __restrict__ E, const int* __restrict__ status, int W,
                            const unsigned long long* __restrict__ n_acc, double* __restrict__ out) {
  __shared__ double s1[256], s2[256], sc[256];
  double a = 0, b = 0, c = 0;
  for (int i = threadIdx.x; i < W; i += blockDim.x) {
    const double e = E[i];
    if (status[i] == PN_WALKER_OK && isfinite(e)) {
      a += e;
      b += e * e;
      c += 1;
    }
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  sc[threadIdx.x] = c;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
      sc[threadIdx.x] += sc[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s1[0];
    out[1] = s2[0];
    out[2] = sc[0];
    out[3] = n_acc ? (double)*n_acc : 0.0;
  }
}

enum JobState { QUEUED, RUNNING, DONE };

struct JobRec {
  uint64_t id;
  pn_system_t sys;
  pn_job job;
  JobState state = QUEUED;
  pn_result res{};
  size_t footprint = 0;
  int slot = -1;
  Clock::time_point t_submit, t_admit, t_done;
  void* mem = nullptr;
};

struct Slot {
  cudaStream_t st = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;  // the job's first and last device work
  double* stats_host = nullptr;            // pinned [4]
  std::shared_ptr<JobRec> job;             // assigned by the scheduler, cleared when done
  std::thread thr;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct pn_server_s {
  pn_server_cfg cfg;
  int device = 0;
  cudaEvent_t t_ref = nullptr;  // recorded at creation: origin of the device times
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_slot;
  std::deque<std::shared_ptr<JobRec>> queue;
  std::map<uint64_t, std::shared_ptr<JobRec>> jobs;
  size_t used = 0;
  uint64_t next_id = 1;
  int admitted = 0;
  bool stop = false;
  std::thread worker;
};

// Walkers per float64 re-evaluation of a serving job's local-energy guard.
constexpr int kGuardCap = 256;

static size_t job_bytes(pn_system_t s, int W, int chunk, size_t* work_bytes, int* Wc, size_t* guard_bytes = nullptr) {
  const DevSys& ds = s->ds;
  const int wc = std::max(1, std::min(W, chunk));
  const int elem = s->precision == PN_FP64 ? 8 : 4;
  const size_t wb = pn_work_bytes(ds, wc, 3 * ds.N + 2, elem);
  // mixed jobs carry the local-energy guard of their own
  const size_t gb = s->precision == PN_MIXED ? pn_guard_bytes(ds, wc, std::min(wc, kGuardCap)) : 0;
  if (work_bytes) *work_bytes = wb;
  if (Wc) *Wc = wc;
  if (guard_bytes) *guard_bytes = gb;
  // workspace + guard + positions, ln|psi|, E_loc, status, statistics
  return align256(wb) + align256(gb) + align256((size_t)W * ds.N * 3 * 8) + 2 * align256((size_t)W * 8) +
         align256((size_t)W * 4) + align256(64) + 4096;
}

extern "C" size_t pn_job_footprint(pn_system_t s, int W, int chunk_walkers) {
  if (!s || W <= 0) return 0;
  return job_bytes(s, W, chunk_walkers > 0 ? chunk_walkers : W, nullptr, nullptr);
}

// Enqueue every step of one job on its slot's stream.
template <typename R>
static int launch_job(pn_server_s* srv, Slot& sl, JobRec& j) {
  pn_system_t s = j.sys;
  const DevSys& ds = s->ds;
  const int W = j.job.W;
  cudaStream_t st = sl.st;
  size_t wb, gb;
  int Wc;
  const size_t total = job_bytes(s, W, srv->cfg.chunk_walkers, &wb, &Wc, &gb);
  PN_CUDA(cudaEventRecord(sl.t0, st));
  PN_CUDA(cudaMallocAsync(&j.mem, total, st));
  char* p = (char*)j.mem;
  Work<R> w = pn_carve_work<R>(ds, Wc, 3 * ds.N + 2, p);
  p += align256(wb);
  Guard guard{};
  const Guard* g = nullptr;
  if (gb) {
    guard = pn_carve_guard(ds, Wc, std::min(Wc, kGuardCap), p);
    guard.net64 = pn_devnet<double>(s);
    guard.tau = s->guard.tau;
    PN_CUDA(cudaMemsetAsync(guard.n_total, 0, 8, st));
    if (guard.tau > 0) g = &guard;
  }
  p += align256(gb);
  double* r = (double*)p; p += align256((size_t)W * ds.N * 3 * 8);
  double* lp = (double*)p; p += align256((size_t)W * 8);
  double* E = (double*)p; p += align256((size_t)W * 8);
  int* stat = (int*)p; p += align256((size_t)W * 4);
  double* stats = (double*)p;
  const DevNet<R> net = pn_devnet<R>(s);
  if (j.job.kind == PN_JOB_SCAN) {
    // E_loc along the line; the configurations live only in the workspace
    if (int e = pn_run_line_scan<R>(ds, net, w, Wc, j.job.r_init, j.job.scan_electron, j.job.scan_dir, j.job.scan_t0,
                                    j.job.scan_t1, W, E, nullptr, nullptr, stat, st))
      return e;
    PN_LAUNCH("k_job_stats", st, k_job_stats<<<1, 256, 0, st>>>(E, stat, W, nullptr, stats));
    PN_CUDA(cudaMemcpyAsync(sl.stats_host, stats, 4 * 8, cudaMemcpyDeviceToHost, st));
    if (j.job.eloc_out) PN_CUDA(cudaMemcpyAsync(j.job.eloc_out, E, (size_t)W * 8, cudaMemcpyDefault, st));
    PN_CUDA(cudaFreeAsync(j.mem, st));
    j.mem = nullptr;
    PN_CUDA(cudaEventRecord(sl.t1, st));
    return PN_OK;
  }
  if (j.job.r_init)
    PN_CUDA(cudaMemcpyAsync(r, j.job.r_init, (size_t)W * ds.N * 3 * 8, cudaMemcpyDefault, st));
  else if (int e = pn_run_init_walkers(ds, r, W, j.job.seed, st))
    return e;
  const unsigned long long* acc = nullptr;
  if (j.job.kind == PN_JOB_SWEEP && j.job.n_steps > 0) {
    if (int e = pn_run_eval<R>(ds, net, w, Wc, r, W, 0, nullptr, lp, nullptr, nullptr, st)) return e;
    if (int e = pn_run_metropolis<R>(ds, net, w, Wc, r, lp, W, j.job.n_steps, j.job.sigma, j.job.seed, 0, nullptr, st))
      return e;
    acc = w.n_acc;
  }
  if (int e = pn_run_eval<R>(ds, net, w, Wc, r, W, 1, E, nullptr, nullptr, stat, st, g)) return e;
  PN_LAUNCH("k_job_stats", st, k_job_stats<<<1, 256, 0, st>>>(E, stat, W, acc, stats));
  PN_CUDA(cudaMemcpyAsync(sl.stats_host, stats, 4 * 8, cudaMemcpyDeviceToHost, st));
  if (j.job.eloc_out) PN_CUDA(cudaMemcpyAsync(j.job.eloc_out, E, (size_t)W * 8, cudaMemcpyDefault, st));
  if (j.job.r_out) PN_CUDA(cudaMemcpyAsync(j.job.r_out, r, (size_t)W * ds.N * 3 * 8, cudaMemcpyDefault, st));
  if (gb) PN_CUDA(cudaMemcpyAsync(&j.res.n_guarded, guard.n_total, 8, cudaMemcpyDeviceToHost, st));
  PN_CUDA(cudaFreeAsync(j.mem, st));
  j.mem = nullptr;
  PN_CUDA(cudaEventRecord(sl.t1, st));
  return PN_OK;
}

static double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

// Results of the job on slot sl (called with srv->mu held).
static void finish(pn_server_s* srv, Slot& sl, int status) {
  JobRec& j = *sl.job;
  j.t_done = Clock::now();
  j.res.status = status;
  j.res.W = j.job.W;
  if (status == PN_OK) {
    const double* h = sl.stats_host;
    const double n = h[2];
    j.res.e_mean = n > 0 ? h[0] / n : NAN;
    const double var = n > 1 ? (h[1] - h[0] * h[0] / n) / (n - 1) : NAN;
    j.res.e_stderr = n > 1 ? sqrt(fmax(var, 0.0) / n) : NAN;
    j.res.n_nonfinite = (int64_t)j.job.W - (int64_t)n;
    j.res.accept_rate =
        (j.job.kind == PN_JOB_SWEEP && j.job.n_steps > 0) ? h[3] / ((double)j.job.W * j.job.n_steps) : 0.0;
    float a = 0, b = 0;
    if (cudaEventElapsedTime(&a, srv->t_ref, sl.t0) == cudaSuccess &&
        cudaEventElapsedTime(&b, srv->t_ref, sl.t1) == cudaSuccess) {
      j.res.dev_start_ms = a;
      j.res.dev_end_ms = b;
    }
    cudaGetLastError();
  }
  j.res.queue_ms = ms_between(j.t_submit, j.t_admit);
  j.res.run_ms = ms_between(j.t_admit, j.t_done);
  j.state = DONE;
  srv->used -= j.footprint;
  sl.job.reset();
}

// One slot's host thread: launch the assigned job on the slot's stream,
// wait for it, publish the result.
static void slot_loop(pn_server_s* srv, int k) {
  cudaSetDevice(srv->device);
  Slot& sl = srv->slots[k];
  std::unique_lock<std::mutex> lk(srv->mu);
  while (true) {
    srv->cv_slot.wait_for(lk, std::chrono::milliseconds(20), [&] { return srv->stop || (bool)sl.job; });
    if (!sl.job) {
      if (srv->stop) break;
      continue;
    }
    auto j = sl.job;
    lk.unlock();
    int rc;
    char tag[64];
    snprintf(tag, sizeof tag, "pn_job %llu slot %d", (unsigned long long)j->id, k);
    nvtxRangePushA(tag);
    if (j->res.status == PN_EDEVICE) {
      rc = PN_EDEVICE;  // injected host-side failure: nothing was launched
    } else {
      rc = j->sys->precision == PN_FP64 ? launch_job<double>(srv, sl, *j) : launch_job<float>(srv, sl, *j);
    }
    if (rc != PN_OK && j->mem) {
      cudaFreeAsync(j->mem, sl.st);
      j->mem = nullptr;
    }
    const cudaError_t e = cudaStreamSynchronize(sl.st);
    if (rc == PN_OK && e != cudaSuccess) {
      rc = PN_EDEVICE;
      pn_set_error("job stream: %s", cudaGetErrorString(e));
    }
    if (rc != PN_OK) {
      cudaGetLastError();
      // PN_SERVER_LOG=1: failed jobs' messages on stderr (the message is
      // thread-local to this slot's thread, so pn_last_error cannot show it)
      const char* log = getenv("PN_SERVER_LOG");
      if (log && log[0] == '1')
        fprintf(stderr, "pn_server: job %llu (slot %d) ended with status %d: %s\n", (unsigned long long)j->id, k, rc,
                pn_last_error());
    }
    nvtxRangePop();
    lk.lock();
    finish(srv, sl, rc);
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();
  }
}

// Admission: first-come order, later jobs may pass one that does not fit
// yet; a job goes to the first free slot.
static void worker_loop(pn_server_s* srv) {
  cudaSetDevice(srv->device);
  std::unique_lock<std::mutex> lk(srv->mu);
  while (true) {
    if (srv->stop && srv->queue.empty()) break;
    bool assigned = false;
    nvtxRangePushA("pn_server tick");
    if (!srv->stop) {
      for (auto it = srv->queue.begin(); it != srv->queue.end();) {
        Slot* free_slot = nullptr;
        int k = 0;
        for (auto& sl : srv->slots) {
          if (!sl.job) { free_slot = &sl; break; }
          ++k;
        }
        if (!free_slot) break;
        auto j = *it;
        if (srv->used + j->footprint > srv->cfg.hbm_budget_bytes) { ++it; continue; }
        it = srv->queue.erase(it);
        srv->used += j->footprint;
        j->state = RUNNING;
        j->slot = k;
        j->t_admit = Clock::now();
        ++srv->admitted;
        if (srv->cfg.debug_fail_nth > 0 && srv->admitted == srv->cfg.debug_fail_nth) {
          j->res.status = PN_EDEVICE;
          pn_set_error("injected failure of admitted job %d", srv->admitted);
        }
        free_slot->job = j;
        assigned = true;
      }
    }
    nvtxRangePop();
    if (assigned) srv->cv_slot.notify_all();
    srv->cv_work.wait_for(lk, std::chrono::milliseconds(20));
  }
}

extern "C" int pn_server_create(const pn_server_cfg* cfg, pn_server_t* out) {
  if (!cfg || !out || cfg->n_slots < 1 || cfg->n_slots > 64 || cfg->hbm_budget_bytes == 0 || cfg->chunk_walkers < 1) {
    pn_set_error("server config: need 1..64 slots, a budget and chunk_walkers >= 1");
    return PN_EINVAL;
  }
  auto* srv = new pn_server_s();
  srv->cfg = *cfg;
  cudaGetDevice(&srv->device);
  // keep the job workspaces freed by finished jobs in the stream-ordered
  // pool (up to the budget) instead of returning them to the driver at
  // every synchronisation; a per-process attribute of this device's pool
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, srv->device) == cudaSuccess) {
    uint64_t thr = cfg->hbm_budget_bytes;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  if (cudaEventCreate(&srv->t_ref) != cudaSuccess || cudaEventRecord(srv->t_ref, 0) != cudaSuccess ||
      cudaEventSynchronize(srv->t_ref) != cudaSuccess) {
    pn_set_error("server: reference event failed");
    return PN_EDEVICE;
  }
  srv->slots.resize(cfg->n_slots);
  for (auto& sl : srv->slots) {
    if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&sl.t0) != cudaSuccess || cudaEventCreate(&sl.t1) != cudaSuccess ||
        cudaMallocHost((void**)&sl.stats_host, 4 * 8) != cudaSuccess) {
      pn_set_error("server: stream/event/pinned buffer creation failed");
      return PN_EDEVICE;
    }
  }
  for (int k = 0; k < cfg->n_slots; ++k) srv->slots[k].thr = std::thread(slot_loop, srv, k);
  srv->worker = std::thread(worker_loop, srv);
  *out = srv;
  return PN_OK;
}

extern "C" int pn_server_destroy(pn_server_t srv) {
  if (!srv) return PN_OK;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
    for (auto& j : srv->queue) {
      j->state = DONE;
      j->res.status = PN_ECANCELLED;
    }
    srv->queue.clear();
  }
  srv->cv_work.notify_all();
  srv->worker.join();
  // the slots finish their running jobs, then see the stop flag
  while (true) {
    std::unique_lock<std::mutex> lk(srv->mu);
    bool busy = false;
    for (auto& sl : srv->slots) busy |= (bool)sl.job;
    if (!busy) break;
    srv->cv_done.wait_for(lk, std::chrono::milliseconds(20));
  }
  srv->cv_slot.notify_all();
  for (auto& sl : srv->slots) sl.thr.join();
  for (auto& sl : srv->slots) {
    cudaStreamSynchronize(sl.st);
    cudaEventDestroy(sl.t0);
    cudaEventDestroy(sl.t1);
    cudaStreamDestroy(sl.st);
    cudaFreeHost(sl.stats_host);
  }
  cudaEventDestroy(srv->t_ref);
  delete srv;
  return PN_OK;
}

extern "C" int pn_submit(pn_server_t srv, pn_system_t sys, const pn_job* job, uint64_t* job_id) {
  if (!srv || !sys || !job || !job_id || job->W < 1 || job->n_steps < 0 ||
      (job->kind != PN_JOB_ELOC && job->kind != PN_JOB_SWEEP && job->kind != PN_JOB_SCAN) ||
      (job->kind == PN_JOB_SWEEP && !(job->sigma > 0)) ||
      (job->kind == PN_JOB_SCAN && (!job->r_init || job->scan_electron < 0 || job->scan_electron >= sys->ds.N ||
                                    !std::isfinite(job->scan_t0) || !std::isfinite(job->scan_t1)))) {
    pn_set_error("submit: bad job");
    return PN_EINVAL;
  }
  auto j = std::make_shared<JobRec>();
  j->sys = sys;
  j->job = *job;
  j->footprint = job_bytes(sys, job->W, srv->cfg.chunk_walkers, nullptr, nullptr);
  if (j->footprint > srv->cfg.hbm_budget_bytes) {
    pn_set_error("submit: job needs %zu bytes, budget is %zu", j->footprint, srv->cfg.hbm_budget_bytes);
    return PN_EBUDGET;
  }
  j->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stop) { pn_set_error("submit: server is stopping"); return PN_EINVAL; }
    j->id = srv->next_id++;
    srv->jobs[j->id] = j;
    srv->queue.push_back(j);
    *job_id = j->id;
  }
  srv->cv_work.notify_all();
  return PN_OK;
}

extern "C" int pn_poll(pn_server_t srv, uint64_t id, pn_result* res, int64_t timeout_us) {
  if (!srv || !res) { pn_set_error("poll: null argument"); return PN_EINVAL; }
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->jobs.find(id);
  if (it == srv->jobs.end()) { pn_set_error("poll: unknown job %llu", (unsigned long long)id); return PN_EINVAL; }
  auto j = it->second;
  if (j->state != DONE) {
    if (timeout_us == 0) return PN_ENOTREADY;
    const auto deadline = Clock::now() + std::chrono::microseconds(timeout_us > 0 ? timeout_us : 0);
    while (j->state != DONE) {
      if (timeout_us > 0) {
        if (srv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && j->state != DONE) return PN_ETIMEOUT;
      } else {
        srv->cv_done.wait_for(lk, std::chrono::milliseconds(100));
      }
    }
  }
  *res = j->res;
  srv->jobs.erase(it);
  return PN_OK;
}

extern "C" int pn_cancel(pn_server_t srv, uint64_t id) {
  if (!srv) return PN_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->jobs.find(id);
  if (it == srv->jobs.end()) { pn_set_error("cancel: unknown job"); return PN_EINVAL; }
  auto j = it->second;
  if (j->state != QUEUED) return j->state == DONE ? PN_OK : PN_ENOTREADY;
  for (auto q = srv->queue.begin(); q != srv->queue.end(); ++q)
    if ((*q)->id == id) { srv->queue.erase(q); break; }
  j->state = DONE;
  j->res.status = PN_ECANCELLED;
  j->res.W = j->job.W;
  j->t_done = Clock::now();
  srv->cv_done.notify_all();
  return PN_OK;
}
