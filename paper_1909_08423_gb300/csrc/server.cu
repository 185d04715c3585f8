// Serving loop: continuous batching of local-energy and sampling jobs for
// molecules of different sizes.
//
// A host worker thread owns n_slots CUDA streams.  Jobs wait in a queue; a
// job is admitted as soon as a slot is free and its device footprint fits
// the remaining memory budget (jobs further back may be admitted past one
// that does not fit yet).  An admitted job gets its own workspace, taken
// from the stream-ordered allocator on its slot's stream, and all of its
// work is enqueued there, so jobs on different slots overlap on the GPU.
// A job's result depends only on its own inputs, seed and chunk size -- not
// on which other jobs run beside it -- so a result is bitwise the same
// alone and in a mix.  Completion is detected by polling CUDA events; every
// host wait is bounded.
#include <math.h>

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
  cudaEvent_t done = nullptr;
  double* stats_host = nullptr;  // pinned [4]
  std::shared_ptr<JobRec> job;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct pn_server_s {
  pn_server_cfg cfg;
  int device = 0;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<JobRec>> queue;
  std::map<uint64_t, std::shared_ptr<JobRec>> jobs;
  size_t used = 0;
  uint64_t next_id = 1;
  int admitted = 0;
  bool stop = false;
  std::thread worker;
};

static size_t job_bytes(pn_system_t s, int W, int chunk, size_t* work_bytes, int* Wc) {
  const DevSys& ds = s->ds;
  const int wc = std::max(1, std::min(W, chunk));
  const int elem = s->precision == PN_FP64 ? 8 : 4;
  const size_t wb = pn_work_bytes(ds, wc, 3 * ds.N + 2, elem);
  if (work_bytes) *work_bytes = wb;
  if (Wc) *Wc = wc;
  // workspace + positions, ln|psi|, E_loc, status, statistics
  return align256(wb) + align256((size_t)W * ds.N * 3 * 8) + 2 * align256((size_t)W * 8) + align256((size_t)W * 4) +
         align256(64) + 4096;
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
  size_t wb;
  int Wc;
  const size_t total = job_bytes(s, W, srv->cfg.chunk_walkers, &wb, &Wc);
  PN_CUDA(cudaMallocAsync(&j.mem, total, st));
  char* p = (char*)j.mem;
  Work<R> w = pn_carve_work<R>(ds, Wc, 3 * ds.N + 2, p);
  p += align256(wb);
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
    PN_CUDA(cudaEventRecord(sl.done, st));
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
  if (int e = pn_run_eval<R>(ds, net, w, Wc, r, W, 1, E, nullptr, nullptr, stat, st)) return e;
  PN_LAUNCH("k_job_stats", st, k_job_stats<<<1, 256, 0, st>>>(E, stat, W, acc, stats));
  PN_CUDA(cudaMemcpyAsync(sl.stats_host, stats, 4 * 8, cudaMemcpyDeviceToHost, st));
  if (j.job.eloc_out) PN_CUDA(cudaMemcpyAsync(j.job.eloc_out, E, (size_t)W * 8, cudaMemcpyDefault, st));
  if (j.job.r_out) PN_CUDA(cudaMemcpyAsync(j.job.r_out, r, (size_t)W * ds.N * 3 * 8, cudaMemcpyDefault, st));
  PN_CUDA(cudaFreeAsync(j.mem, st));
  j.mem = nullptr;
  PN_CUDA(cudaEventRecord(sl.done, st));
  return PN_OK;
}

static double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

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
  }
  j.res.queue_ms = ms_between(j.t_submit, j.t_admit);
  j.res.run_ms = ms_between(j.t_admit, j.t_done);
  j.state = DONE;
  srv->used -= j.footprint;
  sl.job.reset();
}

static void worker_loop(pn_server_s* srv) {
  cudaSetDevice(srv->device);
  std::unique_lock<std::mutex> lk(srv->mu);
  while (true) {
    bool progressed = false;
    // completions
    for (auto& sl : srv->slots) {
      if (!sl.job) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaSuccess) {
        finish(srv, sl, PN_OK);
        progressed = true;
      } else if (q != cudaErrorNotReady) {
        cudaGetLastError();
        finish(srv, sl, PN_EDEVICE);
        progressed = true;
      }
    }
    if (progressed) srv->cv_done.notify_all();
    if (srv->stop && srv->queue.empty()) {
      bool busy = false;
      for (auto& sl : srv->slots) busy |= (bool)sl.job;
      if (!busy) break;
    }
    // admissions: first-come order, later jobs may pass one that does not fit yet
    if (!srv->stop) {
      for (auto it = srv->queue.begin(); it != srv->queue.end();) {
        Slot* free_slot = nullptr;
        for (auto& sl : srv->slots)
          if (!sl.job) { free_slot = &sl; break; }
        if (!free_slot) break;
        auto j = *it;
        if (srv->used + j->footprint > srv->cfg.hbm_budget_bytes) { ++it; continue; }
        it = srv->queue.erase(it);
        srv->used += j->footprint;
        j->state = RUNNING;
        j->t_admit = Clock::now();
        free_slot->job = j;
        ++srv->admitted;
        int rc;
        if (srv->cfg.debug_fail_nth > 0 && srv->admitted == srv->cfg.debug_fail_nth) {
          rc = PN_EDEVICE;  // injected host-side failure: nothing was launched
          pn_set_error("injected failure of admitted job %d", srv->admitted);
        } else {
          rc = j->sys->precision == PN_FP64 ? launch_job<double>(srv, *free_slot, *j)
                                            : launch_job<float>(srv, *free_slot, *j);
        }
        if (rc != PN_OK) {
          if (j->mem) {
            cudaFreeAsync(j->mem, free_slot->st);
            j->mem = nullptr;
          }
          cudaStreamSynchronize(free_slot->st);
          cudaGetLastError();
          finish(srv, *free_slot, rc);
          srv->cv_done.notify_all();
        }
        progressed = true;
      }
    }
    if (!progressed) {
      bool busy = false;
      for (auto& sl : srv->slots) busy |= (bool)sl.job;
      // poll GPU completions every 50 us while jobs run, else sleep until work
      srv->cv_work.wait_for(lk, busy ? std::chrono::microseconds(50) : std::chrono::milliseconds(20));
    }
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
  srv->slots.resize(cfg->n_slots);
  for (auto& sl : srv->slots) {
    if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost((void**)&sl.stats_host, 4 * 8) != cudaSuccess) {
      pn_set_error("server: stream/event/pinned buffer creation failed");
      return PN_EDEVICE;
    }
  }
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
  for (auto& sl : srv->slots) {
    cudaStreamSynchronize(sl.st);
    cudaEventDestroy(sl.done);
    cudaStreamDestroy(sl.st);
    cudaFreeHost(sl.stats_host);
  }
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
