// Serving loop: continuous batching of Monte Carlo TRG estimate jobs.
//
// Jobs (beta, h, L, chi, target standard error of ln Z) arrive at any time.
// A fixed pool of workers, each with its own CUDA stream and a persistent
// context holding an equal share of the device-memory budget, takes queued
// jobs in arrival order as soon as a worker is free; a job advances in rounds
// of trajectories (chunked to fit its worker's memory), so the kernels of all
// running jobs share the device concurrently, and a worker that finishes a
// job immediately starts the next queued one with the buffers it already
// holds.  A job's
// trajectory i always uses Philox counter i under the job's seed and its
// rounds merge through the sufficient statistics of mctrg_merge_estimates,
// so its result is the same alone and in any mix.
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "../../include/mctrg.h"
#include "mctrg_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  uint64_t id = 0;
  double beta = 0, h = 0, target = 0;
  int L = 0, chi = 0;
  int64_t max_samples = 0;
  uint64_t seed = 0;
  size_t footprint = 0;
  Clock::time_point t_submit, t_done;
  int state = 0;            // 0 queued, 1 running, 2 done
  int status = MCTRG_OK;
  mctrg_estimate est{};
};

// Upper bound of the device bytes of a job that runs rounds of R trajectories:
// leg dimensions grow as D' = min(chi, D^2) from D = 2.
size_t job_footprint(int L, int chi, int64_t R) {
  int m = 0;
  while ((1 << m) < L) ++m;
  const int nlev = 2 * m;
  int D = 2;
  size_t per_traj = 64, work = 0, maxpair = 0, prevh = 0;
  for (int k = 0; k < nlev; ++k) {
    const size_t n = (size_t)D * D;
    const int kc = (int)std::min<size_t>((size_t)chi, n);
    const size_t N = ((size_t)L * L) >> k;
    const size_t hk = N * 2 * n * kc * 8;
    maxpair = std::max(maxpair, hk + prevh);
    prevh = hk;
    work = std::max(work, (size_t)(5 * n * n * 8 + (n + 1) * 65 * 8));
    D = kc;
  }
  per_traj += maxpair;
  // trajectories in flight, one matrix of working space, fixed buffers
  return per_traj * (size_t)R + work + (64u << 20);
}

}  // namespace

struct mctrg_server {
  mctrg_options opt{};
  size_t budget = 0;                // whole server
  size_t worker_budget = 0;         // each worker context
  int n_workers = 16;
  std::mutex mu;
  std::condition_variable cv;       // workers wake on submit / stop
  std::condition_variable done_cv;  // waiters wake when a job finishes
  std::deque<Job*> queue;
  std::map<uint64_t, Job*> jobs;
  bool stop = false;
  std::atomic<bool> stop_flag{false};   // running jobs stop at their next round
  uint64_t next_id = 1;
  std::vector<std::thread> workers;

  static constexpr int64_t kRound0 = 256;   // first round; later rounds double up to kRoundMax
  static constexpr int64_t kRoundMax = 8192;

  // One job on a worker's persistent context: rounds of trajectories until the
  // target standard error of ln Z or max_samples is reached.
  void run_job(mctrg_ctx_t ctx, Job* j) {
    int status = mctrg_init_lattice(ctx, j->beta, j->h, j->L, j->chi);
    mctrg_estimate total{};
    bool have = false;
    int64_t done = 0, round = kRound0;
    while (status == MCTRG_OK && done < j->max_samples) {
      if (stop_flag.load(std::memory_order_relaxed)) break;   // server shutting down
      const int64_t R = std::min(round, j->max_samples - done);
      mctrg_estimate e{};
      int s = mctrg_run(ctx, R, j->seed, (uint64_t)done, nullptr, nullptr, nullptr, &e);
      if (s != MCTRG_OK && s != MCTRG_EDOMAIN && s != MCTRG_ENOCONV) { status = s; break; }
      if (!have) { total = e; have = true; }
      else {
        mctrg_estimate parts[2] = {total, e};
        mctrg_merge_estimates(parts, 2, &total);
      }
      done += R;
      if (total.status == MCTRG_OK && total.se_ln_Z <= j->target) break;
      round = std::min(round * 2, kRoundMax);
    }
    if (status == MCTRG_OK && !(total.status == MCTRG_OK && total.se_ln_Z <= j->target))
      status = MCTRG_EUNREACHABLE;
    std::lock_guard<std::mutex> lk(mu);
    j->est = total;
    j->status = status;
    j->t_done = Clock::now();
    j->state = 2;
    done_cv.notify_all();
  }

  // A worker owns one stream and one context for its whole life, so jobs reuse
  // device buffers instead of allocating and freeing them (cudaFree waits for
  // the whole device, which would serialize every running job).
  void worker_loop() {
    cudaSetDevice(opt.device);
    cudaStream_t st = nullptr;
    mctrg_ctx_t ctx = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess) {
      mctrg_options o = opt;
      o.cuda_stream = st;
      o.hbm_budget_bytes = worker_budget;
      o.profile = 0;
      if (mctrg_create(&o, &ctx) != MCTRG_OK) ctx = nullptr;
    }
    for (;;) {
      Job* j = nullptr;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return stop || !queue.empty(); });
        if (stop) break;
        j = queue.front();
        queue.pop_front();
        j->state = 1;
      }
      if (ctx) {
        run_job(ctx, j);
      } else {
        std::lock_guard<std::mutex> lk(mu);
        j->status = MCTRG_ECUDA;
        j->t_done = Clock::now();
        j->state = 2;
        done_cv.notify_all();
      }
    }
    if (ctx) mctrg_destroy(ctx);
    if (st) cudaStreamDestroy(st);
  }
};

extern "C" int mctrg_server_create(const mctrg_options* opt, mctrg_server_t* out) {
  if (!opt || !out) return MCTRG_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) return MCTRG_ECUDA;
  if (opt->device < 0 || opt->device >= ndev) return MCTRG_EINVAL;
  if (cudaSetDevice(opt->device) != cudaSuccess) return MCTRG_ECUDA;
  mctrg_server* s = new mctrg_server();
  s->opt = *opt;
  if (s->opt.hbm_budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { delete s; return MCTRG_ECUDA; }
    s->opt.hbm_budget_bytes = (size_t)(0.8 * (double)fr);
  }
  s->budget = s->opt.hbm_budget_bytes;
  s->worker_budget = s->budget / (size_t)s->n_workers;
  for (int w = 0; w < s->n_workers; ++w) s->workers.emplace_back(&mctrg_server::worker_loop, s);
  *out = s;
  return MCTRG_OK;
}

extern "C" int mctrg_server_submit(mctrg_server_t s, double beta, double h, int L, int chi,
                                   double target_se_lnZ, int64_t max_samples, uint64_t seed,
                                   uint64_t* job_id) {
  if (!s || !job_id) return MCTRG_EINVAL;
  if (L < 2 || (L & (L - 1)) || L > 65536 || chi < 1 || chi > 32 || !(beta >= 0) ||
      !std::isfinite(beta) || !std::isfinite(h) || !(target_se_lnZ > 0) || max_samples < 1 ||
      (uint64_t)max_samples > (1ull << 32))
    return MCTRG_EINVAL;
  Job* j = new Job();
  j->beta = beta; j->h = h; j->L = L; j->chi = chi; j->target = target_se_lnZ;
  j->max_samples = max_samples; j->seed = seed;
  // a job runs in chunks that fit a worker's share of the memory; if even one
  // trajectory cannot fit there, it can never run
  j->footprint = job_footprint(L, chi, 1);
  if (j->footprint > s->worker_budget) {
    delete j;
    return MCTRG_EUNREACHABLE;
  }
  j->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  j->id = s->next_id++;
  s->jobs[j->id] = j;
  s->queue.push_back(j);
  *job_id = j->id;
  s->cv.notify_all();
  return MCTRG_OK;
}

static int take_result(mctrg_server* s, std::map<uint64_t, Job*>::iterator it, mctrg_estimate* est,
                       double* latency_s) {
  Job* j = it->second;
  if (est) *est = j->est;
  if (latency_s) *latency_s = std::chrono::duration<double>(j->t_done - j->t_submit).count();
  const int st = j->status;
  s->jobs.erase(it);
  delete j;
  return st;
}

extern "C" int mctrg_server_poll(mctrg_server_t s, uint64_t job_id, mctrg_estimate* est, double* latency_s) {
  if (!s) return MCTRG_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return MCTRG_ENOTFOUND;
  if (it->second->state != 2) return MCTRG_EAGAIN;
  return take_result(s, it, est, latency_s);
}

extern "C" int mctrg_server_wait(mctrg_server_t s, uint64_t job_id, double timeout_s, mctrg_estimate* est,
                                 double* latency_s) {
  if (!s) return MCTRG_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(std::max(0.0, timeout_s)));
  for (;;) {
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return MCTRG_ENOTFOUND;
    if (it->second->state == 2) return take_result(s, it, est, latency_s);
    if (s->done_cv.wait_until(lk, deadline) == std::cv_status::timeout) {
      it = s->jobs.find(job_id);
      if (it != s->jobs.end() && it->second->state == 2) return take_result(s, it, est, latency_s);
      return MCTRG_ETIMEDOUT;
    }
  }
}

extern "C" void mctrg_server_destroy(mctrg_server_t s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->stop_flag.store(true);
    // queued jobs never start
    for (Job* j : s->queue) { s->jobs.erase(j->id); delete j; }
    s->queue.clear();
    s->cv.notify_all();
  }
  for (std::thread& t : s->workers)
    if (t.joinable()) t.join();   // running jobs finish their current job first
  for (auto& kv : s->jobs) delete kv.second;
  s->jobs.clear();
  delete s;
}
