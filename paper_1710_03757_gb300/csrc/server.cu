// Serving loop: continuous batching of Monte Carlo TRG estimate jobs.
//
// Jobs (beta, h, L, chi, target standard error of ln Z) arrive at any time.
// A pool of workers (slots), each with its own CUDA stream and a persistent
// context, takes queued jobs as soon as a slot is free AND the job's device
// footprint fits the memory the server has not yet handed out: admission by
// HBM footprint.  A job's footprint is the memory plan of its largest round
// (the same planner mctrg_footprint reports, from the largest leg dimensions
// the lattice can have, so it bounds what the context allocates); a worker
// keeps the buffers of the jobs it ran (cudaFree would wait for the whole
// device and serialize every running job) and counts them against the
// budget, and idle workers give theirs back only when a queued job is blocked
// on memory.  A job advances in rounds of trajectories, so the kernels of
// all running jobs share the device on their streams; after each round the
// standard error of ln Z is projected to max_samples by the 1/sqrt(N) law
// (Sec. V, Eq. shrunkDev) and a job that cannot reach its target stops with
// EUNREACHABLE.  A job's trajectory i always uses Philox counter i under the
// job's seed and its rounds merge through the sufficient statistics of
// mctrg_merge_estimates, so its result is the same alone and in any mix.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/mctrg.h"
#include "mctrg_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  uint64_t id = 0;
  double beta = 0, h = 0, target = 0;
  int L = 0, chi = 0;
  int64_t max_samples = 0, round0 = 0;
  uint64_t seed = 0;
  size_t footprint = 0;     // device bytes of the largest round (plan bound)
  int passed_over = 0;      // times a later job was admitted while this one waited for memory
  Clock::time_point t_submit, t_done;
  int state = 0;            // 0 queued, 1 running, 2 done
  int status = MCTRG_OK;
  mctrg_estimate est{};
};

struct Worker {
  mctrg_ctx_t ctx = nullptr;
  size_t held = 0;          // bytes counted against the budget for this worker
  bool release = false;     // give the buffers back before the next job
};

constexpr int64_t kRoundMax = 8192;   // rounds double from the first up to this
constexpr int kMaxPassOver = 32;      // then the oldest job blocks the queue until memory frees

}  // namespace

struct mctrg_server {
  mctrg_options opt{};
  size_t budget = 0;                // device bytes the server may hand out
  size_t reserved = 0;              // sum of the workers' held bytes
  int n_workers = 16;
  std::vector<Worker> w;
  std::mutex mu;
  std::condition_variable cv;       // workers wake on submit / stop / memory released
  std::condition_variable done_cv;  // waiters wake when a job finishes
  std::deque<Job*> queue;
  std::map<uint64_t, Job*> jobs;
  bool stop = false;
  std::atomic<bool> stop_flag{false};   // running jobs stop at their next round
  uint64_t next_id = 1;
  std::vector<std::thread> workers;

  // Under mu: the queued job worker wi may take now, or null.  The oldest job
  // that fits (its footprint beyond what the worker already holds, within the
  // unreserved budget); a job passed over kMaxPassOver times stops the others.
  Job* admit(int wi) {
    const size_t free_b = budget > reserved ? budget - reserved : 0;
    for (auto it = queue.begin(); it != queue.end(); ++it) {
      Job* j = *it;
      const size_t need = j->footprint > w[wi].held ? j->footprint - w[wi].held : 0;
      if (need <= free_b) {
        for (auto q = queue.begin(); q != it; ++q) ++(*q)->passed_over;
        reserved += need;
        w[wi].held += need;
        queue.erase(it);
        return j;
      }
      if (j->passed_over >= kMaxPassOver) break;
    }
    // the oldest job is blocked on memory: idle workers give their buffers back
    if (!queue.empty() && w[wi].held > 0) w[wi].release = true;
    return nullptr;
  }

  // One job on a worker's persistent context: rounds of trajectories until the
  // target standard error of ln Z is reached, projected out of reach, or
  // max_samples is spent.
  void run_job(mctrg_ctx_t ctx, Job* j) {
    int status = mctrg_init_lattice(ctx, j->beta, j->h, j->L, j->chi);
    mctrg_estimate total{};
    bool have = false, reached = false;
    int64_t done = 0, round = j->round0;
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
      if (j->target == 0.0) { round = std::min(round * 2, kRoundMax); continue; }   // fixed-sample job
      if (total.status == MCTRG_OK && total.se_ln_Z <= j->target) { reached = true; break; }
      // projection of the standard error to max_samples (1/sqrt(N)); a margin
      // of 2 absorbs the scatter of an early estimate of it.  A round whose
      // mean Z~ is not positive (EDOMAIN: ln Z^ undefined) or whose SE is not
      // finite projects as unbounded, so such a job stops after it too
      const double se = (total.status == MCTRG_OK && std::isfinite(total.se_ln_Z)) ? total.se_ln_Z : INFINITY;
      if (total.n >= std::min<int64_t>(64, j->round0) &&
          se * std::sqrt((double)total.n / (double)j->max_samples) > 2.0 * j->target)
        break;
      round = std::min(round * 2, kRoundMax);
    }
    if (status == MCTRG_OK && !reached && j->target > 0.0) status = MCTRG_EUNREACHABLE;
    std::lock_guard<std::mutex> lk(mu);
    j->est = total;
    j->status = status;
    j->t_done = Clock::now();
    j->state = 2;
    done_cv.notify_all();
  }

  void finish_failed(Job* j, int status) {
    std::lock_guard<std::mutex> lk(mu);
    j->status = status;
    j->t_done = Clock::now();
    j->state = 2;
    done_cv.notify_all();
  }

  void worker_loop(int wi) {
    cudaSetDevice(opt.device);
    cudaStream_t st = nullptr;
    mctrg_ctx_t ctx = nullptr;
    mctrg_options o = opt;
    o.profile = 0;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess) {
      o.cuda_stream = st;
      o.hbm_budget_bytes = budget;
      if (mctrg_create(&o, &ctx) != MCTRG_OK) ctx = nullptr;
    }
    for (;;) {
      Job* j = nullptr;
      bool release = false;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] {
          if (stop) return true;
          if (queue.empty()) return false;
          j = admit(wi);
          return j != nullptr || w[wi].release;
        });
        if (stop) break;
        if (!j) {                      // give the buffers back, then try again
          release = true;
          w[wi].release = false;
        } else {
          j->state = 1;
        }
      }
      if (release) {
        if (ctx) ctx->release_all();
        std::lock_guard<std::mutex> lk(mu);
        reserved -= w[wi].held;
        w[wi].held = 0;
        cv.notify_all();
        continue;
      }
      if (!ctx) { finish_failed(j, MCTRG_ECUDA); continue; }
      // the context plans its chunks within what this worker holds
      ctx->opt.hbm_budget_bytes = w[wi].held;
      run_job(ctx, j);
      std::lock_guard<std::mutex> lk(mu);
      const size_t actual = ctx->held_bytes();
      if (actual > w[wi].held) {       // the plan bound is exceeded only by the shared prefix
        reserved += actual - w[wi].held;
        w[wi].held = actual;
      }
      cv.notify_all();
    }
    if (ctx) mctrg_destroy(ctx);
    if (st) cudaStreamDestroy(st);
  }
};

extern "C" int mctrg_server_create(const mctrg_options* opt, mctrg_server_t* out) {
  if (!opt || !out) return MCTRG_EINVAL;
  if (opt->precision < MCTRG_FP64 || opt->precision > MCTRG_FP64TC || opt->deterministic_levels < 0)
    return MCTRG_EINVAL;
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
  s->w.resize(s->n_workers);
  for (int i = 0; i < s->n_workers; ++i) s->workers.emplace_back(&mctrg_server::worker_loop, s, i);
  *out = s;
  return MCTRG_OK;
}

// Trajectories of a job's first round: about 0.5 s of SVD work, at least 2
// (a standard error needs two) and at most 256, so that a job whose target is
// out of reach is projected so after one short round whatever its lattice.
// The work is the bidiagonal reduction's n^3 per matrix summed over the levels
// that each trajectory splits on its own (after the first sampled level, which
// is shared), with the Ising site tensor's bond dimensions (D_1 = 2: the level-0
// matrix has rank 2; then D' = min(chi, D^2)), at about 5e11 n^3 per second
// (measured on the 1024 x 1024, chi = 16 lattice).
static int64_t first_round(int L, int chi) {
  int m = 0;
  while ((1 << m) < L) ++m;
  double work = 0.0;
  int D = 2;
  bool sampled = false;
  for (int k = 0; k < 2 * m; ++k) {
    const double n = (double)D * D;
    if (sampled) work += (double)(((int64_t)L * L) >> k) * n * n * n;
    if (n > chi) sampled = true;
    D = k == 0 ? 2 : std::min(chi, D * D);
  }
  if (work <= 0.0) return 256;
  return std::max<int64_t>(2, std::min<int64_t>(256, (int64_t)(2.5e11 / work)));
}

extern "C" int mctrg_server_submit(mctrg_server_t s, double beta, double h, int L, int chi,
                                   double target_se_lnZ, int64_t max_samples, uint64_t seed,
                                   uint64_t* job_id) {
  if (!s || !job_id) return MCTRG_EINVAL;
  if (L < 2 || (L & (L - 1)) || L > 65536 || chi < 1 || chi > mctrg::kMaxChi || !(beta >= 0) ||
      !std::isfinite(beta) || !std::isfinite(h) || !(target_se_lnZ >= 0) || max_samples < 1 ||
      (uint64_t)max_samples > (1ull << 32))
    return MCTRG_EINVAL;
  Job* j = new Job();
  j->beta = beta; j->h = h; j->L = L; j->chi = chi; j->target = target_se_lnZ;
  j->max_samples = max_samples; j->seed = seed;
  j->round0 = first_round(L, chi);
  // footprint of the largest round within half the budget (so that other jobs
  // run beside it); a job of which not even one trajectory fits the whole
  // budget can never run
  const int64_t Rmax = std::min<int64_t>(max_samples, kRoundMax);
  int64_t B = 0, S = 0;
  size_t total = 0;
  mctrg::plan_run_bound(L, chi, 2, s->opt, s->budget, 1, B, S, total);
  if (B < 1) {
    delete j;
    return MCTRG_EUNREACHABLE;
  }
  mctrg::plan_run_bound(L, chi, 2, s->opt, s->budget / 2, Rmax, B, S, total);
  if (B < 1) mctrg::plan_run_bound(L, chi, 2, s->opt, s->budget, Rmax, B, S, total);
  j->footprint = total;
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

extern "C" int mctrg_server_footprint(mctrg_server_t s, int L, int chi, int64_t max_samples, size_t* bytes) {
  if (!s || !bytes || L < 2 || (L & (L - 1)) || L > 65536 || chi < 1 || chi > mctrg::kMaxChi || max_samples < 1)
    return MCTRG_EINVAL;
  int64_t B = 0, S = 0;
  size_t total = 0;
  mctrg::plan_run_bound(L, chi, 2, s->opt, s->budget, 1, B, S, total);
  if (B < 1) return MCTRG_EUNREACHABLE;
  mctrg::plan_run_bound(L, chi, 2, s->opt, s->budget / 2, std::min<int64_t>(max_samples, kRoundMax), B, S,
                        total);
  if (B < 1)
    mctrg::plan_run_bound(L, chi, 2, s->opt, s->budget, std::min<int64_t>(max_samples, kRoundMax), B, S, total);
  *bytes = total;
  return MCTRG_OK;
}

extern "C" int mctrg_server_memory(mctrg_server_t s, size_t* budget, size_t* reserved) {
  if (!s) return MCTRG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (budget) *budget = s->budget;
  if (reserved) *reserved = s->reserved;
  return MCTRG_OK;
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
    if (t.joinable()) t.join();   // running jobs finish their current round first
  for (auto& kv : s->jobs) delete kv.second;
  s->jobs.clear();
  delete s;
}
