// Batching pattern: Monte Carlo TRG jobs of uneven lattice size and chi in
// one run, their levels advanced together so that the SVD stages of all jobs
// share launches.
//
// Every job keeps its own context (shared deterministic prefix, halves of its
// trajectories, per-trajectory accumulators).  The run proceeds in
// sub-batches: each takes, from every job that still has work, one segment of
// items (trajectory, tensor) of the job's current level, packed one after
// another into a workspace owned by the batch.  Per segment, the
// geometry-dependent kernels run with the job's own parameters: X and Yt of
// the plaquettes, the GEMM (FP64, or one of the tensor-core modes), the
// choice of the kept indices and the halves.  The bidiagonalization-route
// SVD of all segments (Householder reduction, bisection, kept vectors) runs
// as one launch per stage over a table of per-matrix descriptors, whatever
// the matrices' sizes, so small jobs fill the device together.  A job's level
// completes when all its items have passed; then its per-trajectory
// accumulation runs and the next level starts in a later sub-batch.
//
// Trajectory i of a job uses counter first_traj + i under the job's seed, and
// every kernel treats items independently, so each job's results are those
// of mctrg_run with the same arguments, bit for bit, whatever the mix.
//
// Sub-batch sizes: the SVD launches' item count per shape (n, route) and the
// sampler's CTA count are launch geometry with identical arithmetic.  They
// are chosen by timing candidates on the device (the autotuner below) and
// stored in the file options.autotune_cache, read back by later runs.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mctrg.h"
#include "common.cuh"
#include "kernels.h"
#include "kernels_bd.h"
#include "kernels_tc.h"
#include "mctrg_internal.h"

using namespace mctrg;

namespace {

#define BCK(call)                                   \
  do {                                              \
    cudaError_t e__ = (call);                       \
    if (e__ != cudaSuccess) {                       \
      set_last_cuda_error(e__);                     \
      return MCTRG_ECUDA;                           \
    }                                               \
  } while (0)

// ---- autotuner ------------------------------------------------------------
struct TuneKey {
  int n, kc;
  bool operator<(const TuneKey& o) const { return n != o.n ? n < o.n : kc < o.kc; }
};
struct TuneVal {
  int svd_items;      // matrices per SVD launch of this shape
  int sample_grid;    // CTAs of the sampler launches
};

std::mutex g_tune_mu;

// Cache file: one line per shape, "n kc svd_items sample_grid".
void read_cache(const char* path, std::map<TuneKey, TuneVal>& m) {
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  int n, kc, s, g;
  while (std::fscanf(f, "%d %d %d %d", &n, &kc, &s, &g) == 4)
    if (n > 0 && kc > 0 && s > 0 && g > 0) m[TuneKey{n, kc}] = TuneVal{s, g};
  std::fclose(f);
}

void write_cache(const char* path, const std::map<TuneKey, TuneVal>& m) {
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "w");
  if (!f) return;
  for (const auto& kv : m) std::fprintf(f, "%d %d %d %d\n", kv.first.n, kv.first.kc, kv.second.svd_items,
                                        kv.second.sample_grid);
  std::fclose(f);
}

// ---- per-job state ------------------------------------------------------------
struct JobRun {
  mctrg_ctx* ctx = nullptr;
  mctrg_job job{};
  int64_t B = 0;           // trajectories (one chunk)
  int k = 0;               // current level
  int64_t next = 0;        // next item of the level
  int64_t items = 0;       // items of the level
  int cur = 0, prev = 1;   // halves written / read at this level
  bool done = false;
};

// A segment of a sub-batch: items i0 .. i0+cnt-1 of job j's level k, at byte
// offset off of the workspace.
struct Segment {
  int j, k;
  int64_t i0, cnt;
  size_t off;
  bool bidiag;
};

size_t align_up(size_t b) { return (b + 255) & ~size_t(255); }

// A device buffer released when it goes out of scope.
struct OwnedBuf : DevBuf {
  ~OwnedBuf() { release(); }
};

// Uniform values in (-1, 1) from a counter hash (splitmix64), for the tuner's
// test matrices.
__global__ void k_fill_random(double* x, int64_t n, uint64_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    x[i] = (double)(int64_t)z * 0x1.0p-63;
  }
}

// Workspace bytes of one item of level k of a job (packed per segment).
struct ItemLayout {
  size_t x, m, w, bd, sig, perm, nnz, kept, sigt, nk, vrows, oz, ozexp, total;
};

ItemLayout layout(const mctrg_ctx* c, int k, int prec) {
  const LevelInfo& a = c->lv[k];
  const LevelInfo& p = c->lv[k - 1];
  const size_t n = a.n, np = a.n_pad, d2 = (size_t)p.D * p.D;
  ItemLayout L{};
  L.x = n * d2 * sizeof(double);
  L.m = n * n * sizeof(double);
  L.w = np * n * sizeof(double);
  L.bd = 3 * n * sizeof(double);
  L.sig = np * sizeof(double);
  L.perm = np * sizeof(int);
  L.nnz = sizeof(int);
  const size_t ks = kept_stride(c->chi);
  L.kept = ks * sizeof(int);
  L.sigt = ks * sizeof(double);
  L.nk = sizeof(int);
  L.vrows = ks * n * sizeof(double);
  L.oz = (prec == MCTRG_FP64TC && gemm_ozaki_supported((int)n, (int)d2)) ? 8 * n * d2 * 2 : 0;
  L.ozexp = L.oz ? n * sizeof(int) : 0;
  L.total = 2 * L.x + L.m + L.w + L.bd + L.sig + L.perm + L.nnz + L.kept + L.sigt + L.nk + L.vrows + 2 * L.oz +
            2 * L.ozexp;
  return L;
}

// Pointers of a segment's arrays inside the workspace (each array covers the
// segment's cnt items contiguously).
struct SegPtrs {
  double *X, *Y, *M, *W, *bd, *sig, *sigt, *vrows;
  int *perm, *nnz, *kept, *nk, *ezX, *ezY;
  void *ozX, *ozY;
};

SegPtrs carve(char* base, size_t off, const ItemLayout& L, int64_t cnt) {
  SegPtrs p{};
  size_t o = off;
  auto take = [&](size_t per) { char* q = base + o; o += align_up(per * (size_t)cnt); return q; };
  p.X = (double*)take(L.x);
  p.Y = (double*)take(L.x);
  p.M = (double*)take(L.m);
  p.W = (double*)take(L.w);
  p.bd = (double*)take(L.bd);
  p.sig = (double*)take(L.sig);
  p.perm = (int*)take(L.perm);
  p.nnz = (int*)take(L.nnz);
  p.kept = (int*)take(L.kept);
  p.sigt = (double*)take(L.sigt);
  p.nk = (int*)take(L.nk);
  p.vrows = (double*)take(L.vrows);
  if (L.oz) {
    p.ozX = take(L.oz);
    p.ozY = take(L.oz);
    p.ezX = (int*)take(L.ozexp);
    p.ezY = (int*)take(L.ozexp);
  }
  return p;
}

size_t segment_bytes(const ItemLayout& L, int64_t cnt) {
  size_t b = 0;
  const size_t per[] = {L.x, L.x, L.m, L.w, L.bd, L.sig, L.perm, L.nnz, L.kept, L.sigt, L.nk, L.vrows};
  for (size_t s : per) b += align_up(s * (size_t)cnt);
  if (L.oz) b += 2 * align_up(L.oz * (size_t)cnt) + 2 * align_up(L.ozexp * (size_t)cnt);
  return b;
}

}  // namespace

// ---------------------------------------------------------------------------
struct BatchRunner {
  mctrg_options opt{};
  cudaStream_t st = nullptr;
  std::vector<JobRun> jr;
  OwnedBuf ws, table, smp_scr, vec_scr, err;
  std::map<TuneKey, TuneVal> tune;
  bool tune_dirty = false;
  int64_t launches = 0;
  double zero_fp64(int n) const { return opt.zero_tol_scale * (double)n * 0x1.0p-52; }

  // ---- level s0: shared SVD, per-(trajectory, tensor) sampling --------------
  int start_job(JobRun& r) {
    mctrg_ctx* c = r.ctx;
    const int64_t B = r.B;
    BCK(c->o_lnabs.ensure(sizeof(double) * B));
    BCK(c->o_sign.ensure((size_t)B));
    BCK(c->o_flags.ensure((size_t)B));
    BCK(c->stats.ensure(8 * sizeof(double)));
    if (c->all_exact) { r.done = true; return MCTRG_OK; }
    size_t max_h = 0, max_items = 0;
    for (int k = c->s0; k < c->nlev; ++k) {
      const LevelInfo& a = c->lv[k];
      max_h = std::max(max_h, (size_t)B * a.N * 2 * a.n * a.kc);
      max_items = std::max(max_items, (size_t)B * a.N);
    }
    const LevelInfo& fl = c->lv[c->nlev - 1];
    BCK(c->Hbuf[0].ensure(sizeof(double) * max_h));
    BCK(c->Hbuf[1].ensure(sizeof(double) * max_h));
    BCK(c->iflags.ensure(sizeof(uint32_t) * max_items));
    BCK(c->ilns1.ensure(sizeof(double) * max_items));
    BCK(c->lnacc.ensure(sizeof(double) * B));
    BCK(c->o_tflags.ensure(sizeof(uint32_t) * B));
    BCK(c->Xb.ensure(sizeof(double) * (size_t)B * fl.kc * fl.kc * fl.n));
    BCK(c->Yb.ensure(sizeof(double) * (size_t)B * fl.kc * fl.kc * fl.n));
    const int g0 = sample_grid(c->lv[c->s0].n, c->chi);
    BCK(c->scratch.ensure(sizeof(double) * sample_scratch_doubles(c->lv[c->s0].n, c->chi, g0)));
    BCK(cudaMemsetAsync(c->lnacc.p, 0, sizeof(double) * B, st));
    BCK(cudaMemsetAsync(c->o_tflags.p, 0, sizeof(uint32_t) * B, st));
    const LevelInfo& a = c->lv[c->s0];
    const int64_t items = B * a.N;
    BCK(cudaMemsetAsync(c->iflags.p, 0, sizeof(uint32_t) * items, st));
    SampleArgs sa{};
    sa.M = c->shM.as<double>(); sa.W = c->shW.as<double>(); sa.sig = c->shSig.as<double>();
    sa.perm = c->shPerm.as<int>(); sa.nnz = c->shNnz.as<int>(); sa.Urows = c->shU.as<double>();
    sa.n = a.n; sa.n_pad = a.n_pad; sa.chi = c->chi; sa.kc = a.kc; sa.stochastic = 1; sa.shared_svd = 1;
    sa.item0 = 0; sa.n_items = items; sa.N = a.N; sa.L = c->L; sa.level = c->s0; sa.seed = r.job.seed;
    sa.traj0 = r.job.first_traj; sa.H = c->Hbuf[0].as<double>(); sa.h_item0 = 0;
    sa.iflags = c->iflags.as<uint32_t>(); sa.scratch = c->scratch.as<double>();
    BCK(launch_sample_split(sa, st, g0));
    BCK(launch_traj_accum(nullptr, c->iflags.as<uint32_t>(), a.N, B, c->lnacc.as<double>(),
                          c->o_tflags.as<uint32_t>(), st));
    launches += 2;
    r.cur = 0;
    return begin_level(r, c->s0 + 1);
  }

  int begin_level(JobRun& r, int k) {
    mctrg_ctx* c = r.ctx;
    if (k >= c->nlev) return finish_job(r);
    r.k = k;
    r.prev = r.cur;
    r.cur ^= 1;
    r.next = 0;
    r.items = r.B * c->lv[k].N;
    BCK(cudaMemsetAsync(c->iflags.p, 0, sizeof(uint32_t) * r.items, st));
    return MCTRG_OK;
  }

  int end_level(JobRun& r) {
    mctrg_ctx* c = r.ctx;
    const LevelInfo& a = c->lv[r.k];
    BCK(launch_traj_accum(c->ilns1.as<double>(), c->iflags.as<uint32_t>(), a.N, r.B, c->lnacc.as<double>(),
                          c->o_tflags.as<uint32_t>(), st));
    ++launches;
    return begin_level(r, r.k + 1);
  }

  // final contraction and trace of a job's trajectories
  int finish_job(JobRun& r) {
    mctrg_ctx* c = r.ctx;
    const LevelInfo& p = c->lv[c->nlev - 1];
    XYArgs xa{};
    xa.H = c->Hbuf[r.cur].as<double>(); xa.h_item0 = 0; xa.d = p.D; xa.D = p.kc; xa.c0 = 0;
    xa.n_items = r.B; xa.Nnew = 1; xa.Nold = p.N; xa.L = c->L; xa.level_old = c->nlev - 1;
    xa.fixed_parents = 0; xa.X = c->Xb.as<double>(); xa.Yt = c->Yb.as<double>();
    BCK(launch_form_xy(xa, st));
    BCK(launch_trace(c->Xb.as<double>(), c->Yb.as<double>(), (int64_t)p.kc * p.kc * p.n, r.B, c->lnacc0,
                     c->lnacc.as<double>(), c->o_lnabs.as<double>(), c->o_sign.as<int8_t>(), st));
    BCK(launch_flags_to_u8(c->o_tflags.as<uint32_t>(), c->o_flags.as<uint8_t>(), r.B, c->prefix_flags, st));
    launches += 3;
    r.done = true;
    return MCTRG_OK;
  }

  TuneVal tuned(int n, int kc) const {
    auto it = tune.find(TuneKey{n, kc});
    if (it != tune.end()) return it->second;
    return TuneVal{1 << 16, sample_grid(n, kc)};
  }

  // ---- one sub-batch ---------------------------------------------------------
  // The segments' own kernels run on a pool of streams (forked from and joined
  // back to the batch's stream around each merged stage), so the small
  // launches of different jobs overlap on the device as the server's workers'
  // do; each stream has its own region of the sampler's scratch.
  static constexpr int kStreams = 8;
  cudaStream_t pool[kStreams] = {};
  std::vector<cudaEvent_t> evs;
  size_t smp_region = 0;          // doubles of sampler scratch per stream

  int make_pool() {
    for (int i = 0; i < kStreams; ++i)
      BCK(cudaStreamCreateWithFlags(&pool[i], cudaStreamNonBlocking));
    evs.resize(kStreams + 1);
    for (cudaEvent_t& e : evs) BCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return MCTRG_OK;
  }
  void free_pool() {
    for (cudaStream_t& p : pool) if (p) { cudaStreamDestroy(p); p = nullptr; }
    for (cudaEvent_t e : evs) cudaEventDestroy(e);
    evs.clear();
  }
  // the pool's streams wait for the batch stream's work so far
  int fork(int used) {
    BCK(cudaEventRecord(evs[kStreams], st));
    for (int i = 0; i < used; ++i) BCK(cudaStreamWaitEvent(pool[i], evs[kStreams], 0));
    return MCTRG_OK;
  }
  // the batch stream waits for the pool's work
  int join(int used) {
    for (int i = 0; i < used; ++i) {
      BCK(cudaEventRecord(evs[i], pool[i]));
      BCK(cudaStreamWaitEvent(st, evs[i], 0));
    }
    return MCTRG_OK;
  }

  int run_segments(const std::vector<Segment>& segs) {
    char* base = (char*)ws.p;
    const int prec = opt.precision;
    const bool oz_mode = prec == MCTRG_FP64TC;
    const bool tc_mode = prec != MCTRG_FP64 && !oz_mode;
    const int used = (int)std::min<size_t>(segs.size(), kStreams);
    std::vector<SegPtrs> ptr(segs.size());
    std::vector<SvdItem> items;
    std::vector<int> item_n;          // side of each item (for chunking by shape)
    int n_max = 0, kmax = 0;
    size_t smem = 0;
    BCK(fork(used) == MCTRG_OK ? cudaSuccess : cudaErrorUnknown);
    for (size_t s = 0; s < segs.size(); ++s) {
      const Segment& g = segs[s];
      JobRun& r = jr[g.j];
      mctrg_ctx* c = r.ctx;
      cudaStream_t ss = pool[s % kStreams];
      const LevelInfo& a = c->lv[g.k];
      const LevelInfo& p = c->lv[g.k - 1];
      const ItemLayout L = layout(c, g.k, prec);
      ptr[s] = carve(base, g.off, L, g.cnt);
      const SegPtrs& q = ptr[s];
      XYArgs xa{};
      xa.H = c->Hbuf[r.prev].as<double>(); xa.h_item0 = 0; xa.d = p.D; xa.D = p.kc; xa.c0 = g.i0;
      xa.n_items = g.cnt; xa.Nnew = a.N; xa.Nold = p.N; xa.L = c->L; xa.level_old = g.k - 1;
      xa.fixed_parents = 0; xa.X = q.X; xa.Yt = q.Y;
      BCK(launch_form_xy(xa, ss));
      const int Kd = p.D * p.D;
      const int tc_kind = (prec == MCTRG_TF32 || prec == MCTRG_TF32X3) ? 0 : 1;
      if (oz_mode && gemm_ozaki_supported(a.n, Kd)) {
        int bits, slices;
        ozaki_params(Kd, &bits, &slices);
        BCK(launch_ozaki_split(q.X, g.cnt * a.n, Kd, q.ozX, q.ezX, ss));
        BCK(launch_ozaki_split(q.Y, g.cnt * a.n, Kd, q.ozY, q.ezY, ss));
        GemmOzArgs ga{};
        ga.M = q.M; ga.D = a.D; ga.n = a.n; ga.K = Kd; ga.c0 = g.i0; ga.n_items = g.cnt; ga.Nnew = a.N;
        ga.L = c->L; ga.level_new = g.k; ga.fixed_parity = -1; ga.expX = q.ezX; ga.expY = q.ezY;
        ga.slices = slices; ga.bits = bits; ga.err = err.as<uint32_t>();
        BCK(launch_gemm_ozaki(ga, q.ozX, q.ozY, ss));
        launches += 3;
      } else if (tc_mode && gemm_tc_supported(a.n, Kd, tc_kind)) {
        return MCTRG_EINVAL;   // the TF32/BF16 modes run through mctrg_run, not batches
      } else {
        GemmArgs gm{};
        gm.X = q.X; gm.Yt = q.Y; gm.M = q.M; gm.D = a.D; gm.K = Kd; gm.c0 = g.i0; gm.n_items = g.cnt;
        gm.Nnew = a.N; gm.L = c->L; gm.level_new = g.k; gm.fixed_parity = -1;
        BCK(launch_gemm_f64(gm, ss));
        ++launches;
      }
      launches += 1;
      if (g.bidiag) {
        for (int64_t i = 0; i < g.cnt; ++i) {
          SvdItem t{};
          t.M = q.M + (size_t)i * a.n * a.n; t.W = q.W + (size_t)i * a.n_pad * a.n; t.bd = q.bd + (size_t)i * 3 * a.n;
          t.sig = q.sig + (size_t)i * a.n_pad; t.perm = q.perm + (size_t)i * a.n_pad; t.nnz = q.nnz + i;
          const size_t ks = kept_stride(c->chi);
          t.lns1 = c->ilns1.as<double>() + g.i0 + i; t.kept = q.kept + (size_t)i * ks; t.nk = q.nk + i;
          t.vrows = q.vrows + (size_t)i * ks * a.n; t.zero_rel = zero_fp64(a.n); t.n = a.n; t.n_pad = a.n_pad;
          items.push_back(t);
          item_n.push_back(a.n);
        }
        n_max = std::max(n_max, a.n);
        kmax = std::max(kmax, a.kc);
        smem = std::max(smem, bidiag_smem_bytes(a.n));
      } else {
        // the Jacobi route (low-rank levels): per segment, as mctrg_run does
        JacobiArgs ja{};
        ja.M = q.M; ja.W = q.W; ja.sig = q.sig; ja.perm = q.perm; ja.lns1 = c->ilns1.as<double>() + g.i0;
        ja.nnz = q.nnz; ja.mflags = c->iflags.as<uint32_t>() + g.i0; ja.n = a.n; ja.n_pad = a.n_pad;
        ja.S = (int)g.cnt; ja.max_sweeps = c->opt.max_sweeps; ja.zero_rel = zero_fp64(a.n);
        BCK(launch_jacobi(ja, ss));
        BCK(launch_sample_split(sample_args(r, g, q, 0, s), ss, tuned(a.n, a.kc).sample_grid));
        launches += 2;
      }
    }
    BCK(join(used) == MCTRG_OK ? cudaSuccess : cudaErrorUnknown);
    if (!items.empty()) {
      // the ragged SVD launches over every bidiagonalization segment, in chunks of
      // the tuned size of the largest shape present
      if (sizeof(SvdItem) * items.size() > table.bytes) BCK(cudaStreamSynchronize(st));
      BCK(table.ensure(sizeof(SvdItem) * items.size()));
      BCK(cudaMemcpyAsync(table.p, items.data(), sizeof(SvdItem) * items.size(), cudaMemcpyHostToDevice, st));
      const int S = (int)items.size();
      const int chunk = std::max(1, tuned(n_max, kmax).svd_items);
      for (int i0 = 0; i0 < S; i0 += chunk) {
        const int cnt = std::min(chunk, S - i0);
        BCK(launch_bidiag_items(table.as<SvdItem>() + i0, cnt, n_max, smem, st));
        BCK(launch_bd_bisect_items(table.as<SvdItem>() + i0, cnt, n_max, st));
        launches += 2;
      }
      BCK(fork(used) == MCTRG_OK ? cudaSuccess : cudaErrorUnknown);
      for (size_t s = 0; s < segs.size(); ++s)
        if (segs[s].bidiag) {
          JobRun& r = jr[segs[s].j];
          const LevelInfo& a = r.ctx->lv[segs[s].k];
          BCK(launch_sample_split(sample_args(r, segs[s], ptr[s], 1, s), pool[s % kStreams],
                                  tuned(a.n, a.kc).sample_grid));
          ++launches;
        }
      BCK(join(used) == MCTRG_OK ? cudaSuccess : cudaErrorUnknown);
      const size_t vneed = sizeof(double) * bd_vectors_scratch_doubles(n_max, std::min(S, chunk), kmax);
      if (vneed > vec_scr.bytes) BCK(cudaStreamSynchronize(st));
      BCK(vec_scr.ensure(vneed));
      for (int i0 = 0; i0 < S; i0 += chunk) {
        BdVecArgs va{};
        va.n = n_max; va.S = std::min(chunk, S - i0); va.kmax = kmax; va.items = table.as<SvdItem>() + i0;
        va.scratch = vec_scr.as<double>();
        BCK(launch_bd_vectors(va, st));
        launches += 2;
      }
      BCK(fork(used) == MCTRG_OK ? cudaSuccess : cudaErrorUnknown);
      for (size_t s = 0; s < segs.size(); ++s)
        if (segs[s].bidiag) {
          JobRun& r = jr[segs[s].j];
          const LevelInfo& a = r.ctx->lv[segs[s].k];
          BCK(launch_sample_split(sample_args(r, segs[s], ptr[s], 2, s), pool[s % kStreams],
                                  tuned(a.n, a.kc).sample_grid));
          ++launches;
        }
      BCK(join(used) == MCTRG_OK ? cudaSuccess : cudaErrorUnknown);
    }
    return MCTRG_OK;
  }

  SampleArgs sample_args(JobRun& r, const Segment& g, const SegPtrs& q, int mode, size_t s) {
    mctrg_ctx* c = r.ctx;
    const LevelInfo& a = c->lv[g.k];
    SampleArgs sa{};
    sa.M = q.M; sa.sig = q.sig; sa.nnz = q.nnz; sa.Urows = nullptr; sa.perm = q.perm;
    sa.n = a.n; sa.n_pad = a.n_pad; sa.chi = c->chi; sa.kc = a.kc; sa.stochastic = 1; sa.shared_svd = 0;
    sa.item0 = g.i0; sa.n_items = g.cnt; sa.N = a.N; sa.L = c->L; sa.level = g.k; sa.seed = r.job.seed;
    sa.traj0 = r.job.first_traj; sa.H = c->Hbuf[r.cur].as<double>(); sa.h_item0 = 0;
    sa.iflags = c->iflags.as<uint32_t>(); sa.scratch = smp_scr.as<double>() + (s % kStreams) * smp_region;
    sa.mode = mode;
    sa.kstride = kept_stride(c->chi);
    if (mode == 0) { sa.W = q.W; }
    else { sa.W = nullptr; sa.kept = q.kept; sa.sigt = q.sigt; sa.nk = q.nk; sa.vrows = q.vrows; }
    return sa;
  }

  // ---- the autotuner ---------------------------------------------------------
  // For one shape (n, kc) of the bidiagonalization route: matrices per SVD
  // launch among 1, 2, 4, 8 and 16 per SM, timed on random matrices of that
  // shape (each candidate's launches over the same number of matrices); the
  // count with the best rate is kept (it sets the chunks of the merged SVD
  // launches).  The sampler's CTA
  // count is timed the same way on the choice pass.  Every candidate computes
  // the same numbers; only the launch geometry differs.
  int tune_shape(int n, int kc) {
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, opt.device);
    const int np = n + (n & 1);
    const int cands[5] = {1, 2, 4, 8, 16};
    // test matrices: up to 16 per SM, within 2 GB
    const int ks = kept_stride(kc);
    const size_t per_mat = ((size_t)2 * np * n + 4 * (size_t)n + (size_t)ks * n) * sizeof(double);
    const int total = (int)std::max<size_t>(sms, std::min<size_t>(16 * (size_t)sms, ((size_t)2 << 30) / per_mat));
    OwnedBuf M, W, bd, sig, perm, nnz, l1, vr, kept, nk, scr, tab;
    BCK(M.ensure(sizeof(double) * (size_t)total * n * n));
    BCK(W.ensure(sizeof(double) * (size_t)total * np * n));
    BCK(bd.ensure(sizeof(double) * (size_t)total * 3 * n));
    BCK(sig.ensure(sizeof(double) * (size_t)total * np));
    BCK(perm.ensure(sizeof(int) * (size_t)total * np));
    BCK(nnz.ensure(sizeof(int) * total));
    BCK(l1.ensure(sizeof(double) * total));
    BCK(kept.ensure(sizeof(int) * ks * (size_t)total));
    BCK(nk.ensure(sizeof(int) * total));
    BCK(vr.ensure(sizeof(double) * ks * (size_t)total * n));
    k_fill_random<<<1024, 256, 0, st>>>(M.as<double>(), (int64_t)total * n * n, 0x7E57ull);
    BCK(cudaGetLastError());
    std::vector<int> hk(ks * (size_t)total), hn(total, kc);
    for (int i = 0; i < total; ++i)
      for (int q = 0; q < ks; ++q) hk[(size_t)i * ks + q] = q < kc ? q : 0;
    BCK(cudaMemcpyAsync(kept.p, hk.data(), sizeof(int) * hk.size(), cudaMemcpyHostToDevice, st));
    BCK(cudaMemcpyAsync(nk.p, hn.data(), sizeof(int) * hn.size(), cudaMemcpyHostToDevice, st));
    std::vector<SvdItem> its(total);
    for (int i = 0; i < total; ++i) {
      SvdItem& t = its[i];
      t.M = M.as<double>() + (size_t)i * n * n; t.W = W.as<double>() + (size_t)i * np * n;
      t.bd = bd.as<double>() + (size_t)i * 3 * n; t.sig = sig.as<double>() + (size_t)i * np;
      t.perm = perm.as<int>() + (size_t)i * np; t.nnz = nnz.as<int>() + i; t.lns1 = l1.as<double>() + i;
      t.kept = kept.as<int>() + (size_t)i * ks; t.nk = nk.as<int>() + i; t.vrows = vr.as<double>() + (size_t)i * ks * n;
      t.zero_rel = zero_fp64(n); t.n = n; t.n_pad = np;
    }
    BCK(tab.ensure(sizeof(SvdItem) * its.size()));
    BCK(cudaMemcpyAsync(tab.p, its.data(), sizeof(SvdItem) * its.size(), cudaMemcpyHostToDevice, st));
    BCK(scr.ensure(sizeof(double) * bd_vectors_scratch_doubles(n, total, kc)));
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    double rate[5] = {0, 0, 0, 0, 0};
    int status = MCTRG_OK;
    for (int ci = 0; ci < 5 && status == MCTRG_OK; ++ci) {
      const int per = cands[ci] * sms;
      if (per > total) break;
      for (int rep = 0; rep < 2 && status == MCTRG_OK; ++rep) {   // the first pass warms up
        if (cudaEventRecord(e0, st) != cudaSuccess) { status = MCTRG_ECUDA; break; }
        for (int i0 = 0; i0 < total; i0 += per) {
          const int cnt = std::min(per, total - i0);
          const SvdItem* t = tab.as<SvdItem>() + i0;
          BdVecArgs va{};
          va.n = n; va.S = cnt; va.kmax = kc; va.items = t; va.scratch = scr.as<double>();
          if (launch_bidiag_items(t, cnt, n, bidiag_smem_bytes(n), st) != cudaSuccess ||
              launch_bd_bisect_items(t, cnt, n, st) != cudaSuccess || launch_bd_vectors(va, st) != cudaSuccess) {
            status = MCTRG_ECUDA;
            break;
          }
        }
        float ms = 0.f;
        if (status != MCTRG_OK || cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          status = MCTRG_ECUDA;
          break;
        }
        rate[ci] = total / (ms * 1e-3);
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status != MCTRG_OK) return status;
    double best = 0.0;
    for (double r : rate) best = std::max(best, r);
    int pick = 1;
    for (int ci = 0; ci < 5; ++ci)
      if (rate[ci] > 0.0 && rate[ci] >= best) pick = cands[ci];
    tune[TuneKey{n, kc}] = TuneVal{pick * sms, 8 * sms};
    tune_dirty = true;
    return MCTRG_OK;
  }
};

extern "C" int mctrg_batch_run(const mctrg_options* opt, const mctrg_job* jobs, int n_jobs, mctrg_estimate* est,
                               double* lnabsZ, int8_t* sign, uint8_t* flags) {
  if (!opt || !jobs || !est || n_jobs < 1) return MCTRG_EINVAL;
  if (opt->precision != MCTRG_FP64 && opt->precision != MCTRG_FP64TC) return MCTRG_EINVAL;
  if (opt->svd == MCTRG_SVD_BAND) return MCTRG_EINVAL;   // ragged launches take the one-stage route
  for (int j = 0; j < n_jobs; ++j) {
    const mctrg_job& b = jobs[j];
    if (b.n_samples < 1 || b.first_traj + (uint64_t)b.n_samples > (1ull << 32)) return MCTRG_EINVAL;
  }
  BatchRunner R;
  R.opt = *opt;
  if (R.opt.max_sweeps <= 0) R.opt.max_sweeps = 40;
  if (R.opt.zero_tol_scale == 0.0) R.opt.zero_tol_scale = 1.0;
  R.st = (cudaStream_t)opt->cuda_stream;
  int status = MCTRG_OK;
  R.jr.resize(n_jobs);
  for (int j = 0; j < n_jobs && status == MCTRG_OK; ++j) {
    mctrg_ctx_t c = nullptr;
    mctrg_options o = R.opt;
    o.profile = 0;
    status = mctrg_create(&o, &c);
    if (status != MCTRG_OK) break;
    R.jr[j].ctx = c;
    R.jr[j].job = jobs[j];
    R.jr[j].B = jobs[j].n_samples;
    status = mctrg_init_lattice(c, jobs[j].beta, jobs[j].h, jobs[j].L, jobs[j].chi);
  }
  if (status == MCTRG_OK) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    read_cache(opt->autotune_cache, R.tune);
  }
  // shapes of the bidiagonalization route in this batch: tuned once, cached
  for (int j = 0; j < n_jobs && status == MCTRG_OK; ++j) {
    mctrg_ctx* c = R.jr[j].ctx;
    if (c->all_exact) continue;
    for (int k = c->s0 + 1; k < c->nlev && status == MCTRG_OK; ++k) {
      const int Kd = c->lv[k - 1].D * c->lv[k - 1].D;
      if (!c->use_bidiag(c->lv[k].n, Kd)) continue;
      if (R.tune.count(TuneKey{c->lv[k].n, c->lv[k].kc})) continue;
      status = R.tune_shape(c->lv[k].n, c->lv[k].kc);
    }
  }
  if (status == MCTRG_OK && R.tune_dirty) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    write_cache(opt->autotune_cache, R.tune);
  }
  // workspace: a quarter of the budget left after the jobs' own buffers
  if (status == MCTRG_OK) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) status = MCTRG_ECUDA;
    else {
      const size_t budget = R.opt.hbm_budget_bytes ? R.opt.hbm_budget_bytes : (size_t)(0.8 * (double)fr);
      if (R.err.ensure(sizeof(uint32_t)) != cudaSuccess) status = MCTRG_ENOMEM;
      for (JobRun& r : R.jr)
        if (status == MCTRG_OK) status = R.start_job(r);
      size_t held = 0;
      for (JobRun& r : R.jr) held += r.ctx->held_bytes();
      if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) status = MCTRG_ECUDA;
      size_t wsb = std::min(budget > held ? (budget - held) / 4 : 0, (size_t)(0.7 * (double)fr));
      wsb = std::max<size_t>(wsb, (size_t)64 << 20);
      if (status == MCTRG_OK && R.ws.ensure(wsb) != cudaSuccess) status = MCTRG_ENOMEM;
      size_t scr = 0;
      for (JobRun& r : R.jr)
        if (!r.ctx->all_exact)
          for (int k = r.ctx->s0 + 1; k < r.ctx->nlev; ++k)
            scr = std::max(scr, sample_scratch_doubles(r.ctx->lv[k].n, r.ctx->chi,
                                                       R.tuned(r.ctx->lv[k].n, r.ctx->lv[k].kc).sample_grid));
      R.smp_region = std::max<size_t>(scr, 1);
      if (status == MCTRG_OK && R.smp_scr.ensure(sizeof(double) * R.smp_region * BatchRunner::kStreams) != cudaSuccess)
        status = MCTRG_ENOMEM;
      if (status == MCTRG_OK) status = R.make_pool();
      if (status == MCTRG_OK && cudaMemsetAsync(R.err.p, 0, sizeof(uint32_t), R.st) != cudaSuccess)
        status = MCTRG_ECUDA;
      // sub-batches until every job has finished its levels
      size_t rr = 0;
      while (status == MCTRG_OK) {
        std::vector<Segment> segs;
        size_t used = 0;
        for (size_t q = 0; q < R.jr.size(); ++q) {
          const int j = (int)((rr + q) % R.jr.size());
          JobRun& r = R.jr[j];
          if (r.done || r.next >= r.items) continue;
          mctrg_ctx* c = r.ctx;
          const ItemLayout L = layout(c, r.k, R.opt.precision);
          const int Kd = c->lv[r.k - 1].D * c->lv[r.k - 1].D;
          const bool bd = c->use_bidiag(c->lv[r.k].n, Kd);
          int64_t cap = std::min<int64_t>(r.items - r.next, 1 << 16);
          // every job still at work gets an equal share of the workspace
          int active = 0;
          for (const JobRun& o : R.jr) active += !o.done;
          const size_t share = std::max<size_t>(R.ws.bytes / std::max(1, active), segment_bytes(L, 1));
          int64_t cnt = cap;
          while (cnt > 0 && (used + segment_bytes(L, cnt) > R.ws.bytes || segment_bytes(L, cnt) > share)) cnt /= 2;
          if (cnt <= 0) continue;
          segs.push_back(Segment{j, r.k, r.next, cnt, used, bd});
          used += segment_bytes(L, cnt);
        }
        ++rr;
        if (segs.empty()) {
          bool all = true;
          for (JobRun& r : R.jr) all = all && r.done;
          if (!all) status = MCTRG_ENOMEM;     // a single item does not fit the workspace
          break;
        }
        status = R.run_segments(segs);
        for (const Segment& g : segs) {
          if (status != MCTRG_OK) break;
          JobRun& r = R.jr[g.j];
          r.next += g.cnt;
          if (r.next >= r.items) status = R.end_level(r);
        }
      }
    }
  }
  // results: per job its outputs and estimate
  int64_t off = 0;
  uint32_t tc_err = 0;
  if (status == MCTRG_OK && R.err.p &&
      (cudaMemcpyAsync(&tc_err, R.err.p, sizeof(tc_err), cudaMemcpyDeviceToHost, R.st) != cudaSuccess ||
       cudaStreamSynchronize(R.st) != cudaSuccess))
    status = MCTRG_ECUDA;
  if (status == MCTRG_OK && tc_err) status = MCTRG_ECUDA;
  for (int j = 0; j < n_jobs && status == MCTRG_OK; ++j) {
    JobRun& r = R.jr[j];
    mctrg_ctx* c = r.ctx;
    const int64_t B = r.B;
    if (c->all_exact) {
      std::vector<double> hl((size_t)B, c->const_lnabs);
      std::vector<int8_t> hs((size_t)B, (int8_t)c->const_sign);
      if (cudaMemcpyAsync(c->o_lnabs.p, hl.data(), sizeof(double) * B, cudaMemcpyHostToDevice, R.st) != cudaSuccess ||
          cudaMemcpyAsync(c->o_sign.p, hs.data(), (size_t)B, cudaMemcpyHostToDevice, R.st) != cudaSuccess ||
          launch_flags_to_u8(nullptr, c->o_flags.as<uint8_t>(), B, c->prefix_flags, R.st) != cudaSuccess ||
          cudaStreamSynchronize(R.st) != cudaSuccess) {
        status = MCTRG_ECUDA;
        break;
      }
    }
    double hs[6];
    if (launch_estimate(c->o_lnabs.as<double>(), c->o_sign.as<int8_t>(), c->o_flags.as<uint8_t>(), B,
                        c->stats.as<double>(), R.st) != cudaSuccess ||
        cudaMemcpyAsync(hs, c->stats.p, sizeof(hs), cudaMemcpyDeviceToHost, R.st) != cudaSuccess ||
        (lnabsZ && cudaMemcpyAsync(lnabsZ + off, c->o_lnabs.p, sizeof(double) * B, cudaMemcpyDefault, R.st) != cudaSuccess) ||
        (sign && cudaMemcpyAsync(sign + off, c->o_sign.p, (size_t)B, cudaMemcpyDefault, R.st) != cudaSuccess) ||
        (flags && cudaMemcpyAsync(flags + off, c->o_flags.p, (size_t)B, cudaMemcpyDefault, R.st) != cudaSuccess) ||
        cudaStreamSynchronize(R.st) != cudaSuccess) {
      status = MCTRG_ECUDA;
      break;
    }
    mctrg_estimate& e = est[j];
    std::memset(&e, 0, sizeof(e));
    e.n = B; e.ln_scale = hs[0]; e.sum_x = hs[1]; e.m2_x = hs[2]; e.n_negative = (int64_t)hs[3];
    e.n_flagged = (int64_t)hs[4];
    finish_estimate(&e);
    if (e.status == MCTRG_OK && c->any_noconv(B)) e.status = MCTRG_ENOCONV;
    off += B;
  }
  cudaStreamSynchronize(R.st);
  R.free_pool();
  for (JobRun& r : R.jr) mctrg_destroy(r.ctx);
  return status;
}
