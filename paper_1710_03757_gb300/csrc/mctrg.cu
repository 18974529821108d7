// Host runtime of the MC-TRG library: contexts, the shared deterministic
// prefix, the chunked per-trajectory level loop and the estimate.
//
// Trajectory pipeline (Sec. III): for the level s0 where sampling first
// happens, every tensor of every trajectory shares one SVD (all tensors of
// the translation-invariant network are still identical), so only the
// sampling and the split run per (trajectory, tensor).  Every later level
// runs, per sub-batch of (trajectory, tensor) items:
//   form X, Yt -> GEMM (+ matricization) -> Jacobi SVD -> sample + split,
// then adds each tensor's ln s_1 to its trajectory.  The last level's halves
// are contracted and traced directly.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/mctrg.h"
#include "common.cuh"
#include "kernels.h"
#include "kernels_band.h"
#include "kernels_bd.h"
#include "kernels_tc.h"
#include "mctrg_internal.h"

using namespace mctrg;

#define CK(call)                                     \
  do {                                               \
    cudaError_t e__ = (call);                        \
    if (e__ != cudaSuccess) return fail_cuda(e__);   \
  } while (0)

namespace {

int fail_cuda(cudaError_t e) {
  set_last_cuda_error(e);
  return MCTRG_ECUDA;
}

}  // namespace

namespace mctrg {

static thread_local char g_last_msg[256] = "";

void set_last_cuda_error(cudaError_t e) {
  std::snprintf(g_last_msg, sizeof(g_last_msg), "%s", cudaGetErrorString(e));
}

const char* last_message() { return g_last_msg; }

cudaError_t DevBuf::ensure(size_t b) {
  if (b <= bytes) return cudaSuccess;
  release();
  if (b == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(&p, b);
  if (e == cudaSuccess) bytes = b;
  else p = nullptr;
  return e;
}

void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

}  // namespace mctrg

// ---------------------------------------------------------------------------
extern "C" int mctrg_options_default(mctrg_options* opt) {
  if (!opt) return MCTRG_EINVAL;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = MCTRG_FP64;
  return MCTRG_OK;
}

extern "C" int mctrg_create(const mctrg_options* opt, mctrg_ctx_t* out) {
  if (!opt || !out) return MCTRG_EINVAL;
  if (opt->precision < MCTRG_FP64 || opt->precision > MCTRG_FP64TC) return MCTRG_EINVAL;
  if (opt->svd < MCTRG_SVD_AUTO || opt->svd > MCTRG_SVD_BAND) return MCTRG_EINVAL;
  if (!(opt->zero_tol_scale >= 0.0) || !std::isfinite(opt->zero_tol_scale)) return MCTRG_EINVAL;
  if (opt->deterministic_levels < 0) return MCTRG_EINVAL;
  *out = nullptr;
  int ndev = 0;
  CK(cudaGetDeviceCount(&ndev));
  if (opt->device < 0 || opt->device >= ndev) return MCTRG_EINVAL;
  CK(cudaSetDevice(opt->device));
  mctrg_ctx* c = new (std::nothrow) mctrg_ctx();
  if (!c) return MCTRG_ENOMEM;
  c->opt = *opt;
  if (c->opt.max_sweeps <= 0) c->opt.max_sweeps = 40;
  if (c->opt.zero_tol_scale == 0.0) c->opt.zero_tol_scale = 1.0;
  c->st = (cudaStream_t)opt->cuda_stream;
  if (c->opt.hbm_budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    cudaError_t e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) { delete c; return fail_cuda(e); }
    c->opt.hbm_budget_bytes = (size_t)(0.8 * (double)fr);
  }
  *out = c;
  return MCTRG_OK;
}

extern "C" void mctrg_destroy(mctrg_ctx_t c) {
  if (!c) return;
  cudaSetDevice(c->opt.device);
  cudaStreamSynchronize(c->st);
  c->release_all();
  delete c;
}

extern "C" const char* mctrg_strerror(int s) {
  switch (s) {
    case MCTRG_OK: return "ok";
    case MCTRG_EINVAL: return "invalid argument";
    case MCTRG_ENOMEM: return "device memory budget exceeded or allocation failed";
    case MCTRG_ENOCONV: return "a Jacobi SVD hit the sweep cap";
    case MCTRG_EDOMAIN: return "sample mean of Z is not positive; ln Z undefined";
    case MCTRG_ECUDA: return "CUDA runtime error";
    case MCTRG_ESTATE: return "call out of order";
    case MCTRG_ETIMEDOUT: return "timed out";
    case MCTRG_EAGAIN: return "not finished yet";
    case MCTRG_EUNREACHABLE: return "target error unreachable within the sample budget";
    case MCTRG_ENOTFOUND: return "unknown job";
    default: return "unknown status";
  }
}

cudaEvent_t mctrg_ctx::take_event() {
  if (!event_pool.empty()) {
    cudaEvent_t e = event_pool.back();
    event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void mctrg_ctx::resolve_events() {
  for (const Pending& p : pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) kstat[p.cls].ms += ms;
    event_pool.push_back(p.a);
    event_pool.push_back(p.b);
  }
  pending.clear();
}

extern "C" int mctrg_kernel_stats(mctrg_ctx_t c, int kernel, mctrg_kernel_stat* out) {
  if (!c || !out || kernel < 0 || kernel >= MCTRG_K_COUNT) return MCTRG_EINVAL;
  if (!c->opt.profile) return MCTRG_ESTATE;
  *out = c->kstat[kernel];
  return MCTRG_OK;
}

extern "C" int mctrg_reset_kernel_stats(mctrg_ctx_t c) {
  if (!c) return MCTRG_EINVAL;
  for (auto& k : c->kstat) k = mctrg_kernel_stat{};
  return MCTRG_OK;
}

size_t mctrg_ctx::held_bytes() const {
  const DevBuf* all[] = {&T0, &shM, &shW, &shSig, &shPerm, &shNnz, &shLns1, &shU, &shH, &Hbuf[0], &Hbuf[1],
                         &Mb, &Wb, &Xb, &Yb, &sigb, &permb, &nnzb, &ilns1, &iflags, &lnacc, &tflags,
                         &scratch, &o_lnabs, &o_sign, &o_flags, &o_tflags, &stats, &tcXh, &tcYh, &tcXl,
                         &tcYl, &tcScale, &tcErr, &ozExp, &Timp, &bdb, &keptb, &sigtb, &nkb, &vrowsb, &bdscr,
                         &bandb};
  size_t b = 0;
  for (const DevBuf* d : all) b += d->bytes;
  return b;
}

void mctrg_ctx::release_all() {
  resolve_events();
  for (cudaEvent_t e : event_pool) cudaEventDestroy(e);
  event_pool.clear();
  DevBuf* all[] = {&T0, &shM, &shW, &shSig, &shPerm, &shNnz, &shLns1, &shU, &shH, &Hbuf[0], &Hbuf[1],
                   &Mb, &Wb, &Xb, &Yb, &sigb, &permb, &nnzb, &ilns1, &iflags, &lnacc, &tflags,
                   &scratch, &o_lnabs, &o_sign, &o_flags, &o_tflags, &stats, &tcXh, &tcYh, &tcXl,
                   &tcYl, &tcScale, &tcErr, &ozExp, &Timp, &bdb, &keptb, &sigtb, &nkb, &vrowsb, &bdscr,
                   &bandb};
  for (DevBuf* b : all) b->release();
}

// ---------------------------------------------------------------------------
// Shared prefix: while every tensor of the network is identical, one A and
// one B matricization stand for all of them.
int mctrg_ctx::init_from_device_tensor(int D0, int L_, int chi_) {
  ready = false;
  L = L_;
  chi = chi_;
  int m = 0;
  while ((1 << m) < L) ++m;
  nlev = 2 * m;
  lv.clear();
  lnacc0 = 0.0;
  s0 = nlev;
  all_exact = false;
  prefix_flags = 0;
  level0_distinct = false;
  imp0 = imp1 = -1;
  int D = D0;
  // cur raw tensor lives in T0 (D^4); the plaquette result goes to shM scratch then back
  for (int k = 0; k < nlev; ++k) {
    const int n = D * D, np = n + (n & 1);
    const int64_t N = level_count(L, k);
    CK(shM.ensure(sizeof(double) * 2 * n * n));
    CK(shW.ensure(sizeof(double) * 2 * np * n));
    CK(shSig.ensure(sizeof(double) * 2 * np));
    CK(shPerm.ensure(sizeof(int) * 2 * np));
    CK(shNnz.ensure(sizeof(int) * 2));
    CK(shLns1.ensure(sizeof(double) * 2));
    CK(launch_matricize2(T0.as<double>(), D, shM.as<double>(), st));
    JacobiArgs ja{};
    ja.M = shM.as<double>(); ja.W = shW.as<double>(); ja.sig = shSig.as<double>();
    ja.perm = shPerm.as<int>(); ja.lns1 = shLns1.as<double>(); ja.nnz = shNnz.as<int>();
    ja.mflags = nullptr; ja.n = n; ja.n_pad = np; ja.S = 2; ja.max_sweeps = opt.max_sweeps;
    ja.zero_rel = opt.zero_tol_scale * (double)n * 0x1.0p-52;
    CK(launch_jacobi(ja, st));
    int hn[2];
    double hl[2];
    CK(cudaMemcpyAsync(hn, shNnz.p, sizeof(hn), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hl, shLns1.p, sizeof(hl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    lnacc0 += (double)(N / 2) * (hl[0] + hl[1]);
    const int nu = std::max(hn[0], hn[1]);
    const int kc = std::max(1, std::min(chi, nu));
    LevelInfo li{N, D, n, np, kc};
    lv.push_back(li);
    if (nu <= chi || k < opt.deterministic_levels) {
      // exact level: keep every nonzero value of both matricizations;
      // deterministic level (Sec. II, Eq. approxSVD): keep the kc largest,
      // flagged when a kept and a dropped value are closer than GAP_TOL s_1
      // (the truncated tensor then depends on the basis inside that cluster)
      if (nu > chi) {
        std::vector<double> hs(2 * (size_t)np);
        CK(cudaMemcpyAsync(hs.data(), shSig.p, sizeof(double) * 2 * np, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int p = 0; p < 2; ++p) {
          const double* sp = hs.data() + (size_t)p * np;
          if (hn[p] > kc && sp[kc - 1] - sp[kc] <= GAP_TOL * sp[0]) prefix_flags |= FLAG_SPLIT_CLUSTER;
        }
      }
      CK(shH.ensure(sizeof(double) * 2 * (2 * (size_t)n * kc)));
      CK(scratch.ensure(sizeof(double) * sample_scratch_doubles(n, chi, 2)));
      SampleArgs sa{};
      sa.M = shM.as<double>(); sa.W = shW.as<double>(); sa.sig = shSig.as<double>();
      sa.perm = shPerm.as<int>(); sa.nnz = shNnz.as<int>(); sa.Urows = nullptr;
      sa.n = n; sa.n_pad = np; sa.chi = chi; sa.kc = kc; sa.stochastic = 0; sa.shared_svd = 0;
      sa.item0 = 0; sa.n_items = 2; sa.N = 2; sa.L = L; sa.level = k; sa.seed = 0; sa.traj0 = 0;
      sa.H = shH.as<double>(); sa.h_item0 = 0; sa.iflags = nullptr; sa.scratch = scratch.as<double>();
      CK(launch_sample_split(sa, st, 2));
      CK(Xb.ensure(sizeof(double) * (size_t)kc * kc * n));
      CK(Yb.ensure(sizeof(double) * (size_t)kc * kc * n));
      XYArgs xa{};
      xa.H = shH.as<double>(); xa.h_item0 = 0; xa.d = D; xa.D = kc; xa.c0 = 0; xa.n_items = 1;
      xa.Nnew = 1; xa.Nold = 2; xa.L = L; xa.level_old = k; xa.fixed_parents = 1;
      xa.X = Xb.as<double>(); xa.Yt = Yb.as<double>();
      CK(launch_form_xy(xa, st));
      if (k == nlev - 1) {
        CK(o_lnabs.ensure(sizeof(double)));
        CK(o_sign.ensure(1));
        CK(launch_trace(Xb.as<double>(), Yb.as<double>(), (int64_t)kc * kc * n, 1, lnacc0, nullptr,
                        o_lnabs.as<double>(), o_sign.as<int8_t>(), st));
        int8_t sg = 0;
        CK(cudaMemcpyAsync(&const_lnabs, o_lnabs.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(&sg, o_sign.p, 1, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const_sign = sg;
        all_exact = true;
        break;
      }
      const size_t tbytes = sizeof(double) * (size_t)kc * kc * kc * kc;
      CK(Mb.ensure(tbytes));
      GemmArgs gm{};
      gm.X = Xb.as<double>(); gm.Yt = Yb.as<double>(); gm.M = Mb.as<double>(); gm.D = kc; gm.K = n;
      gm.c0 = 0; gm.n_items = 1; gm.Nnew = 1; gm.L = L; gm.level_new = k + 1; gm.fixed_parity = 0;
      CK(launch_gemm_f64(gm, st));
      CK(T0.ensure(tbytes));
      CK(cudaMemcpyAsync(T0.p, Mb.p, tbytes, cudaMemcpyDeviceToDevice, st));
      D = kc;
      continue;
    }
    // first stochastic level: keep its shared SVD for the per-trajectory draws
    s0 = k;
    CK(shU.ensure(sizeof(double) * 2 * (size_t)np * n));
    CK(launch_u_rows(shM.as<double>(), shW.as<double>(), shSig.as<double>(), shPerm.as<int>(),
                     shNnz.as<int>(), shU.as<double>(), n, np, 2, st));
    break;
  }
  if (!all_exact) {
    for (int k = s0 + 1; k < nlev; ++k) {
      const int D2 = lv[k - 1].kc, n = D2 * D2, np = n + (n & 1);
      lv.push_back(LevelInfo{level_count(L, k), D2, n, np, std::min(chi, n)});
    }
  }
  CK(cudaStreamSynchronize(st));
  ready = true;
  return MCTRG_OK;
}

// SVD route of a level whose n x n matrices are X Yt^T with inner dimension K.
namespace mctrg {
bool route_bidiag(const mctrg_options& o, int n, int K) {
  if (n > 1024) return true;            // beyond the Jacobi kernels' layouts, whatever the option
  if (o.svd == MCTRG_SVD_JACOBI) return false;
  if (o.svd == MCTRG_SVD_BIDIAG) return n >= 2;
  return n >= 64 && 2 * K >= n;
}
// The two-stage route replaces the one-stage one on the sizes it takes.
bool route_band(const mctrg_options& o, int n, int K) {
  return o.svd == MCTRG_SVD_BAND && band_supported(n) && route_bidiag(o, n, K);
}
}  // namespace mctrg

bool mctrg_ctx::use_bidiag(int n, int K) const { return route_bidiag(opt, n, K); }
bool mctrg_ctx::use_band(int n, int K) const { return route_band(opt, n, K); }

static bool is_pow2(int L) { return L >= 2 && (L & (L - 1)) == 0; }

extern "C" int mctrg_init_lattice(mctrg_ctx_t c, double beta, double h, int L, int chi) {
  if (!c) return MCTRG_EINVAL;
  if (!is_pow2(L) || L > 65536 || chi < 1 || chi > kMaxChi || !(beta >= 0.0) || !std::isfinite(beta) ||
      !std::isfinite(h))
    return MCTRG_EINVAL;
  CK(cudaSetDevice(c->opt.device));
  CK(c->T0.ensure(16 * sizeof(double)));
  CK(launch_site_tensor(beta, h, c->T0.as<double>(), c->st));
  return c->init_from_device_tensor(2, L, chi);
}

extern "C" int mctrg_init_bond_lattice(mctrg_ctx_t c, double beta, double h, int L, int chi) {
  if (!c) return MCTRG_EINVAL;
  if (!is_pow2(L) || L > 65536 || chi < 1 || chi > kMaxChi || !(beta >= 0.0) || !std::isfinite(beta) ||
      !std::isfinite(h))
    return MCTRG_EINVAL;
  CK(cudaSetDevice(c->opt.device));
  CK(c->T0.ensure(16 * sizeof(double)));
  CK(launch_bond_tensor(beta, h, c->T0.as<double>(), c->st));
  return c->init_from_device_tensor(2, L, chi);
}

extern "C" int mctrg_init_impurity(mctrg_ctx_t c, double beta, double h, int L, int chi, int n_imp) {
  if (!c) return MCTRG_EINVAL;
  if (!is_pow2(L) || L > 65536 || chi < 1 || chi > kMaxChi || !(beta >= 0.0) || !std::isfinite(beta) ||
      !std::isfinite(h) || (n_imp != 1 && n_imp != 2) || c->opt.deterministic_levels > 0)
    return MCTRG_EINVAL;
  CK(cudaSetDevice(c->opt.device));
  c->ready = false;
  CK(c->T0.ensure(16 * sizeof(double)));
  CK(c->Timp.ensure(16 * sizeof(double)));
  CK(launch_site_tensor(beta, h, c->T0.as<double>(), c->st));
  CK(launch_impurity_tensor(beta, h, c->Timp.as<double>(), c->st));
  // every level split per tensor from level 0: D' = min(chi, D^2) from D = 2
  c->L = L;
  c->chi = chi;
  int m = 0;
  while ((1 << m) < L) ++m;
  c->nlev = 2 * m;
  c->lv.clear();
  int D = 2;
  for (int k = 0; k < c->nlev; ++k) {
    const int n = D * D;
    c->lv.push_back(LevelInfo{level_count(L, k), D, n, n + (n & 1), std::min(chi, n)});
    D = std::min(chi, n);
  }
  c->s0 = 0;
  c->lnacc0 = 0.0;
  c->all_exact = false;
  c->prefix_flags = 0;
  c->level0_distinct = true;
  c->imp0 = 0;                       // site (0, 0)
  c->imp1 = n_imp == 2 ? 1 : -1;     // site (1, 0), its right neighbour
  CK(cudaStreamSynchronize(c->st));
  c->ready = true;
  return MCTRG_OK;
}

extern "C" int mctrg_ratio_estimate(const mctrg_estimate* num, const mctrg_estimate* den, double* ratio,
                                    double* se) {
  if (!num || !den || !ratio || num->n < 2 || den->n < 2) return MCTRG_EINVAL;
  if (!(den->mean_Z_scaled > 0.0)) return MCTRG_EDOMAIN;
  const double r = std::exp(num->ln_scale - den->ln_scale) * num->mean_Z_scaled / den->mean_Z_scaled;
  *ratio = r;
  if (se) {
    const double a = num->mean_Z_scaled != 0.0 ? num->se_Z_scaled / num->mean_Z_scaled : INFINITY;
    const double b = den->se_Z_scaled / den->mean_Z_scaled;
    *se = std::fabs(r) * std::sqrt(a * a + b * b);
    if (num->mean_Z_scaled == 0.0)   // an exactly zero numerator: the SE from its spread alone
      *se = std::exp(num->ln_scale - den->ln_scale) * num->se_Z_scaled / den->mean_Z_scaled;
  }
  return MCTRG_OK;
}

extern "C" int mctrg_init_tensor(mctrg_ctx_t c, const double* T0, int D, int L, int chi) {
  if (!c || !T0) return MCTRG_EINVAL;
  if (!is_pow2(L) || L > 65536 || chi < 1 || chi > kMaxChi || D < 1 || D > 8) return MCTRG_EINVAL;
  CK(cudaSetDevice(c->opt.device));
  const size_t bytes = sizeof(double) * (size_t)D * D * D * D;
  CK(c->T0.ensure(bytes));
  CK(cudaMemcpyAsync(c->T0.p, T0, bytes, cudaMemcpyHostToDevice, c->st));
  return c->init_from_device_tensor(D, L, chi);
}

// ---------------------------------------------------------------------------
// Device bytes of one item's tensor-core operands (X and Yt, n x d2 each):
// the rounded operands (and residuals) of the mixed modes, or the BF16 slice
// planes and row exponents of the FP64-accurate mode.
static size_t tc_operand_bytes(int prec, int n, int d2) {
  const size_t e = (size_t)n * d2;
  switch (prec) {
    case MCTRG_TF32: return 2 * 4 * e;
    case MCTRG_BF16: return 2 * 2 * e;
    case MCTRG_TF32X3: return 2 * 2 * 4 * e;
    case MCTRG_BF16X3: return 2 * 2 * 2 * e;
    case MCTRG_FP64TC: return gemm_ozaki_supported(n, d2) ? 2 * 8 * 2 * e + 2 * (size_t)n * sizeof(int) : 0;
    default: return 0;
  }
}

namespace mctrg {
// The sampler's CTA count for a run over levels s0 .. nlev-1 (from the largest
// side), and the table scratch it needs.
int run_sample_grid(const std::vector<LevelInfo>& lv, int s0, int nlev, int chi) {
  int nmax = 1;
  for (int k = s0; k < nlev; ++k) nmax = std::max(nmax, lv[k].n);
  return sample_grid(nmax, chi);
}
size_t run_sample_scratch(const std::vector<LevelInfo>& lv, int s0, int nlev, int chi) {
  const int g = run_sample_grid(lv, s0, nlev, chi);
  size_t m = 0;
  for (int k = s0; k < nlev; ++k) m = std::max(m, sample_scratch_doubles(lv[k].n, chi, g));
  return m;
}

// Memory plan of a run of n_samples trajectories over levels s0 .. nlev-1 of
// lv (sampled; the shared prefix is held separately): B trajectories per
// chunk, S items per sub-batch, and the device bytes the run holds.  At most
// a quarter of the budget holds the per-item working set (and no more items
// than a level of one chunk has), the rest the trajectories of a chunk.
// B < 1 means that not even one trajectory fits.
void plan_run(const std::vector<LevelInfo>& lv, int s0, int nlev, int chi, const mctrg_options& opt,
              size_t budget, int64_t n_samples, int64_t& B, int64_t& S, size_t& total) {
  size_t per_traj = 2 * sizeof(double) + sizeof(uint32_t);   // lnacc, tflags
  size_t max_pair = 0, max_items = 0, per_item = 0, bd_scr = 0;
  int64_t maxN = 1;
  for (int k = s0; k < nlev; ++k) {
    const LevelInfo& a = lv[k];
    size_t hk = (size_t)a.N * 2 * a.n * a.kc * sizeof(double);
    size_t hp = (k > s0) ? (size_t)lv[k - 1].N * 2 * lv[k - 1].n * lv[k - 1].kc * sizeof(double) : 0;
    max_pair = std::max(max_pair, hk + hp);
    max_items = std::max(max_items, (size_t)a.N);
    if (k > s0) {
      maxN = std::max<int64_t>(maxN, a.N);
      const size_t d2 = (size_t)lv[k - 1].D * lv[k - 1].D;
      size_t pi = (2 * (size_t)a.n * d2 + (size_t)a.n * a.n + (size_t)a.n_pad * a.n + a.n_pad) * sizeof(double) +
                  (a.n_pad + 1) * sizeof(int) + sizeof(double) + sizeof(uint32_t);
      pi += tc_operand_bytes(opt.precision, a.n, (int)d2);
      if (route_bidiag(opt, a.n, (int)d2)) {   // d, e, tau; kept values and vectors
        const size_t ks = kept_stride(chi);
        pi += (3 * (size_t)a.n + ks + ks * (size_t)a.n) * sizeof(double) + (ks + 1) * sizeof(int);
        bd_scr = std::max(bd_scr, bd_vectors_scratch_doubles(a.n, 1 << 16, a.kc) * sizeof(double));
        // the band route: band, panel scratch, chase reflectors, exponent
        if (route_band(opt, a.n, (int)d2)) pi += band_item_bytes(a.n);
      }
      per_item = std::max(per_item, pi);
    }
  }
  {  // final contraction X, Yt per trajectory
    const LevelInfo& a = lv[nlev - 1];
    size_t fin = 2 * (size_t)a.kc * a.kc * a.n * sizeof(double);
    per_traj += fin;
  }
  per_traj += max_pair + max_items * (sizeof(double) + sizeof(uint32_t));
  {  // level s0 split per item (a lattice with impurities): its matrices, rows and values
    const LevelInfo& a = lv[s0];
    per_item = std::max(per_item, ((size_t)a.n * a.n + (size_t)a.n_pad * a.n + a.n_pad) * sizeof(double) +
                                      (a.n_pad + 1) * sizeof(int) + sizeof(double) + sizeof(uint32_t));
  }
  const size_t tables = run_sample_scratch(lv, s0, nlev, chi) * sizeof(double) + bd_scr;
  const int64_t Bmax = opt.max_chunk > 0 ? std::min<int64_t>(opt.max_chunk, n_samples) : n_samples;
  const size_t work_budget = std::max<size_t>(budget / 4, 1);
  S = per_item ? (int64_t)std::max<size_t>(1, std::min<size_t>(work_budget / per_item, 1 << 16)) : 1;
  S = std::max<int64_t>(1, std::min<int64_t>(S, Bmax * maxN));   // no more than a level's items
  const size_t work = per_item * (size_t)S + tables;
  const size_t rest = budget > work ? budget - work : 0;
  B = (int64_t)(rest / std::max<size_t>(per_traj, 1));
  B = std::min<int64_t>(B, Bmax);
  total = work + (size_t)std::max<int64_t>(B, 1) * per_traj + (size_t)n_samples * 14;
}

// The same plan for a lattice not yet set up, from the largest leg dimensions
// its levels can have (D' = min(chi, D^2) from D0, sampling from the first
// level with D^2 > chi): an upper bound of what plan_run gives after
// mctrg_init_*, where ranks can only be smaller and exact levels longer.
void plan_run_bound(int L, int chi, int D0, const mctrg_options& opt, size_t budget, int64_t n_samples,
                    int64_t& B, int64_t& S, size_t& total) {
  int m = 0;
  while ((1 << m) < L) ++m;
  const int nlev = 2 * m;
  std::vector<LevelInfo> lv;
  int D = D0, s0 = nlev;
  for (int k = 0; k < nlev; ++k) {
    const int n = D * D;
    const int kc = std::min(chi, n);
    lv.push_back(LevelInfo{level_count(L, k), D, n, n + (n & 1), kc});
    if (s0 == nlev && n > chi && k >= opt.deterministic_levels) s0 = k;
    D = kc;
  }
  if (s0 == nlev) { B = n_samples; S = 1; total = (size_t)n_samples * 14; return; }
  plan_run(lv, s0, nlev, chi, opt, budget, n_samples, B, S, total);
}
}  // namespace mctrg

void mctrg_ctx::plan_chunks(int64_t n_samples, int64_t& B, int64_t& S, size_t& total) const {
  plan_run(lv, s0, nlev, chi, opt, opt.hbm_budget_bytes, n_samples, B, S, total);
}

extern "C" int mctrg_footprint(mctrg_ctx_t c, int64_t n_samples, size_t* bytes) {
  if (!c || !bytes || n_samples < 1) return MCTRG_EINVAL;
  if (!c->ready) return MCTRG_ESTATE;
  if (c->all_exact) { *bytes = (size_t)n_samples * 14; return MCTRG_OK; }
  int64_t B, S;
  c->plan_chunks(n_samples, B, S, *bytes);
  return B >= 1 ? MCTRG_OK : MCTRG_ENOMEM;
}

static void finalize_estimate(const double* s, int64_t n, mctrg_estimate* est) {
  std::memset(est, 0, sizeof(*est));
  est->n = n;
  est->ln_scale = s[0];
  est->sum_x = s[1];
  est->m2_x = s[2];
  est->n_negative = (int64_t)s[3];
  est->n_flagged = (int64_t)s[4];
  finish_estimate(est);
}

namespace mctrg {
void finish_estimate(mctrg_estimate* e) {
  const double n = (double)e->n;
  const double mean = e->sum_x / n;
  e->mean_Z_scaled = mean;
  e->se_Z_scaled = e->n > 1 ? std::sqrt(std::max(0.0, e->m2_x / (n - 1.0)) / n) : NAN;
  const double sumsq = e->m2_x + n * mean * mean;
  e->ess = sumsq > 0 ? e->sum_x * e->sum_x / sumsq : 0.0;
  if (mean > 0) {
    e->ln_mean_Z = e->ln_scale + std::log(mean);
    e->se_ln_Z = e->se_Z_scaled / mean;
    e->status = MCTRG_OK;
  } else {
    e->ln_mean_Z = NAN;
    e->se_ln_Z = NAN;
    e->status = MCTRG_EDOMAIN;
  }
}
}  // namespace mctrg

// Unit roundoff of the tensor-core operands of a precision mode.
static double tc_unit_roundoff(int prec) {
  switch (prec) {
    case MCTRG_TF32: return 0x1.0p-11;
    case MCTRG_BF16: return 0x1.0p-8;
    case MCTRG_TF32X3: return 0x1.0p-22;
    case MCTRG_BF16X3: return 0x1.0p-17;
    default: return 0x1.0p-52;
  }
}

int mctrg_ctx::run(int64_t n, uint64_t seed, uint64_t first_traj, double* lnabs_out, int8_t* sign_out,
                   uint8_t* flags_out, mctrg_estimate* est) {
  CK(o_lnabs.ensure(sizeof(double) * n));
  CK(o_sign.ensure((size_t)n));
  CK(o_flags.ensure((size_t)n));
  CK(stats.ensure(8 * sizeof(double)));
  if (all_exact) {
    std::vector<double> hl((size_t)n, const_lnabs);
    std::vector<int8_t> hs((size_t)n, (int8_t)const_sign);
    CK(cudaMemcpyAsync(o_lnabs.p, hl.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(o_sign.p, hs.data(), (size_t)n, cudaMemcpyHostToDevice, st));
    CK(launch_flags_to_u8(nullptr, o_flags.as<uint8_t>(), n, prefix_flags, st));
    CK(cudaStreamSynchronize(st));
  } else {
    int64_t B, S;
    size_t total;
    plan_chunks(n, B, S, total);
    if (B < 1) return MCTRG_ENOMEM;
    CK(o_tflags.ensure(sizeof(uint32_t) * (size_t)B));
    CK(lnacc.ensure(sizeof(double) * (size_t)B));
    const int grid_s = run_sample_grid(lv, s0, nlev, chi);
    const int ks = kept_stride(chi);
    size_t max_h = 0, max_items = 0, max_xy = 0, max_m = 0, max_w = 0, max_np = 0, max_scr = 0;
    for (int k = s0; k < nlev; ++k) {
      const LevelInfo& a = lv[k];
      max_h = std::max(max_h, (size_t)B * a.N * 2 * a.n * a.kc);
      max_items = std::max(max_items, (size_t)B * a.N);
      max_scr = std::max(max_scr, sample_scratch_doubles(a.n, chi, grid_s));
      if (k > s0) {
        const size_t d2 = (size_t)lv[k - 1].D * lv[k - 1].D;
        max_xy = std::max(max_xy, (size_t)S * a.n * d2);
        max_m = std::max(max_m, (size_t)S * a.n * a.n);
        max_w = std::max(max_w, (size_t)S * a.n_pad * a.n);
        max_np = std::max(max_np, (size_t)S * a.n_pad);
      }
    }
    {
      const LevelInfo& a = lv[nlev - 1];
      max_xy = std::max(max_xy, (size_t)B * a.kc * a.kc * a.n);
    }
    if (level0_distinct) {   // level 0's own matrices, SVD and sampling per item
      const LevelInfo& a = lv[0];
      max_m = std::max(max_m, (size_t)S * a.n * a.n);
      max_w = std::max(max_w, (size_t)S * a.n_pad * a.n);
      max_np = std::max(max_np, (size_t)S * a.n_pad);
      max_items = std::max(max_items, (size_t)B * a.N);
    }
    CK(Hbuf[0].ensure(sizeof(double) * max_h));
    CK(Hbuf[1].ensure(sizeof(double) * max_h));
    CK(iflags.ensure(sizeof(uint32_t) * max_items));
    CK(ilns1.ensure(sizeof(double) * max_items));
    CK(Xb.ensure(sizeof(double) * std::max<size_t>(max_xy, 1)));
    CK(Yb.ensure(sizeof(double) * std::max<size_t>(max_xy, 1)));
    CK(Mb.ensure(sizeof(double) * std::max<size_t>(max_m, 1)));
    CK(Wb.ensure(sizeof(double) * std::max<size_t>(max_w, 1)));
    CK(sigb.ensure(sizeof(double) * std::max<size_t>(max_np, 1)));
    CK(permb.ensure(sizeof(int) * std::max<size_t>(max_np, 1)));
    CK(nnzb.ensure(sizeof(int) * std::max<int64_t>(S, 1)));
    CK(scratch.ensure(sizeof(double) * max_scr));
    {  // bidiagonalization route buffers (levels that take it)
      size_t bd_n = 0, bd_scr = 0;
      for (int k = s0 + 1; k < nlev; ++k) {
        const LevelInfo& a = lv[k];
        if (!use_bidiag(a.n, lv[k - 1].D * lv[k - 1].D)) continue;
        bd_n = std::max(bd_n, (size_t)a.n);
        bd_scr = std::max(bd_scr, bd_vectors_scratch_doubles(a.n, (int)std::min<int64_t>(S, 1 << 16), a.kc));
      }
      size_t band_n = 0;
      for (int k = s0 + 1; k < nlev; ++k)
        if (use_band(lv[k].n, lv[k - 1].D * lv[k - 1].D)) band_n = std::max(band_n, (size_t)lv[k].n);
      if (band_n) {
        CK(bandb.ensure((size_t)std::max<int64_t>(S, 1) * band_item_bytes((int)band_n) + 256));
        CK(cudaMemsetAsync(bandb.p, 0, bandb.bytes, st));
      }
      if (bd_n) {
        const size_t Ss = (size_t)std::max<int64_t>(S, 1);
        CK(bdb.ensure(sizeof(double) * Ss * 3 * bd_n));
        CK(keptb.ensure(sizeof(int) * Ss * ks));
        CK(sigtb.ensure(sizeof(double) * Ss * ks));
        CK(nkb.ensure(sizeof(int) * Ss));
        CK(vrowsb.ensure(sizeof(double) * Ss * ks * bd_n));
        CK(bdscr.ensure(sizeof(double) * bd_scr));
      }
    }
    // tensor-core operands (mixed precision): per item X and Yt rounded, with scales
    const int prec = opt.precision;
    const bool oz_mode = prec == MCTRG_FP64TC;    // FP64-accurate tensor-core GEMM (BF16 slices)
    const bool tc_mode = prec != MCTRG_FP64 && !oz_mode;
    const int tc_kind = (prec == MCTRG_TF32 || prec == MCTRG_TF32X3) ? 0 : 1;
    const int tc_passes = (prec == MCTRG_TF32X3 || prec == MCTRG_BF16X3) ? 3 : 1;
    const size_t tc_esize = tc_kind == 0 ? 4 : 2;
    if (tc_mode) {
      const size_t elems = std::max<size_t>(max_xy, 1);
      CK(tcXh.ensure(tc_esize * elems));
      CK(tcYh.ensure(tc_esize * elems));
      if (tc_passes == 3) {
        CK(tcXl.ensure(tc_esize * elems));
        CK(tcYl.ensure(tc_esize * elems));
      }
      CK(tcScale.ensure(sizeof(double) * 2 * std::max<int64_t>(S, 1)));
    }
    if (oz_mode) {   // slice planes (at most 8 per operand) and row exponents
      size_t oz_elems = 0, oz_rows = 0;
      for (int k = s0 + 1; k < nlev; ++k) {
        const int Kd = lv[k - 1].D * lv[k - 1].D;
        if (!gemm_ozaki_supported(lv[k].n, Kd)) continue;
        oz_elems = std::max(oz_elems, (size_t)S * lv[k].n * Kd);
        oz_rows = std::max(oz_rows, (size_t)S * lv[k].n);
      }
      if (oz_elems) {
        CK(tcXh.ensure(2 * 8 * oz_elems));
        CK(tcYh.ensure(2 * 8 * oz_elems));
        CK(ozExp.ensure(sizeof(int) * 2 * oz_rows));
      }
    }
    if (prec != MCTRG_FP64 || bandb.p) {
      CK(tcErr.ensure(sizeof(uint32_t)));
      CK(cudaMemsetAsync(tcErr.p, 0, sizeof(uint32_t), st));
    }
    uint32_t* const band_err = tcErr.as<uint32_t>();
    for (int64_t c0 = 0; c0 < n; c0 += B) {
      const int64_t Bc = std::min(B, n - c0);
      const uint64_t traj0 = first_traj + (uint64_t)c0;
      CK(cudaMemsetAsync(lnacc.p, 0, sizeof(double) * Bc, st));
      CK(cudaMemsetAsync(o_tflags.p, 0, sizeof(uint32_t) * Bc, st));
      int cur = 0;
      if (level0_distinct) {  // level 0 of a lattice with impurities: every tensor split on its own
        const LevelInfo& a = lv[0];
        const int64_t items = Bc * a.N;
        CK(cudaMemsetAsync(iflags.p, 0, sizeof(uint32_t) * items, st));
        for (int64_t i0 = 0; i0 < items; i0 += S) {
          const int64_t Si = std::min(S, items - i0);
          CK(timed(MCTRG_K_OTHER, Si, 0.0, 8.0 * Si * a.n * a.n, [&] {
            return launch_level0_matrices(T0.as<double>(), Timp.as<double>(), imp0, imp1, L, i0, Si, a.N,
                                          Mb.as<double>(), st); }));
          JacobiArgs ja{};
          ja.M = Mb.as<double>(); ja.W = Wb.as<double>(); ja.sig = sigb.as<double>();
          ja.perm = permb.as<int>(); ja.lns1 = ilns1.as<double>() + i0; ja.nnz = nnzb.as<int>();
          ja.mflags = iflags.as<uint32_t>() + i0; ja.n = a.n; ja.n_pad = a.n_pad; ja.S = (int)Si;
          ja.max_sweeps = opt.max_sweeps;
          ja.zero_rel = opt.zero_tol_scale * (double)a.n * 0x1.0p-52;
          const double nn = a.n;
          CK(timed(MCTRG_K_JACOBI, Si, Si * ((8.0 / 3.0) * nn * nn * nn + 4.0 * nn * nn * a.kc),
                   8.0 * Si * (nn * nn + (double)a.n_pad * nn + 1.5 * a.n_pad), [&] { return launch_jacobi(ja, st); }));
          SampleArgs sa{};
          sa.M = Mb.as<double>(); sa.W = Wb.as<double>(); sa.sig = sigb.as<double>(); sa.perm = permb.as<int>();
          sa.nnz = nnzb.as<int>(); sa.Urows = nullptr; sa.n = a.n; sa.n_pad = a.n_pad; sa.chi = chi; sa.kc = a.kc;
          sa.stochastic = 1; sa.shared_svd = 0; sa.item0 = i0; sa.n_items = Si; sa.N = a.N; sa.L = L; sa.level = 0;
          sa.seed = seed; sa.traj0 = traj0; sa.H = Hbuf[cur].as<double>(); sa.h_item0 = 0;
          sa.iflags = iflags.as<uint32_t>(); sa.scratch = scratch.as<double>(); sa.mode = 0;
          CK(timed(MCTRG_K_SAMPLE, Si, Si * (4.0 * nn * a.kc + 2.0 * nn * nn * a.kc),
                   8.0 * Si * (2.0 * nn * nn + 2.0 * nn * a.kc), [&] { return launch_sample_split(sa, st, grid_s); }));
        }
        CK(timed(MCTRG_K_OTHER, Bc, 0.0, 12.0 * items, [&] {
          return launch_traj_accum(ilns1.as<double>(), iflags.as<uint32_t>(), a.N, Bc, lnacc.as<double>(),
                                   o_tflags.as<uint32_t>(), st); }));
      } else {  // level s0: shared SVD, per-(trajectory, tensor) sampling
        const LevelInfo& a = lv[s0];
        const int64_t items = Bc * a.N;
        CK(cudaMemsetAsync(iflags.p, 0, sizeof(uint32_t) * items, st));
        SampleArgs sa{};
        sa.M = shM.as<double>(); sa.W = shW.as<double>(); sa.sig = shSig.as<double>();
        sa.perm = shPerm.as<int>(); sa.nnz = shNnz.as<int>(); sa.Urows = shU.as<double>();
        sa.n = a.n; sa.n_pad = a.n_pad; sa.chi = chi; sa.kc = a.kc; sa.stochastic = 1; sa.shared_svd = 1;
        sa.item0 = 0; sa.n_items = items; sa.N = a.N; sa.L = L; sa.level = s0; sa.seed = seed;
        sa.traj0 = traj0; sa.H = Hbuf[cur].as<double>(); sa.h_item0 = 0; sa.iflags = iflags.as<uint32_t>();
        sa.scratch = scratch.as<double>();
        CK(timed(MCTRG_K_SAMPLE, items, items * (4.0 * a.n * a.kc),
                 8.0 * items * (2.0 * a.n * a.kc + a.n_pad), [&] { return launch_sample_split(sa, st, grid_s); }));
        CK(timed(MCTRG_K_OTHER, Bc, 0.0, 4.0 * items, [&] {
          return launch_traj_accum(nullptr, iflags.as<uint32_t>(), a.N, Bc, lnacc.as<double>(),
                                   o_tflags.as<uint32_t>(), st); }));
      }
      for (int k = s0 + 1; k < nlev; ++k) {
        const LevelInfo& a = lv[k];
        const LevelInfo& p = lv[k - 1];
        const int prev = cur;
        cur ^= 1;
        const int64_t items = Bc * a.N;
        CK(cudaMemsetAsync(iflags.p, 0, sizeof(uint32_t) * items, st));
        for (int64_t i0 = 0; i0 < items; i0 += S) {
          const int64_t Si = std::min(S, items - i0);
          XYArgs xa{};
          xa.H = Hbuf[prev].as<double>(); xa.h_item0 = 0; xa.d = p.D; xa.D = p.kc; xa.c0 = i0;
          xa.n_items = Si; xa.Nnew = a.N; xa.Nold = p.N; xa.L = L; xa.level_old = k - 1;
          xa.fixed_parents = 0; xa.X = Xb.as<double>(); xa.Yt = Yb.as<double>();
          const double D2 = (double)p.kc * p.kc, dd = p.D;
          CK(timed(MCTRG_K_FORM_XY, Si, Si * 4.0 * D2 * dd * dd * dd,
                   8.0 * Si * (4.0 * p.kc * dd * dd + 2.0 * D2 * dd * dd), [&] { return launch_form_xy(xa, st); }));
          const int Kd = p.D * p.D;
          const bool used_tc = tc_mode && gemm_tc_supported(a.n, Kd, tc_kind);
          const bool used_oz = oz_mode && gemm_ozaki_supported(a.n, Kd);
          if (used_oz) {
            // FP64-accurate on the tensor cores: BF16 slices of X and Yt, exact slice products
            int oz_bits, oz_slices;
            ozaki_params(Kd, &oz_bits, &oz_slices);
            int* eX = ozExp.as<int>();
            int* eY = eX + Si * a.n;
            const int64_t rows = Si * a.n;
            CK(timed(MCTRG_K_FORM_XY, Si, 0.0, Si * 2.0 * a.n * Kd * (8.0 + 2.0 * oz_slices), [&] {
              cudaError_t e = launch_ozaki_split(Xb.as<double>(), rows, Kd, tcXh.p, eX, st);
              if (e != cudaSuccess) return e;
              return launch_ozaki_split(Yb.as<double>(), rows, Kd, tcYh.p, eY, st); }));
            GemmOzArgs ga{};
            ga.M = Mb.as<double>(); ga.D = a.D; ga.n = a.n; ga.K = Kd; ga.c0 = i0; ga.n_items = Si;
            ga.Nnew = a.N; ga.L = L; ga.level_new = k; ga.fixed_parity = -1; ga.expX = eX; ga.expY = eY;
            ga.slices = oz_slices; ga.bits = oz_bits; ga.err = tcErr.as<uint32_t>();
            CK(timed(MCTRG_K_GEMM, Si, Si * 2.0 * a.n * a.n * Kd,
                     Si * (2.0 * 2.0 * oz_slices * a.n * Kd + 8.0 * a.n * a.n), [&] {
              return launch_gemm_ozaki(ga, tcXh.p, tcYh.p, st); }));
          } else if (used_tc) {
            // tensor cores: scale and round the operands, then tcgen05 GEMM
            double* sX = tcScale.as<double>();
            double* sY = sX + Si;
            const int64_t per = (int64_t)a.n * Kd;
            CK(timed(MCTRG_K_FORM_XY, Si, 0.0, Si * per * (16.0 + 2.0 * tc_esize * tc_passes), [&] {
              cudaError_t e = launch_convert_scaled(Xb.as<double>(), per, Si, tc_kind, tcXh.p,
                                                    tc_passes == 3 ? tcXl.p : nullptr, sX, st);
              if (e != cudaSuccess) return e;
              return launch_convert_scaled(Yb.as<double>(), per, Si, tc_kind, tcYh.p,
                                           tc_passes == 3 ? tcYl.p : nullptr, sY, st); }));
            GemmTcArgs ga{};
            ga.M = Mb.as<double>(); ga.D = a.D; ga.n = a.n; ga.K = Kd; ga.c0 = i0; ga.n_items = Si;
            ga.Nnew = a.N; ga.L = L; ga.level_new = k; ga.fixed_parity = -1; ga.scaleX = sX; ga.scaleY = sY;
            ga.passes = tc_passes; ga.err = tcErr.as<uint32_t>();
            CK(timed(MCTRG_K_GEMM, Si, Si * 2.0 * a.n * a.n * Kd,
                     Si * (2.0 * a.n * Kd * tc_esize * tc_passes + 8.0 * a.n * a.n), [&] {
              return launch_gemm_tc(ga, tc_kind, tcXh.p, tcYh.p, tcXl.p, tcYl.p, st); }));
          } else {
            GemmArgs gm{};
            gm.X = Xb.as<double>(); gm.Yt = Yb.as<double>(); gm.M = Mb.as<double>(); gm.D = a.D;
            gm.K = Kd; gm.c0 = i0; gm.n_items = Si; gm.Nnew = a.N; gm.L = L; gm.level_new = k;
            gm.fixed_parity = -1;
            CK(timed(MCTRG_K_GEMM, Si, Si * 2.0 * a.n * a.n * gm.K, 8.0 * Si * (2.0 * a.n * gm.K + (double)a.n * a.n),
                     [&] { return launch_gemm_f64(gm, st); }));
          }
          const double nn = a.n;
          const double zero_rel = opt.zero_tol_scale *
              (used_tc ? std::min(std::sqrt(nn) * tc_unit_roundoff(prec), 1.0 / 64.0) : nn * 0x1.0p-52);
          SampleArgs sa{};
          sa.M = Mb.as<double>(); sa.sig = sigb.as<double>(); sa.nnz = nnzb.as<int>(); sa.Urows = nullptr;
          sa.n = a.n; sa.n_pad = a.n_pad; sa.chi = chi; sa.kc = a.kc; sa.stochastic = 1; sa.shared_svd = 0;
          sa.item0 = i0; sa.n_items = Si; sa.N = a.N; sa.L = L; sa.level = k; sa.seed = seed;
          sa.traj0 = traj0; sa.H = Hbuf[cur].as<double>(); sa.h_item0 = 0;
          sa.iflags = iflags.as<uint32_t>(); sa.scratch = scratch.as<double>();
          if (use_bidiag(a.n, Kd)) {
            // bidiagonalization (one stage, or dense -> band -> bidiagonal), bisection,
            // choice of the kept indices, their vectors, halves
            const bool band = use_band(a.n, Kd);
            BandArgs bda{};
            if (band) {
              band_carve(bandb.p, a.n, Si, bda);
              bda.M = Mb.as<double>(); bda.Wk = (int64_t*)Wb.p; bda.bd = bdb.as<double>(); bda.S = (int)Si;
              bda.err = band_err;
              CK(timed(MCTRG_K_BAND, Si, Si * (8.0 / 3.0) * nn * nn * nn, 8.0 * Si * (nn * nn + 9.0 * nn),
                       [&] { return launch_band_reduce(bda, false, st); }));
              CK(timed(MCTRG_K_CHASE, Si, Si * 6.0 * kBandW * nn * nn, 8.0 * Si * (12.0 * nn),
                       [&] { return launch_band_chase(bda, st); }));
            } else {
              BidiagArgs ba{};
              ba.M = Mb.as<double>(); ba.W = Wb.as<double>(); ba.bd = bdb.as<double>(); ba.n = a.n; ba.S = (int)Si;
              CK(timed(MCTRG_K_BIDIAG, Si, Si * (8.0 / 3.0) * nn * nn * nn, 8.0 * Si * (2.0 * nn * nn + 3.0 * nn),
                       [&] { return launch_bidiag(ba, st); }));
            }
            CK(timed(MCTRG_K_BISECT, Si, 0.0, 8.0 * Si * (3.0 * nn + a.n_pad) + 4.0 * Si * (a.n_pad + 1), [&] {
              return launch_bd_bisect(bdb.as<double>(), a.n, a.n_pad, (int)Si, sigb.as<double>(), permb.as<int>(),
                                      nnzb.as<int>(), ilns1.as<double>() + i0, zero_rel, st); }));
            sa.mode = 1; sa.kept = keptb.as<int>(); sa.sigt = sigtb.as<double>(); sa.nk = nkb.as<int>();
            sa.kstride = ks;
            sa.W = nullptr; sa.perm = permb.as<int>();
            CK(timed(MCTRG_K_SAMPLE, Si, Si * 4.0 * nn * a.kc, 8.0 * Si * (a.n_pad + 2.0 * ks),
                     [&] { return launch_sample_split(sa, st, grid_s); }));
            BdVecArgs va{};
            va.bd = bdb.as<double>(); va.R = Wb.as<double>(); va.sig = sigb.as<double>(); va.kept = keptb.as<int>();
            va.nk = nkb.as<int>(); va.vrows = vrowsb.as<double>(); va.scratch = bdscr.as<double>();
            va.n = a.n; va.n_pad = a.n_pad; va.S = (int)Si; va.kmax = a.kc; va.kstride = ks;
            va.skip_backtr = band ? 1 : 0;
            CK(timed(MCTRG_K_VECTORS, Si, Si * ((band ? 4.0 : 2.0) * nn * nn * a.kc + 40.0 * nn * a.kc),
                     8.0 * Si * (nn * nn / 2.0 + 3.0 * nn + 2.0 * a.kc * nn), [&] {
              cudaError_t e = launch_bd_vectors(va, st);
              if (e != cudaSuccess || !band) return e;
              BandVecArgs bv{};
              bv.band = &bda; bv.sig = sigb.as<double>(); bv.kept = keptb.as<int>(); bv.nk = nkb.as<int>();
              bv.vrows = vrowsb.as<double>(); bv.n_pad = a.n_pad; bv.kstride = ks; bv.unit_rows = 0;
              return launch_band_backtr(bv, st); }));
            sa.mode = 2; sa.vrows = vrowsb.as<double>();
            CK(timed(MCTRG_K_SAMPLE, Si, Si * 2.0 * nn * nn * a.kc, 8.0 * Si * (2.0 * nn * nn + 2.0 * nn * a.kc),
                     [&] { return launch_sample_split(sa, st, grid_s); }));
          } else {
            JacobiArgs ja{};
            ja.M = Mb.as<double>(); ja.W = Wb.as<double>(); ja.sig = sigb.as<double>();
            ja.perm = permb.as<int>(); ja.lns1 = ilns1.as<double>() + i0; ja.nnz = nnzb.as<int>();
            ja.mflags = iflags.as<uint32_t>() + i0; ja.n = a.n; ja.n_pad = a.n_pad; ja.S = (int)Si;
            ja.max_sweeps = opt.max_sweeps;
            ja.zero_rel = zero_rel;
            if (used_tc) ja.noise_u = tc_unit_roundoff(prec);
            CK(timed(MCTRG_K_JACOBI, Si, Si * ((8.0 / 3.0) * nn * nn * nn + 4.0 * nn * nn * a.kc),
                     8.0 * Si * (nn * nn + (double)a.n_pad * nn + 1.5 * a.n_pad), [&] { return launch_jacobi(ja, st); }));
            sa.mode = 0; sa.W = Wb.as<double>(); sa.perm = permb.as<int>();
            CK(timed(MCTRG_K_SAMPLE, Si, Si * (4.0 * nn * a.kc + 2.0 * nn * nn * a.kc),
                     8.0 * Si * (2.0 * nn * nn + 2.0 * nn * a.kc), [&] { return launch_sample_split(sa, st, grid_s); }));
        
          }
        }
        CK(timed(MCTRG_K_OTHER, Bc, 0.0, 12.0 * items, [&] {
          return launch_traj_accum(ilns1.as<double>(), iflags.as<uint32_t>(), a.N, Bc, lnacc.as<double>(),
                                   o_tflags.as<uint32_t>(), st); }));
      }
      {  // final contraction and trace
        const LevelInfo& p = lv[nlev - 1];
        XYArgs xa{};
        xa.H = Hbuf[cur].as<double>(); xa.h_item0 = 0; xa.d = p.D; xa.D = p.kc; xa.c0 = 0;
        xa.n_items = Bc; xa.Nnew = 1; xa.Nold = p.N; xa.L = L; xa.level_old = nlev - 1;
        xa.fixed_parents = 0; xa.X = Xb.as<double>(); xa.Yt = Yb.as<double>();
        const double D2 = (double)p.kc * p.kc, dd = p.D;
        CK(timed(MCTRG_K_FORM_XY, Bc, Bc * 4.0 * D2 * dd * dd * dd,
                 8.0 * Bc * (4.0 * p.kc * dd * dd + 2.0 * D2 * dd * dd), [&] { return launch_form_xy(xa, st); }));
        CK(timed(MCTRG_K_TRACE, Bc, Bc * 2.0 * D2 * p.n, 8.0 * Bc * 2.0 * D2 * p.n, [&] {
          return launch_trace(Xb.as<double>(), Yb.as<double>(), (int64_t)p.kc * p.kc * p.n, Bc, lnacc0,
                              lnacc.as<double>(), o_lnabs.as<double>() + c0, o_sign.as<int8_t>() + c0, st); }));
        CK(timed(MCTRG_K_OTHER, Bc, 0.0, 5.0 * Bc, [&] {
          return launch_flags_to_u8(o_tflags.as<uint32_t>(), o_flags.as<uint8_t>() + c0, Bc, prefix_flags, st); }));
      }
    }
  }
  CK(timed(MCTRG_K_OTHER, n, 0.0, 10.0 * n, [&] {
    return launch_estimate(o_lnabs.as<double>(), o_sign.as<int8_t>(), o_flags.as<uint8_t>(), n,
                           stats.as<double>(), st); }));
  double hs[6];
  CK(cudaMemcpyAsync(hs, stats.p, sizeof(hs), cudaMemcpyDeviceToHost, st));
  if (lnabs_out) CK(cudaMemcpyAsync(lnabs_out, o_lnabs.p, sizeof(double) * n, cudaMemcpyDefault, st));
  if (sign_out) CK(cudaMemcpyAsync(sign_out, o_sign.p, (size_t)n, cudaMemcpyDefault, st));
  if (flags_out) CK(cudaMemcpyAsync(flags_out, o_flags.p, (size_t)n, cudaMemcpyDefault, st));
  uint32_t tc_err = 0;
  if ((opt.precision != MCTRG_FP64 || opt.svd == MCTRG_SVD_BAND) && tcErr.p)
    CK(cudaMemcpyAsync(&tc_err, tcErr.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  resolve_events();
  if (tc_err) return MCTRG_ECUDA;   // a tensor-core pipeline wait expired
  finalize_estimate(hs, n, est);
  // any trajectory whose SVD hit the sweep cap
  if (est->status == MCTRG_OK && any_noconv(n)) est->status = MCTRG_ENOCONV;
  return est->status == MCTRG_EDOMAIN ? MCTRG_EDOMAIN : est->status;
}

bool mctrg_ctx::any_noconv(int64_t n) {
  std::vector<uint8_t> f((size_t)n);
  if (cudaMemcpyAsync(f.data(), o_flags.p, (size_t)n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return false;
  for (uint8_t v : f)
    if (v & FLAG_NOCONV) return true;
  return false;
}

extern "C" int mctrg_run(mctrg_ctx_t c, int64_t n, uint64_t seed, uint64_t first_traj, double* lnabs,
                         int8_t* sign, uint8_t* flags, mctrg_estimate* est) {
  if (!c || !est || n < 1) return MCTRG_EINVAL;
  if (first_traj + (uint64_t)n > (1ull << 32)) return MCTRG_EINVAL;
  if (!c->ready) return MCTRG_ESTATE;
  CK(cudaSetDevice(c->opt.device));
  return c->run(n, seed, first_traj, lnabs, sign, flags, est);
}

extern "C" int mctrg_merge_estimates(const mctrg_estimate* parts, int k, mctrg_estimate* out) {
  if (!parts || !out || k < 1) return MCTRG_EINVAL;
  double m = -INFINITY;
  int64_t n = 0, nneg = 0, nflag = 0;
  for (int i = 0; i < k; ++i) {
    if (parts[i].n < 1) return MCTRG_EINVAL;
    m = std::max(m, parts[i].ln_scale);
    n += parts[i].n;
    nneg += parts[i].n_negative;
    nflag += parts[i].n_flagged;
  }
  double sum = 0.0;
  for (int i = 0; i < k; ++i) sum += parts[i].sum_x * std::exp(parts[i].ln_scale - m);
  const double mean = sum / (double)n;
  double m2 = 0.0;
  for (int i = 0; i < k; ++i) {
    const double f = std::exp(parts[i].ln_scale - m);
    const double mi = parts[i].sum_x * f / (double)parts[i].n;
    m2 += parts[i].m2_x * f * f + (double)parts[i].n * (mi - mean) * (mi - mean);
  }
  std::memset(out, 0, sizeof(*out));
  out->n = n;
  out->ln_scale = m;
  out->sum_x = sum;
  out->m2_x = m2;
  out->n_negative = nneg;
  out->n_flagged = nflag;
  finish_estimate(out);
  return MCTRG_OK;
}
