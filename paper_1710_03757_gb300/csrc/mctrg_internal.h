// Internal host-side state of an MC-TRG context.
#pragma once
#include <cstdint>
#include <cstdio>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mctrg.h"

namespace mctrg {

// Largest kept count: a level matrix is at most chi^2 = 2304 on a side (the
// bidiagonalization route's limit), the sampler and the vectors take up to 64.
constexpr int kMaxChi = 48;

// A device allocation that only grows.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t b);
  void release();
  template <class T> T* as() const { return (T*)p; }
};

// Shape of one SVD level k: N tensors per trajectory with legs of dimension
// D, matricized as n x n (n = D^2, n_pad = n rounded up to even), split with
// kc kept columns (the leg dimension of level k+1).
struct LevelInfo {
  int64_t N;
  int D, n, n_pad, kc;
};

bool route_bidiag(const mctrg_options& o, int n, int K);
bool route_band(const mctrg_options& o, int n, int K);
void plan_run(const std::vector<LevelInfo>& lv, int s0, int nlev, int chi, const mctrg_options& opt,
              size_t budget, int64_t n_samples, int64_t& B, int64_t& S, size_t& total);
void plan_run_bound(int L, int chi, int D0, const mctrg_options& opt, size_t budget, int64_t n_samples,
                    int64_t& B, int64_t& S, size_t& total);

void set_last_cuda_error(cudaError_t e);
const char* last_message();
void finish_estimate(mctrg_estimate* e);

}  // namespace mctrg

struct mctrg_ctx {
  mctrg_options opt{};
  cudaStream_t st = nullptr;
  bool ready = false;
  int L = 0, chi = 0, nlev = 0;
  std::vector<mctrg::LevelInfo> lv;
  int s0 = 0;               // first level where sampling happens (nlev: none)
  double lnacc0 = 0.0;      // sum of ln s_1 over the shared levels 0..s0
  bool all_exact = false;
  uint32_t prefix_flags = 0; // flags of the shared levels (deterministic truncations), in every trajectory
  // impurity lattices: every level split per tensor from level 0 (no shared
  // prefix); sites imp0 / imp1 (-1: none) hold the tensor Timp instead of T0
  bool level0_distinct = false;
  int imp0 = -1, imp1 = -1;
  double const_lnabs = 0.0;
  int const_sign = 0;
  mctrg::DevBuf T0, shM, shW, shSig, shPerm, shNnz, shLns1, shU, shH;
  mctrg::DevBuf Hbuf[2], Mb, Wb, Xb, Yb, sigb, permb, nnzb, ilns1, iflags, lnacc, tflags, scratch;
  mctrg::DevBuf o_lnabs, o_sign, o_flags, o_tflags, stats;
  mctrg::DevBuf tcXh, tcYh, tcXl, tcYl, tcScale, tcErr;   // tensor-core operands (slice planes in FP64TC)
  mctrg::DevBuf ozExp;                                     // FP64TC: row exponents of X and Yt
  mctrg::DevBuf Timp;                                      // impurity tensor (level0_distinct)
  mctrg::DevBuf bdb, keptb, sigtb, nkb, vrowsb, bdscr;    // bidiagonalization route
  mctrg::DevBuf bandb;                                     // band route: band, scratch, reflectors

  // per-kernel-class statistics (MCTRG_K_*)
  mctrg_kernel_stat kstat[MCTRG_K_COUNT]{};
  struct Pending { int cls; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  // Launch through f(); counts it, and with profiling brackets it with events.
  template <class F>
  cudaError_t timed(int cls, int64_t items, double flops, double bytes, F&& f) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (opt.profile) {
      a = take_event();
      b = take_event();
      if (!a || !b) return cudaErrorMemoryAllocation;
      cudaEventRecord(a, st);
    }
    cudaError_t e = f();
    if (e != cudaSuccess) return e;
    if (opt.profile) {
      cudaEventRecord(b, st);
      pending.push_back(Pending{cls, a, b});
    }
    kstat[cls].launches += 1;
    kstat[cls].items += items;
    kstat[cls].flops_alg += flops;
    kstat[cls].bytes_alg += bytes;
    return cudaSuccess;
  }
  cudaEvent_t take_event();
  void resolve_events();   // after a stream synchronize

  int init_from_device_tensor(int D0, int L, int chi);
  bool use_bidiag(int n, int K) const;
  bool use_band(int n, int K) const;
  void plan_chunks(int64_t n_samples, int64_t& B, int64_t& S, size_t& total) const;
  int run(int64_t n, uint64_t seed, uint64_t first_traj, double* lnabs, int8_t* sign, uint8_t* flags,
          mctrg_estimate* est);
  bool any_noconv(int64_t n);
  void release_all();
  size_t held_bytes() const;   // device bytes the context's buffers hold now
};
