// Shared device/host helpers of the MC-TRG library: TRG geometry on the
// torus, the Philox4x32-10 uniform stream, and error plumbing.
#pragma once
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#define MCTRG_HD __host__ __device__ __forceinline__

namespace mctrg {

// ---------------------------------------------------------------------------
// TRG geometry (Sec. III; Levin-Nave coarse-graining on an L x L torus).
//
// Level-k tensors sit at o_k + i a1 + j a2 with a1 = (1+i)^k, a2 = i (1+i)^k
// read as Gaussian integers (level 0: a1 = right, a2 = down).  Each level-k
// tensor is identified with a level-0 "anchor" site z = x + i y (its chain of
// top-left parents), and z - o_k = i a1 + j a2 exactly, so
//   * the level-k tensors are the sites z with (1+i)^k | z;
//   * sublattice A (i + j even) is (1+i)^(k+1) | z;
//   * the neighbour at +a1 / +a2 has anchor z + a1 / z + a2 (mod L);
//   * tensors are numbered in row-major order of their anchors (this is the
//     same as numbering level k+1 by the level-k id of the top-left parent).
// (1+i)^(2t) = (2i)^t, so for k = 2t the anchors are the sites with x, y
// multiples of 2^t; for k = 2t+1 additionally x/2^t + y/2^t is even.
// ---------------------------------------------------------------------------
MCTRG_HD int64_t level_count(int L, int k) { return ((int64_t)L * L) >> k; }

// (1+i)^k as a Gaussian integer (re, im); |components| <= 2^(k/2).
MCTRG_HD void one_plus_i_pow(int k, int& re, int& im) {
  re = 1; im = 0;
  for (int s = 0; s < k; ++s) { int r = re - im, q = re + im; re = r; im = q; }
}

MCTRG_HD int64_t anchor_rank(int L, int k, int x, int y) {
  int t = k >> 1;
  if ((k & 1) == 0) return (int64_t)(y >> t) * (L >> t) + (x >> t);
  return (int64_t)(y >> t) * (L >> (t + 1)) + ((x >> t) >> 1);
}

MCTRG_HD void anchor_of(int L, int k, int64_t id, int& x, int& y) {
  int t = k >> 1;
  if ((k & 1) == 0) {
    int64_t w = L >> t;
    x = (int)(id % w) << t; y = (int)(id / w) << t;
  } else {
    int64_t w = L >> (t + 1);
    int yy = (int)(id / w), xx = 2 * (int)(id % w) + (yy & 1);
    x = xx << t; y = yy << t;
  }
}

MCTRG_HD int wrap(int v, int L) { v %= L; return v < 0 ? v + L : v; }

// 0 = sublattice A, 1 = sublattice B, for level-k tensor id (k < 2 log2 L).
MCTRG_HD int tensor_parity(int L, int k, int64_t id) {
  int x, y; anchor_of(L, k, id, x, y);
  int t = (k + 1) >> 1;                      // divisibility by (1+i)^(k+1)
  if (((k + 1) & 1) == 0) return ((x | y) & ((1 << t) - 1)) ? 1 : 0;
  int t2 = k >> 1;                           // k+1 = 2 t2 + 1
  if ((x | y) & ((1 << t2) - 1)) return 1;
  return (((x >> t2) + (y >> t2)) & 1) ? 1 : 0;
}

// Parents (at level k) of tensor c of level k+1, in the order
// (p, p+a1, p+a2, p+a1+a2), which contribute F3, F4, F2, F1.
MCTRG_HD void tensor_parents(int L, int k, int64_t c, int64_t par[4]) {
  int x, y; anchor_of(L, k + 1, c, x, y);     // anchor of c = anchor of its p
  int ar, ai; one_plus_i_pow(k, ar, ai);      // a1
  int br = -ai, bi = ar;                      // a2 = i * a1
  par[0] = anchor_rank(L, k, x, y);
  par[1] = anchor_rank(L, k, wrap(x + ar, L), wrap(y + ai, L));
  par[2] = anchor_rank(L, k, wrap(x + br, L), wrap(y + bi, L));
  par[3] = anchor_rank(L, k, wrap(x + ar + br, L), wrap(y + ai + bi, L));
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 3.3).
// key = (seed lo, seed hi); counter = (t >> 1, tensor, level, trajectory);
// draw step t takes words (0,1) of the block for even t and (2,3) for odd t,
// as the 53-bit uniform ((hi << 32 | lo) >> 11) * 2^-53 in [0, 1).
// ---------------------------------------------------------------------------
struct U4 { uint32_t x0, x1, x2, x3; };

MCTRG_HD U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c.x0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c.x2;
    U4 n;
    n.x0 = (uint32_t)(p1 >> 32) ^ c.x1 ^ k0;
    n.x1 = (uint32_t)p1;
    n.x2 = (uint32_t)(p0 >> 32) ^ c.x3 ^ k1;
    n.x3 = (uint32_t)p0;
    c = n;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
  return c;
}

MCTRG_HD double philox_uniform(uint64_t seed, uint32_t traj, uint32_t level,
                               uint32_t tensor, uint32_t t) {
  U4 c{t >> 1, tensor, level, traj};
  U4 o = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  uint32_t lo = (t & 1) ? o.x2 : o.x0, hi = (t & 1) ? o.x3 : o.x1;
  uint64_t w = ((uint64_t)hi << 32) | lo;
  return (double)(w >> 11) * 0x1.0p-53;
}

// Flag bits (kept equal to the MCTRG_FLAG_* values of the public header).
constexpr uint32_t FLAG_SPLIT_CLUSTER = 1u, FLAG_DRAW_TIE = 2u, FLAG_TINY_KEPT = 4u,
                   FLAG_NOCONV = 16u;
constexpr double GAP_TOL = 1e-8, TIE_TOL = 1e-9, TINY_TOL = 1e-7;

// Raise a kernel's dynamic shared-memory limit on the current device, once
// per (kernel, device); safe to call from several host threads at once (a
// race only repeats the call).  `done` holds one bit per device ordinal
// below 64; higher ordinals set the attribute on every call.
template <class Kernel>
inline cudaError_t raise_smem_limit(Kernel* kernel, int bytes, std::atomic<uint64_t>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  // no more than the device allows a block beside the kernel's static shared memory
  cudaFuncAttributes fa{};
  e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  bytes = std::min(bytes, optin - (int)fa.sharedSizeBytes);
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

}  // namespace mctrg
