// K2: batched FP64 one-sided Jacobi SVD (Sec. II, Eq. exactSVD).
//
// Hestenes' method applied to the rows: plane rotations from the left make
// the rows of M mutually orthogonal, J M = B, so the singular values are the
// row norms and the right singular vectors the normalized rows; the left
// vectors of the few kept indices are recovered later as u = M v / s.
// One-sided Jacobi computes small singular values to high relative accuracy,
// which matters here because the sampler divides kept values by inclusion
// rates that scale like s^2.
//
// One CTA per matrix.  The n_pad (even) rows are paired by the round-robin
// ("circle") ordering: n_pad - 1 steps per sweep, n_pad / 2 disjoint pairs per
// step handled by lane groups in parallel.  Rows live in shared memory when
// they fit (n <= 158), otherwise in the caller's global workspace, which the
// batch keeps L2-resident (one matrix per SM).  Stopping rule: a sweep with no
// rotation, where a pair is rotated iff |b_p . b_q| > n_pad 2^-53 |b_p| |b_q|
// (Demmel and Veselic 1992).  Row norms are recomputed exactly at the start
// of every sweep and at the end.  Rows whose norm is below 2^-53 |M|_F are
// rounding noise (they always end below the sampler's zero threshold
// n 2^-52 s_1): each sweep pairs only the remaining active rows, so a
// rank-r matrix costs O(r^2 n) per sweep instead of O(n^3).
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace mctrg {

static __device__ __forceinline__ double group_sum(double v, int G) {
  for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void k_jacobi(JacobiArgs a, int use_smem, int G) {
  extern __shared__ double smem[];
  __shared__ int s_rot;
  const int mat = blockIdx.x;
  const int n = a.n, np = a.n_pad;
  double* A = use_smem ? smem : a.W + (size_t)mat * np * n;
  double* nrm = use_smem ? smem + (size_t)np * n : smem;
  int* act = (int*)(nrm + np);                      // [np + 1] active rows of a sweep
  const double* Mm = a.M + (size_t)mat * n * n;
  for (int idx = threadIdx.x; idx < np * n; idx += blockDim.x)
    A[idx] = idx < n * n ? Mm[idx] : 0.0;
  __syncthreads();

  const int gl = threadIdx.x & (G - 1);
  const int grp = threadIdx.x / G;
  const int ngrp = blockDim.x / G;
  const double tol = (double)np * 0x1.0p-53;
  bool converged = false;
  __shared__ int s_na;
  __shared__ double s_thr2;

  for (int sweep = 0; sweep < a.max_sweeps && !converged; ++sweep) {
    for (int base = 0; base < np; base += ngrp) {
      int r = base + grp;
      double s = 0.0;
      if (r < np)
        for (int c = gl; c < n; c += G) { double v = A[(size_t)r * n + c]; s = fma(v, v, s); }
      s = group_sum(s, G);
      if (r < np && gl == 0) nrm[r] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (sweep == 0) {                       // |M|_F^2 is invariant under the rotations
        double f = 0.0;
        for (int r = 0; r < np; ++r) f += nrm[r];
        s_thr2 = f * 0x1.0p-106;
      }
      int na = 0;
      for (int r = 0; r < np; ++r)
        if (nrm[r] > s_thr2) act[na++] = r;
      if (na & 1) act[na] = -1;
      s_na = na;
      s_rot = 0;
    }
    __syncthreads();
    const int na = s_na, nap = na + (na & 1), npairs = nap >> 1;
    for (int step = 0; step + 1 < nap; ++step) {
      int myrot = 0;
      for (int base = 0; base < npairs; base += ngrp) {
        const int pk = base + grp;
        int P = -1, Q = -1;
        if (pk < npairs) {
          P = act[pk == 0 ? 0 : 1 + (pk - 1 + step) % (nap - 1)];
          Q = act[1 + (nap - 2 - pk + step) % (nap - 1)];
        }
        const bool act_pair = P >= 0 && Q >= 0;
        if (!act_pair) { P = 0; Q = 0; }
        double* ap = A + (size_t)P * n;
        double* aq = A + (size_t)Q * n;
        double g = 0.0;
        if (act_pair)
          for (int c = gl; c < n; c += G) g = fma(ap[c], aq[c], g);
        g = group_sum(g, G);                       // every lane of the warp takes part
        const double al = act_pair ? nrm[P] : 0.0, be = act_pair ? nrm[Q] : 0.0;
        const bool rot = act_pair && al > 0.0 && be > 0.0 && fabs(g) > tol * sqrt(al) * sqrt(be);
        double nal = al, nbe = be;
        if (rot) {                                 // uniform within the lane group
          const double zeta = (be - al) / (2.0 * g);
          double t;
          if (fabs(zeta) > 1e150) t = 0.5 / zeta;
          else t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
          const double cs = 1.0 / sqrt(fma(t, t, 1.0));
          const double sn = cs * t;
          for (int c = gl; c < n; c += G) {
            const double x = ap[c], y = aq[c];
            ap[c] = fma(-sn, y, cs * x);
            aq[c] = fma(sn, x, cs * y);
          }
          nal = fma(-t, g, al);
          nbe = fma(t, g, be);
          ++myrot;
        }
        // heavy cancellation in the norm update: recompute from the rotated rows
        const bool fixP = rot && nal < 0.01 * al, fixQ = rot && nbe < 0.01 * be;
        double sp = 0.0, sq = 0.0;
        if (fixP) for (int c = gl; c < n; c += G) sp = fma(ap[c], ap[c], sp);
        if (fixQ) for (int c = gl; c < n; c += G) sq = fma(aq[c], aq[c], sq);
        sp = group_sum(sp, G);
        sq = group_sum(sq, G);
        if (fixP) nal = sp;
        if (fixQ) nbe = sq;
        if (rot && gl == 0) { nrm[P] = nal; nrm[Q] = nbe; }
      }
      if (myrot && gl == 0) atomicAdd(&s_rot, myrot);
      __syncthreads();
    }
    converged = (s_rot == 0);
    __syncthreads();
  }

  // exact final norms
  for (int base = 0; base < np; base += ngrp) {
    int r = base + grp;
    double s = 0.0;
    if (r < np)
      for (int c = gl; c < n; c += G) { double v = A[(size_t)r * n + c]; s = fma(v, v, s); }
    s = group_sum(s, G);
    if (r < np && gl == 0) nrm[r] = sqrt(s);
  }
  __syncthreads();
  // rank sort, descending; ties keep row order
  double* sg = a.sig + (size_t)mat * np;
  int* pm = a.perm + (size_t)mat * np;
  for (int r = threadIdx.x; r < np; r += blockDim.x) {
    const double v = nrm[r];
    int rank = 0;
    for (int j = 0; j < np; ++j) {
      const double u = nrm[j];
      rank += (u > v) || (u == v && j < r);
    }
    sg[rank] = v;
    pm[rank] = r;
  }
  if (use_smem) {
    double* Wm = a.W + (size_t)mat * np * n;
    for (int idx = threadIdx.x; idx < np * n; idx += blockDim.x) Wm[idx] = A[idx];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s1 = sg[0];
    if (a.lns1) a.lns1[mat] = s1 > 0.0 ? log(s1) : -INFINITY;
    const double tau = (double)n * 0x1.0p-52 * s1;
    int cnt = 0;
    for (int r = 0; r < np; ++r) cnt += sg[r] > tau;
    a.nnz[mat] = s1 > 0.0 ? cnt : 0;
    if (a.mflags && !converged) a.mflags[mat] |= FLAG_NOCONV;
  }
}

cudaError_t launch_jacobi(const JacobiArgs& a, cudaStream_t st) {
  if (a.S <= 0) return cudaSuccess;
  const int n = a.n, np = a.n_pad;
  const size_t rows_bytes = (size_t)np * n * sizeof(double);
  const size_t nrm_bytes = (size_t)np * sizeof(double) + (size_t)(np + 2) * sizeof(int);
  const int use_smem = (rows_bytes + nrm_bytes) <= 200 * 1024;
  // Rows in the global workspace: ask for enough shared memory that one CTA
  // runs per SM, so the rows of the resident matrices stay in L2.
  const size_t smem = use_smem ? rows_bytes + nrm_bytes : std::max<size_t>(nrm_bytes, 120 * 1024);
  int G = 2;
  while (G < 32 && G < n) G <<= 1;
  if (G > 2 && G >= n) G >>= 1;                 // about two elements per lane
  int threads = n <= 16 ? 32 : (n <= 64 ? 256 : 512);
  if (threads < G) threads = G;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024 + 64);
    attr_set = true;
  }
  k_jacobi<<<a.S, threads, smem, st>>>(a, use_smem, G);
  return cudaGetLastError();
}

}  // namespace mctrg
