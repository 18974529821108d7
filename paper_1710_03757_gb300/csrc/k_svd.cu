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
// of every sweep and at the end.  Rows whose norm is below (u/2) |M|_F, u the
// unit roundoff of the arithmetic that produced M (2^-52 for FP64), are
// rounding noise (they always end below the sampler's zero threshold): each
// sweep pairs only the remaining active rows, so a rank-r matrix costs
// O(r^2 n) per sweep instead of O(n^3).
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
  const double nu = a.noise_u > 0.0 ? a.noise_u : 0x1.0p-52;
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
        s_thr2 = f * (0.25 * nu * nu);
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
    const double tau = (a.zero_rel > 0.0 ? a.zero_rel : (double)n * 0x1.0p-52) * s1;
    int cnt = 0;
    for (int r = 0; r < np; ++r) cnt += sg[r] > tau;
    a.nnz[mat] = s1 > 0.0 ? cnt : 0;
    if (a.mflags && !converged) a.mflags[mat] |= FLAG_NOCONV;
  }
}

// ---------------------------------------------------------------------------
// Warp-batched variant for n > 32 (one lane group = the whole warp).
//
// Each warp takes PW disjoint pairs of a round-robin step.  Their PW dot
// products are reduced together by recursive halving (lane bit 4 picks the
// upper or lower half of the pair set, then bit 3, ...), which costs about
// PW additions per lane instead of 5 PW, and leaves the total of pair
// j = lane >> (5 - log2 PW) in every lane; each lane then computes the
// rotation of "its" pair, so the divisions and square roots are shared by
// the PW pairs.  Rotations use scaled rows (Anda and Park 1994, fast plane
// rotations): the true row is d_r * row_r; the rotation by tangent t,
// cosine c becomes
//   row_p <- row_p - t (d_q / d_p) row_q,  row_q <- row_q + t (d_p / d_q) row_p,
//   d_p <- c d_p,  d_q <- c d_q,
// two FMAs per element instead of four.  With |t| <= 1 each rotation scales
// d by at least 2^-1/2, and the scales are folded back into the rows at every
// sweep start, so d stays above 2^-(n-1)/2.  True squared norms are carried
// separately and recomputed exactly at every sweep start.
template <int PW>
__device__ __forceinline__ double batched_reduce(double (&v)[PW], int lane) {
  int cnt = PW;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    if (cnt > 1) {
      const int half = cnt >> 1;
      const bool upper = (lane & o) != 0;
#pragma unroll
      for (int k = 0; k < PW / 2; ++k) {
        if (k < half) {
          const double send = upper ? v[k] : v[k + half];
          const double keep = upper ? v[k + half] : v[k];
          v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
      }
      cnt = half;
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
    }
  }
  return v[0];
}

// Householder QR with column pivoting of the np x n row-major matrix A
// (Businger and Golub 1965; norm downdating with the safeguard of LAPACK's
// xLAQP2): A P = Q R, R overwrites A (zeros below the diagonal), Q is not
// formed and colperm[c] = original column of column c.  The singular values
// of R are those of M, and a right singular vector v~ of R gives v = P v~ for
// M.  The rows of R are graded (|r_kk| decreasing), which cuts one-sided
// Jacobi from ~40 sweeps to ~9 on the TRG level matrices (Drmac and Veselic
// 2008, preconditioned Jacobi).
__device__ void qrcp_rows(double* A, int n, int np, int* colperm, double* cn, double* cn0, double* vbuf,
                          double* redv, int* redi) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int j = tid; j < n; j += nt) {
    double s = 0.0;
    for (int i = 0; i < np; ++i) { const double v = A[(size_t)i * n + j]; s = fma(v, v, s); }
    cn[j] = sqrt(s);
    cn0[j] = cn[j];
    colperm[j] = j;
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    // pivot: largest remaining column norm, ties to the smallest index
    double best = -1.0;
    int bj = n;
    for (int j = k + tid; j < n; j += nt) {
      const double v = cn[j];
      if (v > best) { best = v; bj = j; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
      if (ob > best || (ob == best && oj < bj)) { best = ob; bj = oj; }
    }
    if (lane == 0) { redv[warp] = best; redi[warp] = bj; }
    __syncthreads();
    if (tid == 0) {
      double b = redv[0];
      int q = redi[0];
      for (int w = 1; w < nw; ++w)
        if (redv[w] > b || (redv[w] == b && redi[w] < q)) { b = redv[w]; q = redi[w]; }
      redi[32] = q;
    }
    __syncthreads();
    const int p = redi[32];
    if (p != k && p < n) {
      for (int i = tid; i < np; i += nt) {
        const double t = A[(size_t)i * n + k];
        A[(size_t)i * n + k] = A[(size_t)i * n + p];
        A[(size_t)i * n + p] = t;
      }
      if (tid == 0) {
        double t = cn[k]; cn[k] = cn[p]; cn[p] = t;
        t = cn0[k]; cn0[k] = cn0[p]; cn0[p] = t;
        const int c = colperm[k]; colperm[k] = colperm[p]; colperm[p] = c;
      }
    }
    __syncthreads();
    // Householder reflector of column k below the diagonal
    double s = 0.0;
    for (int i = k + 1 + tid; i < np; i += nt) { const double v = A[(size_t)i * n + k]; s = fma(v, v, s); }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) redv[warp] = s;
    __syncthreads();
    double xn2 = 0.0;
    for (int w = 0; w < nw; ++w) xn2 += redv[w];
    const double alpha = A[(size_t)k * n + k];
    double tau = 0.0, beta = alpha;
    if (xn2 > 0.0) {
      beta = -copysign(sqrt(fma(alpha, alpha, xn2)), alpha);
      tau = (beta - alpha) / beta;
      const double scal = 1.0 / (alpha - beta);
      for (int i = k + 1 + tid; i < np; i += nt) vbuf[i] = A[(size_t)i * n + k] * scal;
    }
    __syncthreads();
    for (int i = k + 1 + tid; i < np; i += nt) A[(size_t)i * n + k] = 0.0;
    if (tid == 0) A[(size_t)k * n + k] = beta;
    // apply (I - tau v v^T) to the trailing columns and downdate their norms
    for (int j = k + 1 + tid; j < n; j += nt) {
      double akj = A[(size_t)k * n + j];
      if (tau != 0.0) {
        double w = akj;
#pragma unroll 8
        for (int i = k + 1; i < np; ++i) w = fma(vbuf[i], A[(size_t)i * n + j], w);
        w *= tau;
        akj -= w;
        A[(size_t)k * n + j] = akj;
#pragma unroll 8
        for (int i = k + 1; i < np; ++i) A[(size_t)i * n + j] = fma(-vbuf[i], w, A[(size_t)i * n + j]);
      }
      const double c = cn[j];
      if (c != 0.0) {
        double t = fabs(akj) / c;
        t = fmax(0.0, (1.0 - t) * (1.0 + t));
        const double r = c / cn0[j];
        if (t * r * r <= 1.4901161193847656e-08) {
          double s2 = 0.0;
          for (int i = k + 1; i < np; ++i) { const double v = A[(size_t)i * n + j]; s2 = fma(v, v, s2); }
          cn[j] = sqrt(s2);
          cn0[j] = cn[j];
        } else {
          cn[j] = c * sqrt(t);
        }
      }
    }
    __syncthreads();
  }
}

template <int PW>
__global__ void __launch_bounds__(512) k_jacobi_warp(JacobiArgs a, int use_smem) {
  extern __shared__ double smem[];
  const double nu = a.noise_u > 0.0 ? a.noise_u : 0x1.0p-52;
  __shared__ int s_rot, s_na;
  __shared__ double s_thr2;
  constexpr int LOGPW = PW == 1 ? 0 : PW == 2 ? 1 : PW == 4 ? 2 : PW == 8 ? 3 : PW == 16 ? 4 : 5;
  constexpr int SH = 5 - LOGPW;                    // lane >> SH = pair index within the warp
  const int mat = blockIdx.x;
  const int n = a.n, np = a.n_pad;
  double* A = use_smem ? smem : a.W + (size_t)mat * np * n;
  double* nrm = use_smem ? smem + (size_t)np * n : smem;
  double* dsc = nrm + np;                          // [np] row scales
  double* cn = dsc + np;                           // [np] column norms (QR)
  double* cn0 = cn + np;                           // [np] reference norms (QR)
  double* vbuf = cn0 + np;                         // [np] Householder vector
  double* redv = vbuf + np;                        // [33] block reductions
  double* wbuf = redv + 34;                        // global rows: [nwarps][n] row staging
  int* act = (int*)(wbuf + (use_smem ? 0 : (size_t)(blockDim.x >> 5) * n));   // [np + 1] active rows
  int* colperm = act + np + 2;                     // [np] column permutation of R
  int* redi = colperm + np;                        // [33]
  const double* Mm = a.M + (size_t)mat * n * n;
  for (int idx = threadIdx.x; idx < np * n; idx += blockDim.x) A[idx] = idx < n * n ? Mm[idx] : 0.0;
  for (int r = threadIdx.x; r < np; r += blockDim.x) dsc[r] = 1.0;
  __syncthreads();
  qrcp_rows(A, n, np, colperm, cn, cn0, vbuf, redv, redi);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const double tol = (double)np * 0x1.0p-53;
  bool converged = false;

  for (int sweep = 0; sweep < a.max_sweeps && !converged; ++sweep) {
    // fold the scales into the rows and take exact squared norms
    for (int r = warp; r < np; r += nwarps) {
      const double dr = dsc[r];
      double s = 0.0;
      double* row = A + (size_t)r * n;
      for (int c = lane; c < n; c += 32) {
        double v = row[c];
        if (dr != 1.0) { v *= dr; row[c] = v; }
        s = fma(v, v, s);
      }
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) { nrm[r] = s; dsc[r] = 1.0; }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (sweep == 0) {
        double f = 0.0;
        for (int r = 0; r < np; ++r) f += nrm[r];
        s_thr2 = f * (0.25 * nu * nu);
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
      for (int base = warp * PW; base < npairs; base += nwarps * PW) {
        int Pj[PW], Qj[PW];
        double g[PW];
#pragma unroll
        for (int j = 0; j < PW; ++j) {
          const int pk = base + j;
          int P = -1, Q = -1;
          if (pk < npairs) {
            P = act[pk == 0 ? 0 : 1 + (pk - 1 + step) % (nap - 1)];
            Q = act[1 + (nap - 2 - pk + step) % (nap - 1)];
          }
          Pj[j] = P; Qj[j] = Q;
          double acc = 0.0;
          if (P >= 0 && Q >= 0) {
            const double* ap = A + (size_t)P * n;
            const double* aq = A + (size_t)Q * n;
            for (int c = lane; c < n; c += 32) acc = fma(ap[c], aq[c], acc);
          }
          g[j] = acc;
        }
        const double gs = batched_reduce<PW>(g, lane);
        // this lane's pair
        const int jm = lane >> SH;
        int P = -1, Q = -1;
#pragma unroll
        for (int j = 0; j < PW; ++j) if (j == jm) { P = Pj[j]; Q = Qj[j]; }
        bool rot = false;
        double mu1 = 0.0, mu2 = 0.0, cs = 1.0, nal = 0.0, nbe = 0.0, al = 0.0, be = 0.0;
        if (P >= 0 && Q >= 0) {
          al = nrm[P]; be = nrm[Q];
          const double dp = dsc[P], dq = dsc[Q];
          const double gam = dp * dq * gs;
          rot = al > 0.0 && be > 0.0 && fabs(gam) > tol * sqrt(al) * sqrt(be);
          if (rot) {
            const double zeta = (be - al) / (2.0 * gam);
            double t;
            if (fabs(zeta) > 1e150) t = 0.5 / zeta;
            else t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
            cs = 1.0 / sqrt(fma(t, t, 1.0));
            mu1 = t * (dq / dp);
            mu2 = t * (dp / dq);
            nal = fma(-t, gam, al);
            nbe = fma(t, gam, be);
          }
        }
        bool fixany = false;
#pragma unroll
        for (int j = 0; j < PW; ++j) {
          const int src = j << SH;
          const bool rj = __shfl_sync(0xffffffffu, rot, src);
          if (!rj) continue;                                   // warp-uniform
          const double m1 = __shfl_sync(0xffffffffu, mu1, src);
          const double m2 = __shfl_sync(0xffffffffu, mu2, src);
          double* ap = A + (size_t)Pj[j] * n;
          double* aq = A + (size_t)Qj[j] * n;
          for (int c = lane; c < n; c += 32) {
            const double x = ap[c], y = aq[c];
            ap[c] = fma(-m1, y, x);
            aq[c] = fma(m2, x, y);
          }
        }
        const bool own = (lane & ((1 << SH) - 1)) == 0;
        const bool fixP = rot && nal < 0.01 * al, fixQ = rot && nbe < 0.01 * be;
        if (own && rot) {
          nrm[P] = nal; nrm[Q] = nbe;
          dsc[P] *= cs; dsc[Q] *= cs;
          ++myrot;
        }
        fixany = __any_sync(0xffffffffu, fixP || fixQ);
        if (fixany) {                                          // rare: recompute from the rows
          __syncwarp();
#pragma unroll
          for (int j = 0; j < PW; ++j) {
            const int src = j << SH;
            const bool fp = __shfl_sync(0xffffffffu, fixP, src), fq = __shfl_sync(0xffffffffu, fixQ, src);
            for (int side = 0; side < 2; ++side) {
              if (!(side == 0 ? fp : fq)) continue;            // warp-uniform
              const int r = side == 0 ? Pj[j] : Qj[j];
              const double* row = A + (size_t)r * n;
              const double dr = dsc[r];
              double s = 0.0;
              for (int c = lane; c < n; c += 32) s = fma(row[c], row[c], s);
              for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
              if (lane == 0) nrm[r] = s * dr * dr;
            }
          }
          __syncwarp();
        }
      }
      if (myrot) atomicAdd(&s_rot, myrot);
      __syncthreads();
    }
    converged = (s_rot == 0);
    __syncthreads();
  }
  // true rows and exact norms
  for (int r = warp; r < np; r += nwarps) {
    const double dr = dsc[r];
    double s = 0.0;
    double* row = A + (size_t)r * n;
    for (int c = lane; c < n; c += 32) {
      double v = row[c];
      if (dr != 1.0) { v *= dr; row[c] = v; }
      s = fma(v, v, s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) nrm[r] = sqrt(s);
  }
  __syncthreads();
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
  // rows of W are right vectors of M: undo the column pivoting of R
  if (use_smem) {
    double* Wm = a.W + (size_t)mat * np * n;
    for (int idx = threadIdx.x; idx < np * n; idx += blockDim.x) {
      const int r = idx / n, c = idx - r * n;
      Wm[(size_t)r * n + colperm[c]] = A[idx];
    }
  } else {
    double* buf = wbuf + (size_t)warp * n;
    for (int r = warp; r < np; r += nwarps) {
      double* row = A + (size_t)r * n;
      for (int c = lane; c < n; c += 32) buf[c] = row[c];
      __syncwarp();
      for (int c = lane; c < n; c += 32) row[colperm[c]] = buf[c];
      __syncwarp();
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double s1 = sg[0];
    if (a.lns1) a.lns1[mat] = s1 > 0.0 ? log(s1) : -INFINITY;
    const double tau = (a.zero_rel > 0.0 ? a.zero_rel : (double)n * 0x1.0p-52) * s1;
    int cnt = 0;
    for (int r = 0; r < np; ++r) cnt += sg[r] > tau;
    a.nnz[mat] = s1 > 0.0 ? cnt : 0;
    if (a.mflags && !converged) a.mflags[mat] |= FLAG_NOCONV;
  }
}

template <int PW>
static cudaError_t launch_warp_variant(const JacobiArgs& a, int threads, cudaStream_t st) {
  const int n = a.n, np = a.n_pad;
  const size_t rows_bytes = (size_t)np * n * sizeof(double);
  const size_t aux = (size_t)np * 5 * sizeof(double) + 34 * sizeof(double) +
                     (size_t)(2 * np + 2 + 34) * sizeof(int);
  const int use_smem = (rows_bytes + aux) <= 200 * 1024;
  // Rows in the global workspace: stage one row per warp in shared memory for
  // the final column permutation, and ask for enough shared memory that one
  // CTA runs per SM, so the rows of the resident matrices stay in L2.
  const size_t staging = (size_t)(threads / 32) * n * sizeof(double);
  const size_t smem = use_smem ? rows_bytes + aux : std::max<size_t>(aux + staging, 120 * 1024);
  static std::atomic<uint64_t> attr{0};
  cudaError_t e = raise_smem_limit(k_jacobi_warp<PW>, 200 * 1024 + 64, attr);
  if (e != cudaSuccess) return e;
  k_jacobi_warp<PW><<<a.S, threads, smem, st>>>(a, use_smem);
  return cudaGetLastError();
}

cudaError_t launch_jacobi(const JacobiArgs& a, cudaStream_t st) {
  if (a.S <= 0) return cudaSuccess;
  if (a.n > 32) {
    // pairs per warp so that one pass of the warps covers a step
    const int npairs = a.n_pad / 2;
    const int threads = a.n <= 64 ? 256 : 512;
    const int nw = threads / 32;
    int pw = 1;
    while (pw < 32 && pw * nw < npairs) pw <<= 1;
    switch (pw) {
      case 1: return launch_warp_variant<1>(a, threads, st);
      case 2: return launch_warp_variant<2>(a, threads, st);
      case 4: return launch_warp_variant<4>(a, threads, st);
      case 8: return launch_warp_variant<8>(a, threads, st);
      case 16: return launch_warp_variant<16>(a, threads, st);
      default: return launch_warp_variant<32>(a, threads, st);
    }
  }

  // n <= 32: lane groups of G < 32 lanes per pair

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
  static std::atomic<uint64_t> attr{0};
  cudaError_t e = raise_smem_limit(k_jacobi, 200 * 1024 + 64, attr);
  if (e != cudaSuccess) return e;
  k_jacobi<<<a.S, threads, smem, st>>>(a, use_smem, G);
  return cudaGetLastError();
}

}  // namespace mctrg
