// K2, bidiagonalization route: the SVD of a level matrix (Sec. II, Eq. exactSVD)
// at the flop count of a bidiagonal reduction, (8/3) n^3, instead of the
// repeated sweeps of one-sided Jacobi, with singular vectors computed only
// for the indices the sampler keeps.
//
//  1. k_bidiag        Householder bidiagonalization M = Q_L B Q_R^T (Golub and
//                     Kahan 1965), one CTA per matrix; d, e of the upper
//                     bidiagonal B and the right reflectors kept in place.
//  2. k_bd_bisect     every singular value of B by bisection on Sturm counts of
//                     the Golub-Kahan tridiagonal T (zero diagonal, off-
//                     diagonal d_0 e_0 d_1 e_1 ... d_{n-1}; eigenvalues +-s_i),
//                     one thread per singular value.  The count is the number
//                     of sign changes of the leading principal minors P_k of
//                     T - x I, P_k = -x P_{k-1} - o_{k-2}^2 P_{k-2} (Barth,
//                     Martin and Wilkinson 1967), with power-of-two rescaling
//                     against underflow; it is the exact count of a matrix
//                     within a few ulps of T entrywise, so each value carries
//                     an absolute error of a few eps |B|, the accuracy class
//                     of LAPACK's SVD.  FP32 counts narrow each bracket (their
//                     rounding is relative too), FP64 counts verify it, and
//                     Illinois steps on det(T - x I) finish isolated values.
//  (the sampler then chooses the kept indices)
//  3. k_bd_invit      right singular vectors of B for the kept indices: inverse
//                     iteration on T - s I (LU with partial pivoting) whose
//                     eigenvector for +s is (v_0, u_0, v_1, u_1, ...),
//                     reorthogonalized within clusters of close kept values
//                     (as LAPACK's dstein), one lane per kept vector.
//  4. k_bd_backtr     v = Q_R v_B through the stored reflectors, written as
//                     s v (the scaling of a one-sided Jacobi row).
//
// On GB300 FP64 runs at 1/64 of the FP32 rate, so every stage is laid out
// for lane parallelism: no stage runs a long dependent FP64 chain in a
// single lane per matrix (the implicit-shift QR of the bidiagonal would).
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "kernels_bd.h"

namespace mctrg {

namespace {
constexpr int kBdThreads = 256;
constexpr int kBisThreads = 256;
constexpr int kInvitIters = 3;
constexpr int kCh = 8;          // steps per block of the inverse iteration's serial loops
constexpr double kEps = 0x1.0p-52;

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s += red[w];
  return s;
}

__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s = fmax(s, red[w]);
  return s;
}

// Biased exponent field of a double (0 for zero and subnormals).
__device__ __forceinline__ int exp_field(double x) { return (__double2hiint(x) >> 20) & 0x7ff; }
}  // namespace

// ---------------------------------------------------------------------------
// 1. Householder bidiagonalization, one CTA (8 warps) per matrix.  Step k:
//    left reflector H = I - tau v v^T, v = (1, x_{k+1..}/(alpha - beta)), from
//    column k; w_j = tau (A[k][j] + sum_{i>k} v_i A[i][j]); row k becomes
//    A[k][j] - w_j, from which the right reflector G = I - tauR u u^T,
//    u = (1, r_{k+2..}/(r_{k+1} - betaR)), is formed; then one fused pass per
//    row i > k applies both: a = A[i][:] - v_i w, y = tauR a.u, a -= y u, and
//    hands column k+1 of the result to step k+1 together with step k+1's
//    column dots (w is linear in the unnormalized column, so the fused pass
//    accumulates sum_i A'[i][k+1] A'[i][:] from the rows it holds).  The
//    trailing matrix is read and written once per step.
//    Lane l holds the trailing columns k+1+l, k+1+l+32, ... of a row in
//    registers; the number of live 32-column chunks, QL, is a template
//    argument chosen per step, so no FMA is issued for a finished column.  A
//    warp takes up to four rows at a time and reduces their dots together;
//    the right reflector enters as us = sqrt(tauR) u (G = I - us us^T).

// 4-value warp sum: on return lanes 0, 8, 16, 24 hold the sums of p0, p1, p2, p3.
__device__ __forceinline__ double reduce4(double p0, double p1, double p2, double p3, int lane) {
  const bool hi16 = lane & 16, hi8 = lane & 8;
  double q0 = hi16 ? p2 : p0, q1 = hi16 ? p3 : p1;
  const double r0 = hi16 ? p0 : p2, r1 = hi16 ? p1 : p3;
  q0 += __shfl_xor_sync(0xffffffffu, r0, 16);
  q1 += __shfl_xor_sync(0xffffffffu, r1, 16);
  double t = hi8 ? q1 : q0;
  const double tr = hi8 ? q0 : q1;
  t += __shfl_xor_sync(0xffffffffu, tr, 8);
  t += __shfl_xor_sync(0xffffffffu, t, 4);
  t += __shfl_xor_sync(0xffffffffu, t, 2);
  t += __shfl_xor_sync(0xffffffffu, t, 1);
  return t;
}

struct BdStep {
  double* A;
  const double* vcol;
  const double* wv;
  const double* uv;
  double* wpart;
  int n, k, lane, warp;
};

// w pass: per-warp partial sums sum_{i>k} v_i A[i][c] over the warp's rows.
template <int QL>
__device__ __forceinline__ void bd_w_pass(const BdStep& s) {
  constexpr int NW = kBdThreads / 32;
  const int n = s.n, c0 = s.k + 1 + s.lane;
  double acc[QL];
#pragma unroll
  for (int q = 0; q < QL; ++q) acc[q] = 0.0;
  for (int i = s.k + 1 + s.warp; i < n; i += NW) {
    const double vi = s.vcol[i];
    const double* row = s.A + (size_t)i * n;
#pragma unroll
    for (int q = 0; q < QL; ++q)
      if (c0 + 32 * q < n) acc[q] = fma(vi, row[c0 + 32 * q], acc[q]);
  }
#pragma unroll
  for (int q = 0; q < QL; ++q)
    if (c0 + 32 * q < n) s.wpart[s.warp * n + c0 + 32 * q] = acc[q];
}

// R consecutive rows i0 .. i0+R-1 (all < n) of the fused pass: a = A[i] - v_i w,
// y = a.us (us = sqrt(tauR) u, so the right update is a -= y us), reduced for
// the R rows together; returns this lane's share of the new column k+1 squared.
template <int QL, int R>
__device__ __forceinline__ double bd_rows(const BdStep& s, int i0, const double (&wr)[QL], const double (&ur)[QL],
                                          double (&acc)[QL], double* vcol_out) {
  const int n = s.n, k = s.k, lane = s.lane, c0 = k + 1 + lane;
  double av[R][QL];
  double y[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const double vi = s.vcol[i0 + r];
    const double* row = s.A + (size_t)(i0 + r) * n;
#pragma unroll
    for (int q = 0; q < QL; ++q) {
      // columns past the edge load the last column and carry zero multipliers
      // (wr = ur = 0 there), so every FMA is issued unconditionally
      av[r][q] = fma(-vi, wr[q], row[min(c0 + 32 * q, n - 1)]);
      y[r] = fma(av[r][q], ur[q], y[r]);
    }
  }
  const double t = reduce4(y[0], y[1], y[2], y[3], lane);
  double yr[R];
#pragma unroll
  for (int r = 0; r < R; ++r) yr[r] = __shfl_sync(0xffffffffu, t, 8 * r);
  double nsq = 0.0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = i0 + r;
    double* row = s.A + (size_t)i * n;
#pragma unroll
    for (int q = 0; q < QL; ++q) {
      const double v = fma(-yr[r], ur[q], av[r][q]);
      av[r][q] = v;
      if (c0 + 32 * q < n) row[c0 + 32 * q] = v;
    }
    if (lane == 0) {
      vcol_out[i] = av[r][0];                    // column k+1 for the next step
      if (i > k + 1) nsq = fma(av[r][0], av[r][0], nsq);
    }
    // the next step's column dots: sum_{i > k+1} A'[i][k+1] A'[i][c], c > k+1
    // (edge lanes accumulate values that are never written out)
    const double xk1 = __shfl_sync(0xffffffffu, av[r][0], 0);
    const double xm = i > k + 1 ? xk1 : 0.0;
#pragma unroll
    for (int q = 0; q < QL; ++q) acc[q] = fma(xm, av[r][q], acc[q]);
  }
  return nsq;
}

// fused pass: rows i > k, RPW per warp (full groups), then the leftover rows of
// the last group one at a time; leaves this warp's share of the next step's
// column dots in wpart and returns its sum of the new column k+1 squared below
// the diagonal (valid in lane 0).
template <int QL>
__device__ __forceinline__ double bd_fused_pass(const BdStep& s, double* vcol_out) {
  constexpr int NW = kBdThreads / 32;
  constexpr int RPW = QL <= 8 ? 4 : (QL <= 16 ? 2 : 1);   // rows per warp and pass (register budget)
  const int n = s.n, k = s.k, c0 = k + 1 + s.lane;
  double wr[QL], ur[QL];
#pragma unroll
  for (int q = 0; q < QL; ++q) {
    const bool in = c0 + 32 * q < n;
    wr[q] = in ? s.wv[c0 + 32 * q] : 0.0;
    ur[q] = in ? s.uv[c0 + 32 * q] : 0.0;
  }
  double nsq = 0.0;
  double acc[QL];
#pragma unroll
  for (int q = 0; q < QL; ++q) acc[q] = 0.0;
  int i0 = k + 1 + RPW * s.warp;
  for (; i0 + RPW <= n; i0 += RPW * NW) nsq += bd_rows<QL, RPW>(s, i0, wr, ur, acc, vcol_out);
  if (RPW > 1)
    for (int i = i0; i < n && i < i0 + RPW; ++i) nsq += bd_rows<QL, 1>(s, i, wr, ur, acc, vcol_out);
#pragma unroll
  for (int q = 0; q < QL; ++q)
    if (c0 + 32 * q < n && c0 + 32 * q > k + 1) s.wpart[s.warp * n + c0 + 32 * q] = acc[q];
  return nsq;
}

template <int QL, int NQ>
struct BdDispatch {
  static __device__ __forceinline__ void w_pass(int ql, const BdStep& s) {
    if (ql == QL) bd_w_pass<QL>(s); else BdDispatch<QL + 1, NQ>::w_pass(ql, s);
  }
  static __device__ __forceinline__ double fused(int ql, const BdStep& s, double* vo) {
    if (ql == QL) return bd_fused_pass<QL>(s, vo);
    return BdDispatch<QL + 1, NQ>::fused(ql, s, vo);
  }
};
template <int NQ>
struct BdDispatch<NQ + 1, NQ> {
  static __device__ __forceinline__ void w_pass(int, const BdStep&) {}
  static __device__ __forceinline__ double fused(int, const BdStep&, double*) { return 0.0; }
};

// Wide form (sides above 1024, whose rows no longer fit in registers; the
// matrix is in the global workspace): each step's fused pass sweeps a group of
// R rows twice -- the first sweep forms a = A[i] - v_i w and y = a.us, the
// second recomputes a, applies a -= y us, stores it and adds the next step's
// column dots into this warp's row of wpart (shared memory; lane l owns the
// columns k+1+l+32j throughout, so no other lane touches them).  One FMA per
// element more than the register form; the same operations in the same order
// otherwise.
__device__ __forceinline__ void bdw_w_pass(const BdStep& s) {
  constexpr int NW = kBdThreads / 32;
  const int n = s.n, k = s.k;
  double* wp = s.wpart + (size_t)s.warp * n;
  for (int c = k + 1 + s.lane; c < n; c += 32) wp[c] = 0.0;
  for (int i = k + 1 + s.warp; i < n; i += NW) {
    const double vi = s.vcol[i];
    const double* row = s.A + (size_t)i * n;
    for (int c = k + 1 + s.lane; c < n; c += 32) wp[c] = fma(vi, row[c], wp[c]);
  }
}

template <int R>
__device__ __forceinline__ double bdw_rows(const BdStep& s, int i0, double* vcol_out) {
  const int n = s.n, k = s.k, lane = s.lane;
  double vi[R];
  double* row[R];
  double y[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int r = 0; r < R; ++r) {
    vi[r] = s.vcol[i0 + r];
    row[r] = s.A + (size_t)(i0 + r) * n;
  }
#pragma unroll 2
  for (int c = k + 1 + lane; c < n; c += 32) {
    const double wc = s.wv[c], uc = s.uv[c];
#pragma unroll
    for (int r = 0; r < R; ++r) y[r] = fma(fma(-vi[r], wc, row[r][c]), uc, y[r]);
  }
  const double t = reduce4(y[0], y[1], y[2], y[3], lane);
  double yr[R], xm[R];
  double nsq = 0.0;
  const double wk = s.wv[k + 1], uk = s.uv[k + 1];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    yr[r] = __shfl_sync(0xffffffffu, t, 8 * r);
    const int i = i0 + r;
    // column k+1 of the updated row (every lane forms it; lane 0's sweep below
    // writes the same value)
    const double x = fma(-yr[r], uk, fma(-vi[r], wk, row[r][k + 1]));
    if (lane == 0) {
      vcol_out[i] = x;                           // column k+1 for the next step
      if (i > k + 1) nsq = fma(x, x, nsq);
    }
    xm[r] = i > k + 1 ? x : 0.0;
  }
  __syncwarp();
  double* wp = s.wpart + (size_t)s.warp * n;
#pragma unroll 2
  for (int c = k + 1 + lane; c < n; c += 32) {
    const double wc = s.wv[c], uc = s.uv[c];
    double acc = wp[c];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const double v = fma(-yr[r], uc, fma(-vi[r], wc, row[r][c]));
      row[r][c] = v;
      acc = fma(xm[r], v, acc);
    }
    wp[c] = acc;
  }
  return nsq;
}

__device__ __forceinline__ double bdw_fused_pass(const BdStep& s, double* vcol_out) {
  constexpr int NW = kBdThreads / 32;
  constexpr int RPW = 4;
  const int n = s.n, k = s.k;
  double* wp = s.wpart + (size_t)s.warp * n;
  for (int c = k + 1 + s.lane; c < n; c += 32) wp[c] = 0.0;
  double nsq = 0.0;
  int i0 = k + 1 + RPW * s.warp;
  for (; i0 + RPW <= n; i0 += RPW * NW) nsq += bdw_rows<RPW>(s, i0, vcol_out);
  for (int i = i0; i < n && i < i0 + RPW; ++i) nsq += bdw_rows<1>(s, i, vcol_out);
  return nsq;
}

// NQ > 0: the register form for sides up to 32 NQ; NQ = 0: the wide form.
template <int NQ>
__global__ void __launch_bounds__(kBdThreads) k_bidiag(BidiagArgs a, int use_smem) {
  extern __shared__ double sm[];
  int n = a.n;
  const int mat = blockIdx.x;
  constexpr int NW = kBdThreads / 32;
  const double* Mm;
  double* Wm;
  double* bd;
  if (a.items) {                     // ragged: this matrix's size and buffers
    const SvdItem& t = a.items[mat];
    n = t.n; Mm = t.M; Wm = t.W; bd = t.bd;
    use_smem = NQ > 0 && ((size_t)n * n + (size_t)(3 + NW) * n + 32) * sizeof(double) <= 200 * 1024;
  } else {
    Mm = a.M + (size_t)mat * n * n; Wm = a.W + (size_t)mat * n * n; bd = a.bd + (size_t)mat * 3 * n;
  }
  double* A = use_smem ? sm : Wm;
  double* base = use_smem ? sm + (size_t)n * n : sm;
  double* vcol = base;               // [n] column k (then v), below and on the diagonal
  double* wv = vcol + n;             // [n] w
  double* uv = wv + n;               // [n] u
  double* wpart = uv + n;            // [NW][n] per-warp partial column dots
  double* red = wpart + (size_t)NW * n;   // [32]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ double s_xn2;
  for (int e = tid; e < n * n; e += kBdThreads) A[e] = Mm[e];
  for (int e = tid; e < 3 * n; e += kBdThreads) bd[e] = 0.0;
  __syncthreads();
  {
    double sq = 0.0;
    for (int i = tid; i < n; i += kBdThreads) {
      const double x = A[(size_t)i * n];
      vcol[i] = x;
      if (i > 0) sq = fma(x, x, sq);
    }
    const double t = block_sum(sq, red);
    if (tid == 0) s_xn2 = t;
  }
  __syncthreads();
  BdStep st{A, vcol, wv, uv, wpart, n, 0, lane, warp};
  // the column dots of step 0 with the unnormalized column 0: later steps get
  // theirs from the previous fused pass (w is linear in the column)
  if (n > 1) {
    if constexpr (NQ == 0) bdw_w_pass(st);
    else BdDispatch<1, NQ>::w_pass((n - 1 + 31) >> 5, st);
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    st.k = k;
    const int ql = (n - k - 1 + 31) >> 5;     // live 32-column chunks right of column k
    // ---- left reflector from column k
    const double xn2 = s_xn2;
    const double alpha = vcol[k];
    double tau = 0.0, beta = alpha, scal = 0.0;
    if (xn2 > 0.0) {
      beta = -copysign(sqrt(fma(alpha, alpha, xn2)), alpha);
      tau = (beta - alpha) / beta;
      scal = 1.0 / (alpha - beta);
      for (int i = k + 1 + tid; i < n; i += kBdThreads) vcol[i] *= scal;
    }
    if (tid == 0) bd[k] = beta;
    if (k == n - 1) break;
    __syncthreads();
    // ---- w = tau (A[k][:] + v^T A[k+1:, :]) on columns > k; wpart holds
    //      sum_{i>k} x_i A[i][:] for the unnormalized column x (v = scal x)
    if (tau != 0.0) {
      for (int jj = k + 1 + tid; jj < n; jj += kBdThreads) {
        double sum = 0.0;
        for (int w = 0; w < NW; ++w) sum += wpart[w * n + jj];
        wv[jj] = tau * fma(scal, sum, A[(size_t)k * n + jj]);
      }
    } else {
      for (int jj = k + 1 + tid; jj < n; jj += kBdThreads) wv[jj] = 0.0;
    }
    __syncthreads();
    // ---- row k after the left reflector, and the right reflector from it
    double sq = 0.0;
    for (int jj = k + 2 + tid; jj < n; jj += kBdThreads) {
      const double r = A[(size_t)k * n + jj] - wv[jj];
      uv[jj] = r;
      sq = fma(r, r, sq);
    }
    const double yn2 = block_sum(sq, red);
    const double ar = A[(size_t)k * n + k + 1] - wv[k + 1];
    double taur = 0.0, betar = ar;
    if (yn2 > 0.0) {
      betar = -copysign(sqrt(fma(ar, ar, yn2)), ar);
      taur = (betar - ar) / betar;
      const double scal = 1.0 / (ar - betar);
      const double rt = sqrt(taur);               // G = I - us us^T with us = sqrt(tauR) u
      for (int jj = k + 2 + tid; jj < n; jj += kBdThreads) {
        const double u = uv[jj] * scal;
        uv[jj] = rt * u;
        A[(size_t)k * n + jj] = u;              // kept for the back-transformation
      }
    } else {
      for (int jj = k + 2 + tid; jj < n; jj += kBdThreads) uv[jj] = 0.0;
    }
    if (tid == 0) { uv[k + 1] = sqrt(taur); bd[n + k] = betar; bd[2 * n + k] = taur; }
    __syncthreads();
    // ---- fused pass over rows i > k
    double nsq;
    if constexpr (NQ == 0) nsq = bdw_fused_pass(st, vcol);
    else nsq = BdDispatch<1, NQ>::fused(ql, st, vcol);
    __syncthreads();                            // everyone done with red / vcol reads
    if (lane == 0) red[warp] = nsq;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < NW; ++w) t += red[w];
      s_xn2 = t;
    }
    __syncthreads();
  }
  if (use_smem) {
    __syncthreads();
    for (int e = tid; e < n * n; e += kBdThreads) Wm[e] = A[e];
  }
}

// ---------------------------------------------------------------------------
// 2. Sturm count and determinant: for the bidiagonal whose Golub-Kahan
//    tridiagonal has squared off-diagonals oo[0 .. 2n-2] (normalized so that
//    |T| <= 1) and x > 0, returns #{s_i < x} (sign changes of P_0 .. P_2n count
//    the eigenvalues of T below x: the n values -s_i and those s_i < x) and
//    det(T - x I) = P_2n = f 2^fe.  Four steps between checks of the pair's
//    magnitude: after a check the larger of |P_k|, |P_{k-1}| is >= 2^-100, and
//    four steps shrink it by at most 2^-416 (x >= 2^-53, one cancellation), so
//    nothing underflows.  Unscaled, every P_k is at most about 1 in magnitude
//    at any n (the eigenvalues of each leading block of the zero-diagonal T
//    come in +- pairs within [-1, 1], so |P_k| <= prod |x^2 - l^2| <=
//    (1 + 2^-20)^k for x <= 1 + 2^-20): the stored values exceed 1 only by the
//    factors a rescaling put in.
#define MCTRG_STURM_STEP(K)                                          \
  {                                                                  \
    double q = fma(-x, p, -oo[(K) - 2] * pp);                        \
    long long qb = __double_as_longlong(q);                          \
    if ((qb << 1) == 0) {                                            \
      q = -p * 0x1.0p-60;                                            \
      qb = __double_as_longlong(q);                                  \
    }                                                                \
    neg += (int)((unsigned long long)(qb ^ __double_as_longlong(p)) >> 63); \
    pp = p;                                                          \
    p = q;                                                           \
  }

__device__ __forceinline__ int sturm_eval(const double* __restrict__ oo, int n, double x, double& f, int& fe) {
  double pp = 1.0, p = -x;
  int neg = 1, E = 0;
  const int m = 2 * n;
  int k = 2;
  for (; k + 3 <= m; k += 4) {
    MCTRG_STURM_STEP(k)
    MCTRG_STURM_STEP(k + 1)
    MCTRG_STURM_STEP(k + 2)
    MCTRG_STURM_STEP(k + 3)
    const int em = max(exp_field(p), exp_field(pp));
    if (em < 1023 - 100) {                // rescale both by 2^(1023 - em), exactly
      const double sc = __hiloint2double((2046 - em) << 20, 0);
      p *= sc;
      pp *= sc;
      E -= 1023 - em;
    }
  }
  for (; k <= m; ++k) MCTRG_STURM_STEP(k)
  f = p;
  fe = E;
  return neg - n;
}
#undef MCTRG_STURM_STEP

// The same count in FP32 (FP64 runs at 1/64 of the FP32 rate on GB300).  Its
// rounding perturbs each off-diagonal and the shift x relatively (the terms
// are products, no absolute error enters), so it is the exact count for a
// matrix whose singular values are within a relative 2n 2^-23 of B's; it
// serves to narrow a bracket that FP64 counts then verify.  The pair is
// rescaled every step (x >= 2^-53 shrinks it by at most 2^-77 a step).
__device__ __forceinline__ int sturm_count_f32(const float* __restrict__ oo, int n, float x) {
  float pp = 1.0f, p = -x;
  int neg = 1;
  const int m = 2 * n;
  for (int k = 2; k <= m; ++k) {
    float q = fmaf(-x, p, -oo[k - 2] * pp);
    int qb = __float_as_int(q);
    if ((qb << 1) == 0) {
      q = -p * 0x1.0p-30f;
      qb = __float_as_int(q);
    }
    neg += (int)((unsigned)(qb ^ __float_as_int(p)) >> 31);
    pp = p;
    p = q;
    const int em = max((__float_as_int(p) >> 23) & 0xff, (__float_as_int(pp) >> 23) & 0xff);
    if (em < 127 - 40) {
      const float sc = __int_as_float((254 - em) << 23);
      p *= sc;
      pp *= sc;
    }
  }
  return neg - n;
}

// 2^d as a double, |d| clamped to 1000.
__device__ __forceinline__ double pow2i(int d) {
  d = max(-1000, min(1000, d));
  return __hiloint2double((1023 + d) << 20, 0);
}

// Each thread finds the values of its ranks: the bracket from a coarse grid of
// FP32 counts (the lowest bin starting at the zero bound), narrowed with FP32
// counts and verified with FP64 ones, then bisection while the bracket holds
// more than one value (geometric while it spans more than a factor 2), and
// Illinois steps (regula falsi on det(T - x I), halving the retained end's
// value when the same end moves twice) once it holds exactly one; three moves
// of one end in a row force a bisection step.  The bracket always satisfies
// count(lo) <= j < count(hi), so the result is within the final width of the
// count's crossing, whatever the interpolation does.
__global__ void __launch_bounds__(kBisThreads) k_bd_bisect(const double* bd, int n, int n_pad, double* sig,
                                                            int* perm, int* nnz, double* lns1, double zero_rel,
                                                            const SvdItem* items) {
  extern __shared__ double sm[];
  int mat = blockIdx.x;
  if (items) {                       // ragged: this matrix's size and buffers
    const SvdItem& t = items[mat];
    bd = t.bd; n = t.n; n_pad = t.n_pad; sig = t.sig; perm = t.perm; nnz = t.nnz; lns1 = t.lns1;
    zero_rel = t.zero_rel;
    mat = 0;
  }
  double* oo = sm;                                   // [2n]
  int* cnt = (int*)(oo + 2 * n);                     // [kBisThreads] FP32 grid counts
  float* oof = (float*)(cnt + kBisThreads);          // [2n] oo in FP32
  __shared__ double red[32];
  __shared__ double s_f0;
  __shared__ int s_zlo, s_nnz, s_e0;
  const int tid = threadIdx.x;
  const double* d = bd + (size_t)mat * 3 * n;
  const double* e = d + n;
  double* sg = sig + (size_t)mat * n_pad;
  // G = max_k (|o_{k-1}| + |o_k|) >= |T| >= s_1 (Gershgorin), omax = max |o_k| <= s_1
  double g = 0.0, om = 0.0;
  for (int k = tid; k < 2 * n - 1; k += kBisThreads) {
    const double ok = fabs((k & 1) ? e[k >> 1] : d[k >> 1]);
    const double on = (k + 1 < 2 * n - 1) ? fabs(((k + 1) & 1) ? e[(k + 1) >> 1] : d[(k + 1) >> 1]) : 0.0;
    g = fmax(g, ok + on);
    om = fmax(om, ok);
  }
  const double G = block_max(g, red);
  const double omax = block_max(om, red);
  if (!(G > 0.0)) {                                  // the zero matrix
    for (int r = tid; r < n_pad; r += kBisThreads) { sg[r] = 0.0; perm[(size_t)mat * n_pad + r] = r; }
    if (tid == 0) { nnz[mat] = 0; if (lns1) lns1[mat] = -INFINITY; }
    return;
  }
  const double invG = 1.0 / G;
  for (int k = tid; k < 2 * n - 1; k += kBisThreads) {
    const double ok = ((k & 1) ? e[k >> 1] : d[k >> 1]) * invG;
    oo[k] = ok * ok;
    oof[k] = (float)(ok * ok);
  }
  const double zr = zero_rel > 0.0 ? zero_rel : (double)n * kEps;
  const double tlo = zr * omax * invG;               // <= the zero threshold zr s_1 / G
  __syncthreads();
  // coarse grid of FP32 counts: x_t = (t + 1) / T, the last point above |T|
  const double top = 1.0 + 0x1.0p-20;
  {
    const double xt = (tid == kBisThreads - 1) ? top : (double)(tid + 1) / kBisThreads;
    cnt[tid] = sturm_count_f32(oof, n, (float)xt);
    if (tid == 0) {
      double f0;
      int e0;
      s_zlo = sturm_eval(oo, n, tlo, f0, e0);
      s_f0 = f0;
      s_e0 = e0;
    }
  }
  __syncthreads();
  const int zlo = s_zlo;
  const double tol = 0x1.0p-51;
  for (int r = tid; r < n; r += kBisThreads) {
    const int j = n - 1 - r;                         // ascending index of the r-th largest
    if (j < zlo) { sg[r] = 0.0; continue; }          // below tlo: a zero
    // FP32: the grid bin, then bisection (geometric across decades) to a
    // relative width of 2^-16
    int t = 0;
    while (t < kBisThreads - 1 && cnt[t] < j + 1) ++t;
    float lo32 = t > 0 ? (float)t / kBisThreads : (float)tlo;
    float hi32 = (t == kBisThreads - 1) ? (float)top : (float)(t + 1) / kBisThreads;
    for (int it = 0; it < 48 && hi32 > lo32 * (1.0f + 0x1.0p-16f); ++it) {
      const float x = (hi32 > 2.0f * lo32) ? sqrtf(lo32 * hi32) : 0.5f * (lo32 + hi32);
      if (!(x > lo32 && x < hi32)) break;
      if (sturm_count_f32(oof, n, x) >= j + 1) hi32 = x; else lo32 = x;
    }
    // FP64: verify the bracket widened by 2^-12 on each side (the FP32 count's
    // error is a relative 2n 2^-23 at most); if it does not hold, start from
    // the whole range [zero bound, |T|]
    double lo = fmax(tlo, (double)lo32 * (1.0 - 0x1.0p-12));
    double hi = fmin(top, (double)hi32 * (1.0 + 0x1.0p-12));
    // a bracket already within the tolerance (the small values: their FP32
    // bracket, a relative 2^-11 wide, is below 2^-51 |T| in absolute terms)
    // needs no FP64 count: the refinement below would not move it
    if (hi - lo <= tol) { sg[r] = G * (0.5 * (lo + hi)); continue; }
    double f_lo, f_hi;
    int e_lo, e_hi;
    int c_lo = sturm_eval(oo, n, lo, f_lo, e_lo);
    int c_hi = sturm_eval(oo, n, hi, f_hi, e_hi);
    if (!(c_lo <= j && c_hi >= j + 1)) {
      lo = tlo; c_lo = zlo; f_lo = s_f0; e_lo = s_e0;
      hi = top; c_hi = sturm_eval(oo, n, hi, f_hi, e_hi);
    }
    // FP64 refinement to 2^-51 |T|: Illinois steps while the bracket holds one
    // value, bisection otherwise
    int last = 0, run = 0;
    for (int it = 0; it < 80 && hi - lo > tol; ++it) {
      const bool interp = c_lo == j && c_hi == j + 1 && run < 3;
      // a bracket spanning more than a factor 2 is split geometrically (the
      // spectrum decays over many decades), a narrower one in the middle
      double x = (lo > 0.0 && hi > 2.0 * lo) ? sqrt(lo * hi) : 0.5 * (lo + hi);
      if (interp) {
        const int dd = e_lo - e_hi;
        const double al = fabs(f_lo) * (dd < 0 ? pow2i(dd) : 1.0);
        const double ah = fabs(f_hi) * (dd > 0 ? pow2i(-dd) : 1.0);
        const double den = al + ah;
        if (den > 0.0) {
          const double xi = lo + (al / den) * (hi - lo);
          if (xi > lo && xi < hi) x = xi;
        }
      }
      double f;
      int fe;
      const int c = sturm_eval(oo, n, x, f, fe);
      if (c >= j + 1) {
        hi = x; c_hi = c; f_hi = f; e_hi = fe;
        if (interp && last == 1) e_lo -= 1;          // Illinois: halve the retained end
        run = (last == 1) ? run + 1 : 1;
        last = 1;
      } else {
        lo = x; c_lo = c; f_lo = f; e_lo = fe;
        if (interp && last == -1) e_hi -= 1;
        run = (last == -1) ? run + 1 : 1;
        last = -1;
      }
      if (!interp) run = 0;
    }
    sg[r] = G * (0.5 * (lo + hi));
  }
  for (int r = n + tid; r < n_pad; r += kBisThreads) sg[r] = 0.0;
  for (int r = tid; r < n_pad; r += kBisThreads) perm[(size_t)mat * n_pad + r] = r;
  if (tid == 0) s_nnz = 0;
  __syncthreads();
  const double s1 = sg[0];
  const double tau = zr * s1;
  int c = 0;
  for (int r = tid; r < n; r += kBisThreads) c += sg[r] > tau;
  if (c) atomicAdd(&s_nnz, c);
  __syncthreads();
  if (tid == 0) {
    nnz[mat] = s1 > 0.0 ? s_nnz : 0;
    if (lns1) lns1[mat] = s1 > 0.0 ? log(s1) : -INFINITY;
  }
}

// ---------------------------------------------------------------------------
// Vector c of a set (at(v, i): entry i of vector v) made orthogonal to the
// orthonormal vectors p0 .. c-1 and normalized, by every thread of the block
// (32 or 64): the dots one thread per earlier vector (four partial sums), the
// update and the norm spread over the entries; classical Gram-Schmidt applied
// twice, which keeps orthogonality to rounding.  Called by all threads alike.
template <class At>
__device__ void block_cgs2(At at, int p0, int c, int len, double* s_dot, double* s_red) {
  const int t = threadIdx.x, T = blockDim.x;
  for (int pass = 0; pass < 2; ++pass) {
    if (t >= p0 && t < c) {
      double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
      int i = 0;
      for (; i + 4 <= len; i += 4) {
        d0 = fma(at(t, i), at(c, i), d0);
        d1 = fma(at(t, i + 1), at(c, i + 1), d1);
        d2 = fma(at(t, i + 2), at(c, i + 2), d2);
        d3 = fma(at(t, i + 3), at(c, i + 3), d3);
      }
      for (; i < len; ++i) d0 = fma(at(t, i), at(c, i), d0);
      s_dot[t] = (d0 + d1) + (d2 + d3);
    }
    __syncthreads();
    for (int i = t; i < len; i += T) {
      double x = at(c, i);
      for (int p = p0; p < c; ++p) x = fma(-s_dot[p], at(p, i), x);
      at(c, i) = x;
    }
    __syncthreads();
  }
  double s2 = 0.0;
  for (int i = t; i < len; i += T) s2 = fma(at(c, i), at(c, i), s2);
  for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  if ((t & 31) == 0) s_red[t >> 5] = s2;
  __syncthreads();
  double tot = 0.0;
  for (int w = 0; w < (T >> 5); ++w) tot += s_red[w];
  const double inv = tot > 0.0 ? 1.0 / sqrt(tot) : 0.0;
  for (int i = t; i < len; i += T) at(c, i) *= inv;
  __syncthreads();
}

// ---------------------------------------------------------------------------
// 3. Inverse iteration, one CTA of one or two warps per matrix (persistent
//    over matrices), thread a for the a-th kept index.  Scratch per CTA slot,
//    interleaved by thread with stride ls (16, 32 or 64): DG, DU, DU2 (the LU
//    factors of T - s I with partial pivoting, in the layout of LAPACK's dgtsv)
//    and X (the iterate), each 2n entries.  The factorization streams the
//    current row in registers and applies L^-1 P^T to the right-hand side as
//    it goes; the scale of the previous iterate is folded into the next
//    right-hand side.
__global__ void __launch_bounds__(64) k_bd_invit(BdVecArgs a, int ls) {
  __shared__ double s_dot[kKeptMax];
  __shared__ double s_red[2];
  const int lane = threadIdx.x;             // kept index of this thread
  const int wl = threadIdx.x & 31;          // lane within its warp
  double* scr = a.scratch + (size_t)blockIdx.x * 4 * (2 * a.n) * ls;   // a slot for the largest n
#define DG(i) scr[((size_t)0 * m + (i)) * ls + lane]
#define DU(i) scr[((size_t)1 * m + (i)) * ls + lane]
#define DU2(i) scr[((size_t)2 * m + (i)) * ls + lane]
#define XB(i) scr[((size_t)3 * m + (i)) * ls + lane]
#define XL(l, i) scr[((size_t)3 * m + (i)) * ls + (l)]
  for (int s = blockIdx.x; s < a.S; s += gridDim.x) {
    int n = a.n, nk;
    const int* kept;
    const double* sg;
    const double* bd;
    double* vout;
    if (a.items) {                   // ragged: this matrix's size and buffers
      const SvdItem& t = a.items[s];
      n = t.n; nk = t.nk[0]; kept = t.kept; sg = t.sig; bd = t.bd; vout = t.vrows;
    } else {
      nk = a.nk[s];
      kept = a.kept + (size_t)s * a.kstride;
      sg = a.sig + (size_t)s * a.n_pad;
      bd = a.bd + (size_t)s * 3 * n;
      vout = a.vrows + (size_t)s * a.kstride * n;
    }
    const int m = 2 * n;
    // |T| (max |o_k|): T and s are scaled by 1/|T|, the pivot floor is eps
    // (each warp reduces over all of T)
    double tn = 0.0;
    for (int i = wl; i < n; i += 32) tn = fmax(tn, fmax(fabs(bd[i]), fabs(bd[n + i])));
    for (int o = 16; o > 0; o >>= 1) tn = fmax(tn, __shfl_xor_sync(0xffffffffu, tn, o));
    const double its = tn > 0.0 ? 1.0 / tn : 0.0;
    const bool on = lane < nk && lane < ls;
    const double sgm = on ? sg[kept[lane]] * its : 0.0;
    // is this lane's value chained (within 1e-3 |T|) to a neighbouring kept value?
    bool clustered = false;
    if (on) {
      if (lane > 0 && sg[kept[lane - 1]] - sg[kept[lane]] <= 1e-3 * tn) clustered = true;
      if (lane + 1 < nk && sg[kept[lane]] - sg[kept[lane + 1]] <= 1e-3 * tn) clustered = true;
    }
#define OFFD(i) (((i) & 1) ? bd[n + ((i) >> 1)] : bd[(i) >> 1]) * its
    if (on) {                                        // start vector, different per lane
      for (int i = 0; i < m; ++i) XB(i) = 1.0 + 0.25 * (double)((i * (2 * lane + 3)) % 17) * (1.0 / 17.0);
    }
    double rs = 1.0;                                 // scale owed by the stored iterate
    for (int iter = 0; iter < kInvitIters; ++iter) {
      if (on) {
        // factor T - s I = P L U, applying L^-1 P^T to the right-hand side as it
        // goes; the loads of each block of kCh steps are issued together, so the
        // serial chain waits on memory once per block instead of once per step
        double dg = -sgm, du = OFFD(0), xi = XB(0) * rs;
        for (int base = 0; base < m - 1; base += kCh) {
          double xnb[kCh], odb[kCh + 1];
#pragma unroll
          for (int c = 0; c < kCh; ++c) {
            const int i = base + c;
            xnb[c] = (i + 1 < m) ? XB(i + 1) : 0.0;
            odb[c] = (i < m - 1) ? OFFD(i) : 0.0;
          }
          odb[kCh] = (base + kCh < m - 1) ? OFFD(base + kCh) : 0.0;
#pragma unroll
          for (int c = 0; c < kCh; ++c) {
            const int i = base + c;
            if (i >= m - 1) break;
            const double dli = odb[c];                 // sub-diagonal = off-diagonal
            const double dun = (i + 1 < m - 1) ? odb[c + 1] : 0.0;
            const double xn = xnb[c] * rs;
            if (fabs(dg) >= fabs(dli)) {
              const double g = (dg == 0.0) ? kEps : dg;
              const double f = dli / g;
              DG(i) = g; DU(i) = du; DU2(i) = 0.0; XB(i) = xi;
              dg = -sgm - f * du;
              du = dun;
              xi = xn - f * xi;
            } else {
              const double f = dg / dli;
              DG(i) = dli; DU(i) = -sgm; DU2(i) = dun; XB(i) = xn;
              dg = du + f * sgm;
              du = -f * dun;
              xi = xi - f * xn;
            }
          }
        }
        const double glast = (dg == 0.0) ? kEps : dg;
        DG(m - 1) = glast;
        // back substitution U x = y, carrying x_{i+1}, x_{i+2}, in blocks of kCh
        double x1 = xi / glast;
        XB(m - 1) = x1;
        double s2 = x1 * x1;
        double x2 = 0.0;
        for (int top = m - 2; top >= 0; top -= kCh) {
          double yb[kCh], ub[kCh], u2b[kCh], gb[kCh];
#pragma unroll
          for (int c = 0; c < kCh; ++c) {
            const int i = top - c;
            yb[c] = i >= 0 ? XB(i) : 0.0;
            ub[c] = i >= 0 ? DU(i) : 0.0;
            u2b[c] = i >= 0 ? DU2(i) : 0.0;
            gb[c] = i >= 0 ? DG(i) : 1.0;
          }
#pragma unroll
          for (int c = 0; c < kCh; ++c) {
            const int i = top - c;
            if (i < 0) break;
            double x = (yb[c] - ub[c] * x1 - u2b[c] * x2) / gb[c];
            if (exp_field(x) > 1023 + 600) {         // growth through tiny pivots: rescale x[i..]
              for (int q = i + 1; q < m; ++q) XB(q) *= 0x1.0p-600;
              x *= 0x1.0p-600; x1 *= 0x1.0p-600; x2 *= 0x1.0p-600; s2 *= 0x1.0p-1200;
            }
            XB(i) = x;
            s2 = fma(x, x, s2);
            x2 = x1;
            x1 = x;
          }
        }
        rs = s2 > 0.0 ? 1.0 / sqrt(s2) : 0.0;
        if (clustered) {                             // unit iterates for the Gram-Schmidt below
          for (int i = 0; i < m; ++i) XB(i) *= rs;
          rs = 1.0;
        }
      }
      // orthonormalize against the earlier kept vectors of the same cluster
      // (a chain of kept values less than 1e-3 |T| apart), in index order
      __syncthreads();
      for (int c = 1; c < nk && c < ls; ++c) {
        if (sg[kept[c - 1]] - sg[kept[c]] > 1e-3 * tn) continue;
        int p0 = c - 1;
        while (p0 > 0 && sg[kept[p0 - 1]] - sg[kept[p0]] <= 1e-3 * tn) --p0;
        block_cgs2([&](int v, int i) -> double& { return XL(v, i); }, p0, c, m, s_dot, s_red);
      }
    }
#undef OFFD
    if (on) {                                        // v_B = even entries, normalized
      double s2 = 0.0;
      for (int i = 0; i < n; ++i) s2 = fma(XB(2 * i), XB(2 * i), s2);
      const double inv = s2 > 0.0 ? 1.0 / sqrt(s2) : 0.0;
      for (int i = 0; i < n; ++i) vout[(size_t)lane * n + i] = XB(2 * i) * inv;
    }
    // orthogonal z's of a cluster need not have orthogonal halves (values near
    // the noise level mix +s and -s): orthonormalize the v's of each cluster too
    __syncthreads();
    for (int c = 1; c < nk && c < ls; ++c) {
      if (sg[kept[c - 1]] - sg[kept[c]] > 1e-3 * tn) continue;
      int p0 = c - 1;
      while (p0 > 0 && sg[kept[p0 - 1]] - sg[kept[p0]] <= 1e-3 * tn) --p0;
      block_cgs2([&](int v, int i) -> double& { return vout[(size_t)v * n + i]; }, p0, c, n, s_dot, s_red);
    }
    __syncthreads();
  }
#undef DG
#undef DU
#undef DU2
#undef XB
#undef XL
}

// ---------------------------------------------------------------------------
// 4. v = H_0 H_1 ... H_{n-3} v_B, one CTA of gs / 4 warps per (matrix, group
//    of gs kept vectors; gs = 16, or 8 for sides whose 16 vectors would not fit
//    in shared memory), the group in shared memory, 4 vectors per warp (warps
//    independent: no block barrier inside the reflector loop).  The four dot
//    products of a warp are reduced together (reduce4).
__global__ void __launch_bounds__(128) k_bd_backtr(BdVecArgs a, int gs) {
  extern __shared__ double V[];                      // [gs][n]
  const int s = blockIdx.x, g0 = blockIdx.y * gs;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int n = a.n, nk_all;
  double* vrow;
  const double* R;
  const double* tauR;
  const int* kept;
  const double* sg;
  if (a.items) {                     // ragged: this matrix's size and buffers
    const SvdItem& t = a.items[s];
    n = t.n; nk_all = t.nk[0]; vrow = t.vrows + (size_t)g0 * n; R = t.W; tauR = t.bd + 2 * n;
    kept = t.kept + g0; sg = t.sig;
  } else {
    nk_all = a.nk[s];
    vrow = a.vrows + ((size_t)s * a.kstride + g0) * n;
    R = a.R + (size_t)s * n * n;
    tauR = a.bd + (size_t)s * 3 * n + 2 * n;
    kept = a.kept + (size_t)s * a.kstride + g0;
    sg = a.sig + (size_t)s * a.n_pad;
  }
  const int nk = min(nk_all - g0, gs);               // vectors of this group
  if (nk <= 0) return;
  for (int e = threadIdx.x; e < nk * n; e += blockDim.x) V[e] = vrow[e];
  __syncthreads();
  const int a0 = warp * 4;
  if (a0 < nk) {
    double* V0 = V + (size_t)a0 * n;
    const int na = min(4, nk - a0);
    for (int k = n - 3; k >= 0; --k) {
      const double taur = tauR[k];
      if (taur == 0.0) continue;
      const double* u = R + (size_t)k * n;           // u[k+1] = 1, u[k+2..n-1] stored
      double p0 = 0.0, p1 = 0.0, p2 = 0.0, p3 = 0.0;
      for (int j = k + 1 + lane; j < n; j += 32) {
        const double uj = (j == k + 1) ? 1.0 : u[j];
        p0 = fma(uj, V0[j], p0);
        if (na > 1) p1 = fma(uj, V0[n + j], p1);
        if (na > 2) p2 = fma(uj, V0[2 * n + j], p2);
        if (na > 3) p3 = fma(uj, V0[3 * n + j], p3);
      }
      const double t = reduce4(p0, p1, p2, p3, lane);
      const double w0 = taur * __shfl_sync(0xffffffffu, t, 0);
      const double w1 = taur * __shfl_sync(0xffffffffu, t, 8);
      const double w2 = taur * __shfl_sync(0xffffffffu, t, 16);
      const double w3 = taur * __shfl_sync(0xffffffffu, t, 24);
      for (int j = k + 1 + lane; j < n; j += 32) {
        const double uj = (j == k + 1) ? 1.0 : u[j];
        V0[j] = fma(-w0, uj, V0[j]);
        if (na > 1) V0[n + j] = fma(-w1, uj, V0[n + j]);
        if (na > 2) V0[2 * n + j] = fma(-w2, uj, V0[2 * n + j]);
        if (na > 3) V0[3 * n + j] = fma(-w3, uj, V0[3 * n + j]);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nk * n; e += blockDim.x) vrow[e] = a.unit_rows ? V[e] : sg[kept[e / n]] * V[e];
}

// ---------------------------------------------------------------------------
// Largest side of the bidiagonalization route: the wide form's per-step
// vectors (3 + 8 per-warp rows of n doubles) fill shared memory at 2304.
constexpr int kBdMaxN = 2304;
constexpr size_t kBdSmemCap = 227 * 1024;

// Dynamic shared memory of a launch over matrices of side n (the working copy
// in shared memory when it fits, else the per-step vectors with enough
// memory requested that one CTA runs per SM and the matrices stay in L2).
size_t bidiag_smem_bytes(int n) {
  const size_t rows = (size_t)n * n * sizeof(double);
  const size_t aux = ((size_t)(3 + kBdThreads / 32) * n + 32) * sizeof(double);
  return rows + aux <= 200 * 1024 ? rows + aux : std::max<size_t>(aux, 120 * 1024);
}

template <int NQ>
static cudaError_t launch_bidiag_nq(const BidiagArgs& a, cudaStream_t st) {
  const int n = a.n;
  const int use_smem = NQ > 0 && (size_t)n * n * sizeof(double) +
                                         ((size_t)(3 + kBdThreads / 32) * n + 32) * sizeof(double) <=
                                     200 * 1024;
  const size_t smem = bidiag_smem_bytes(n);
  static std::atomic<uint64_t> attr{0};
  cudaError_t e = raise_smem_limit(k_bidiag<NQ>, kBdSmemCap, attr);
  if (e != cudaSuccess) return e;
  k_bidiag<NQ><<<a.S, kBdThreads, smem, st>>>(a, use_smem);
  return cudaGetLastError();
}

template <int NQ>
static cudaError_t launch_bidiag_items_nq(const SvdItem* items, int S, size_t smem, cudaStream_t st) {
  static std::atomic<uint64_t> attr{0};
  cudaError_t e = raise_smem_limit(k_bidiag<NQ>, kBdSmemCap, attr);
  if (e != cudaSuccess) return e;
  BidiagArgs a{};
  a.S = S; a.items = items;
  k_bidiag<NQ><<<S, kBdThreads, smem, st>>>(a, 0);
  return cudaGetLastError();
}

cudaError_t launch_bidiag_items(const SvdItem* items, int S, int n_max, size_t smem, cudaStream_t st) {
  if (S <= 0) return cudaSuccess;
  if (smem > kBdSmemCap || smem < bidiag_smem_bytes(n_max)) return cudaErrorInvalidValue;
  if (n_max <= 64) return launch_bidiag_items_nq<2>(items, S, smem, st);
  if (n_max <= 128) return launch_bidiag_items_nq<4>(items, S, smem, st);
  if (n_max <= 256) return launch_bidiag_items_nq<8>(items, S, smem, st);
  if (n_max <= 512) return launch_bidiag_items_nq<16>(items, S, smem, st);
  if (n_max <= 768) return launch_bidiag_items_nq<24>(items, S, smem, st);
  if (n_max <= 1024) return launch_bidiag_items_nq<32>(items, S, smem, st);
  if (n_max <= kBdMaxN) return launch_bidiag_items_nq<0>(items, S, smem, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_bidiag(const BidiagArgs& a, cudaStream_t st) {
  if (a.S <= 0) return cudaSuccess;
  if (a.n <= 64) return launch_bidiag_nq<2>(a, st);
  if (a.n <= 128) return launch_bidiag_nq<4>(a, st);
  if (a.n <= 256) return launch_bidiag_nq<8>(a, st);
  if (a.n <= 512) return launch_bidiag_nq<16>(a, st);
  if (a.n <= 768) return launch_bidiag_nq<24>(a, st);
  if (a.n <= 1024) return launch_bidiag_nq<32>(a, st);
  if (a.n <= kBdMaxN) return launch_bidiag_nq<0>(a, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_bd_bisect(const double* bd, int n, int n_pad, int S, double* sig, int* perm, int* nnz,
                             double* lns1, double zero_rel, cudaStream_t st) {
  if (S <= 0) return cudaSuccess;
  const size_t smem = (size_t)2 * n * (sizeof(double) + sizeof(float)) + kBisThreads * sizeof(int);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  static std::atomic<uint64_t> attr{0};
  cudaError_t e = raise_smem_limit(k_bd_bisect, 200 * 1024, attr);
  if (e != cudaSuccess) return e;
  k_bd_bisect<<<S, kBisThreads, smem, st>>>(bd, n, n_pad, sig, perm, nnz, lns1, zero_rel, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_bd_bisect_items(const SvdItem* items, int S, int n_max, cudaStream_t st) {
  if (S <= 0) return cudaSuccess;
  const size_t smem = (size_t)2 * n_max * (sizeof(double) + sizeof(float)) + kBisThreads * sizeof(int);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  static std::atomic<uint64_t> attr{0};
  cudaError_t e = raise_smem_limit(k_bd_bisect, 200 * 1024, attr);
  if (e != cudaSuccess) return e;
  k_bd_bisect<<<S, kBisThreads, smem, st>>>(nullptr, 0, 0, nullptr, nullptr, nullptr, nullptr, 0.0, items);
  return cudaGetLastError();
}

// Thread stride of the inverse iteration's scratch: 16, 32 or 64 kept vectors.
static int invit_stride(int kmax) { return kmax <= 16 ? 16 : (kmax <= 32 ? 32 : 64); }

// CTA slots of the inverse iteration: up to eight per SM (each runs one
// thread-serial chain per kept vector, so the SMs need several to hide the
// FP64 latency), and no more than 512 MB of scratch (4 x 2n x ls doubles each).
static int invit_slots(int n, int S, int kmax) {
  const size_t per = (size_t)4 * 2 * n * invit_stride(kmax) * sizeof(double);
  const int by_mem = (int)std::max<size_t>(152, ((size_t)512 << 20) / per);
  return std::max(1, std::min(S, std::min(152 * 8, by_mem)));
}

size_t bd_vectors_scratch_doubles(int n, int S, int kmax) {
  return (size_t)invit_slots(n, S, kmax) * 4 * 2 * n * invit_stride(kmax);
}

// Ragged: a.items holds a.S matrices, a.n the largest side, a.kmax the largest
// kept count, a.scratch bd_vectors_scratch_doubles(a.n, a.S, a.kmax) doubles.
cudaError_t launch_bd_vectors(const BdVecArgs& a, cudaStream_t st) {
  if (a.S <= 0) return cudaSuccess;
  if (a.kmax > kKeptMax || (!a.items && a.kstride < a.kmax)) return cudaErrorInvalidValue;
  constexpr size_t kSmemCap = 227 * 1024;
  const int gs = (size_t)16 * a.n * sizeof(double) <= kSmemCap ? 16 : 8;
  const size_t smem = (size_t)gs * a.n * sizeof(double);
  if (smem > kSmemCap) return cudaErrorInvalidValue;
  const int ls = invit_stride(a.kmax);
  k_bd_invit<<<invit_slots(a.n, a.S, a.kmax), ls > 32 ? 64 : 32, 0, st>>>(a, ls);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || a.skip_backtr) return e;
  static std::atomic<uint64_t> attr{0};
  e = raise_smem_limit(k_bd_backtr, kSmemCap, attr);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)a.S, (unsigned)((std::max(1, a.kmax) + gs - 1) / gs));
  k_bd_backtr<<<grid, 32 * (gs / 4), smem, st>>>(a, gs);
  return cudaGetLastError();
}

}  // namespace mctrg
