// Monte Carlo HOTRG: the stochastic truncation of Sec. II applied to the
// higher-order TRG of Xie et al. (2012), one of the other SVD-based
// coarse-graining schemes to which Secs. III and V say the method extends.
//
// A step merges pairs of rows of the lattice: the tensors at (x, 2j) (top, T1)
// and (x, 2j+1) (bottom, T2) contract over their vertical bond into
//   M(x, j)[(l1 l2), u1, (r1 r2), d2] = sum_k T1[l1,u1,r1,k] T2[l2,k,r2,d2].
// Each merged horizontal bond -- the one to the right of M(x, j) -- gets its
// own random projector P~ = sum_{i in e} u_i u_i^T / r_i: (u_i, lambda_i) are
// the eigenpairs of the Gram matrix of M(x, j)'s right unfolding,
//   G[(r1 r2), (r1' r2')] = sum_{k,k'} A1[(r1,k),(r1',k')] A2[(k,r2),(k',r2')],
//   A1 = sum_{l1,u1} T1[l1,u1,r1,k] T1[l1,u1,r1',k'],
//   A2 = sum_{l2,d2} T2[l2,k,r2,d2] T2[l2,k',r2',d2]
// (formed without M), split by the bidiagonalization route of the TRG path
// (G is symmetric positive semidefinite: its singular values are lambda_i,
// its right singular vectors u_i; eigenvalues at or below n 2^-52 lambda_1
// are zeros).  A chi-subset e of the nonzero ones is drawn with
// p(e) ~ prod lambda_i by the TRG sampler fed s_i = sqrt(lambda_i) (Sec. II,
// p(e) ~ prod s_i^2), r_i are its inclusion rates, and only the kept
// eigenvectors are computed.  E[P~] is the projector onto the range of G,
// outside which M vanishes, so every trajectory samples Z without bias.
// With U~ = [u_i / sqrt(r_i)] (n x kc, zero-padded) the new tensor is
//   T'(x, j)[a, u1, b, d2] = sum U~_left[(l1 l2), a] M[(l1 l2), u1, (r1 r2), d2] U~_right[(r1 r2), b]
// / sqrt(lambda_1 of its right bond), evaluated as
//   P[a, u1, r1, l2, k] = sum_l1 U~_left[(l1 l2), a] T1[l1, u1, r1, k]
//   Q[a, u1, r1, r2, d2] = sum_{l2,k} P[a, u1, r1, l2, k] T2[l2, k, r2, d2]
//   T'[a, u1, b, d2]     = sum_{r1,r2} Q[a, u1, r1, r2, d2] U~_right[(r1 r2), b]
// and written reflected across the diagonal (position (x, j) -> (j, x), legs
// (l,u,r,d) -> (u,l,d,r)), so that the next step again merges rows.  After
// 2 log2 L steps one tensor remains: Z~ = sum_{l,u} T[l,u,l,u] (Sec. IV).
// Uniforms: Philox counter (t >> 1, bond, step, trajectory), bond = j Lx + x.
//
// Tensors of one lattice are stored [trajectory][y Lx + x][Dh][Dv][Dh][Dv]
// (legs l, u, r, d).  Every contraction kernel computes one output element
// per thread; consecutive threads take consecutive output columns, so the
// operand that varies with the column is read coalesced and the other is a
// warp broadcast.  The work is FP64-issue bound.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/mctrg.h"
#include "common.cuh"
#include "kernels.h"
#include "kernels_bd.h"
#include "mctrg_internal.h"

using namespace mctrg;

namespace {

int hfail(cudaError_t e) {
  set_last_cuda_error(e);
  return MCTRG_ECUDA;
}

#define HCK(call)                                 \
  do {                                            \
    cudaError_t e__ = (call);                     \
    if (e__ != cudaSuccess) return hfail(e__);    \
  } while (0)

struct Buf {     // a device allocation owned by one call
  void* p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t b) {
    if (b <= bytes) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(b, 8));
    if (e == cudaSuccess) bytes = b;
    return e;
  }
  ~Buf() { if (p) cudaFree(p); }
  template <class T> T* as() const { return (T*)p; }
};

// Geometry and shapes of one row-merging step.
struct Step {
  int Lx, Ly, Dh, Dv;    // lattice and leg dimensions before the step
  int n, n_pad, kc, Lj;  // bond dimension n = Dh^2, kept kc, merged rows Lj = Ly / 2
  int64_t N;             // bonds (= new tensors) per trajectory: Lx Lj
  int64_t tin, tout;     // doubles per tensor before and after
};

std::vector<Step> schedule(int L, int D0, int chi) {
  std::vector<Step> s;
  int Lx = L, Ly = L, Dh = D0, Dv = D0;
  while (Lx * Ly > 1) {
    Step a{};
    a.Lx = Lx; a.Ly = Ly; a.Dh = Dh; a.Dv = Dv;
    a.n = Dh * Dh; a.n_pad = a.n + (a.n & 1); a.kc = std::min(chi, a.n); a.Lj = Ly / 2;
    a.N = (int64_t)Lx * a.Lj;
    a.tin = (int64_t)Dh * Dv * Dh * Dv;
    a.tout = (int64_t)Dv * a.kc * Dv * a.kc;
    s.push_back(a);
    const int nLx = a.Lj, nLy = Lx;
    Lx = nLx; Ly = nLy;
    const int nDh = Dv, nDv = a.kc;
    Dh = nDh; Dv = nDv;
  }
  return s;
}

// ---- stage A: the bond Gram matrices ------------------------------------------
// A1[(r1,k),(r1',k')] and A2[(k,r2),(k',r2')] of the merged pair right of
// bond item (b, t = j Lx + x); q = Dh Dv outputs per row.
__global__ void k_hotrg_pair_gram(const double* __restrict__ tens, int64_t item0, int64_t n_items, int64_t N,
                                  int Lx, int Dh, int Dv, int64_t ntens, double* __restrict__ A1,
                                  double* __restrict__ A2) {
  const int q = Dh * Dv;
  const int64_t per = (int64_t)q * q;
  const int64_t total = n_items * 2 * per;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t it = e / (2 * per);
    const int64_t rem = e - it * 2 * per;
    const int which = (int)(rem / per);
    const int64_t o = rem - which * per;
    const int p = (int)(o / q), pp = (int)(o - (int64_t)p * q);
    const int64_t item = item0 + it, b = item / N, t = item - b * N;
    const int j = (int)(t / Lx), x = (int)(t - (int64_t)j * Lx);
    const int64_t tq = (int64_t)q * q;
    double acc = 0.0;
    if (which == 0) {
      // T1 as a q x q matrix, rows (l1, u1), columns (r1, k): A1 = T1^T T1
      const double* T1 = tens + (b * ntens + (int64_t)(2 * j) * Lx + x) * tq;
      for (int c = 0; c < q; ++c) acc = fma(T1[(int64_t)c * q + p], T1[(int64_t)c * q + pp], acc);
      A1[it * per + o] = acc;
    } else {
      // T2[l2][(k r2)][d2]: rows (k, r2) with k = p / Dh, r2 = p % Dh
      const double* T2 = tens + (b * ntens + (int64_t)(2 * j + 1) * Lx + x) * tq;
      for (int l2 = 0; l2 < Dh; ++l2)
        for (int d2 = 0; d2 < Dv; ++d2)
          acc = fma(T2[((int64_t)l2 * q + p) * Dv + d2], T2[((int64_t)l2 * q + pp) * Dv + d2], acc);
      A2[it * per + o] = acc;
    }
  }
}

// G[(r1 r2),(r1' r2')] = sum_{k,k'} A1[(r1,k),(r1',k')] A2[(k,r2),(k',r2')].
__global__ void k_hotrg_gram(const double* __restrict__ A1, const double* __restrict__ A2, int64_t n_items, int Dh,
                             int Dv, double* __restrict__ G) {
  const int q = Dh * Dv, n = Dh * Dh;
  const int64_t per = (int64_t)n * n, aper = (int64_t)q * q;
  const int64_t total = n_items * per;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t it = e / per;
    const int64_t o = e - it * per;
    const int row = (int)(o / n), col = (int)(o - (int64_t)row * n);
    const int r1 = row / Dh, r2 = row - r1 * Dh, s1 = col / Dh, s2 = col - s1 * Dh;
    const double* a1 = A1 + it * aper;
    const double* a2 = A2 + it * aper;
    double acc = 0.0;
    for (int k = 0; k < Dv; ++k)
      for (int kk = 0; kk < Dv; ++kk)
        acc = fma(a1[(int64_t)(r1 * Dv + k) * q + s1 * Dv + kk], a2[(int64_t)(k * Dh + r2) * q + kk * Dh + s2], acc);
    G[it * per + o] = acc;
  }
}

// s_i = sqrt(lambda_i) for the sampler (lambda, the singular values of G, stay
// for the vectors); ln s_1 = ln(lambda_1) / 2 per bond.
__global__ void k_hotrg_roots(const double* sig, double* sroot, double* lns, int64_t n_items, int n_pad) {
  const int64_t total = n_items * n_pad;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    sroot[e] = sqrt(fmax(sig[e], 0.0));
    if (e % n_pad == 0) lns[e / n_pad] *= 0.5;
  }
}

// U~ rows: the unit eigenvector of kept value a times 1 / sqrt(r_a), where
// r_a = (s_a / s_1) / sigt_a; rows past the kept count are zero.
__global__ void k_hotrg_scale(double* U, const double* sroot, const double* sigt, const int* kept, const int* nk,
                              int64_t n_items, int n, int n_pad, int kc, int ks) {
  const int64_t total = n_items * kc * (int64_t)n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t it = e / ((int64_t)kc * n);
    const int64_t rem = e - it * kc * n;
    const int a = (int)(rem / n), i = (int)(rem - (int64_t)a * n);
    double* row = U + (it * ks + a) * n;
    if (a >= nk[it]) { row[i] = 0.0; continue; }
    const double s1 = sroot[it * n_pad];
    const double sa = sroot[it * n_pad + kept[it * ks + a]];
    row[i] *= sqrt(sigt[it * ks + a] * s1 / sa);
  }
}

// ---- stage B: the new tensors ----------------------------------------------------
// P[it][a][u1][r1][l2][k] = sum_l1 U~_left[a][(l1 l2)] T1[l1][u1][r1][k].
__global__ void k_hotrg_p(const double* __restrict__ tens, const double* __restrict__ U, int64_t item0,
                          int64_t n_items, int64_t N, int Lx, int Dh, int Dv, int kc, int ks, int64_t ntens,
                          double* __restrict__ P) {
  const int n = Dh * Dh;
  const int64_t per = (int64_t)kc * Dv * Dh * Dh * Dv;
  const int64_t total = n_items * per;
  const int64_t tq = (int64_t)Dh * Dv * Dh * Dv;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t it = e / per;
    int64_t o = e - it * per;
    const int k = (int)(o % Dv); o /= Dv;
    const int l2 = (int)(o % Dh); o /= Dh;
    const int r1 = (int)(o % Dh); o /= Dh;
    const int u1 = (int)(o % Dv); o /= Dv;
    const int a = (int)o;
    const int64_t item = item0 + it, b = item / N, t = item - b * N;
    const int j = (int)(t / Lx), x = (int)(t - (int64_t)j * Lx);
    const int xl = x == 0 ? Lx - 1 : x - 1;
    const double* UL = U + ((b * N + (int64_t)j * Lx + xl) * ks + a) * n;
    const double* T1 = tens + (b * ntens + (int64_t)(2 * j) * Lx + x) * tq;
    double acc = 0.0;
    for (int l1 = 0; l1 < Dh; ++l1)
      acc = fma(UL[l1 * Dh + l2], T1[(((int64_t)l1 * Dv + u1) * Dh + r1) * Dv + k], acc);
    P[e] = acc;
  }
}

// Q[it][a][u1][r1][r2][d2] = sum_{l2,k} P[it][a][u1][r1][l2][k] T2[l2][k][r2][d2].
__global__ void k_hotrg_q(const double* __restrict__ tens, const double* __restrict__ P, int64_t item0,
                          int64_t n_items, int64_t N, int Lx, int Dh, int Dv, int kc, int64_t ntens,
                          double* __restrict__ Q) {
  const int q = Dh * Dv;
  const int64_t per = (int64_t)kc * Dv * Dh * Dh * Dv;
  const int64_t total = n_items * per;
  const int64_t tq = (int64_t)q * q;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t it = e / per;
    const int64_t o = e - it * per;
    const int c = (int)(o % q);               // (r2, d2)
    const int64_t arow = o / q;                // (a, u1, r1)
    const int64_t item = item0 + it, b = item / N, t = item - b * N;
    const int j = (int)(t / Lx), x = (int)(t - (int64_t)j * Lx);
    const double* T2 = tens + (b * ntens + (int64_t)(2 * j + 1) * Lx + x) * tq;
    const double* p = P + it * per + arow * q;   // [(l2, k)]
    double acc = 0.0;
    for (int m = 0; m < q; ++m) acc = fma(p[m], T2[(int64_t)m * q + c], acc);
    Q[e] = acc;
  }
}

// T'[a][u1][b][d2] = sum_{(r1 r2)} Q[a][u1][(r1 r2)][d2] U~_right[b][(r1 r2)] / s_1,
// written reflected: out[(x Lj + j)][u1][a][d2][b].
__global__ void k_hotrg_t(const double* __restrict__ Q, const double* __restrict__ U, const double* __restrict__ lns,
                          int64_t item0, int64_t n_items, int64_t N, int Lx, int Lj, int Dh, int Dv, int kc, int ks,
                          double* __restrict__ out) {
  const int n = Dh * Dh;
  const int64_t per = (int64_t)kc * Dv * kc * Dv;
  const int64_t qper = (int64_t)kc * Dv * n * Dv;
  const int64_t total = n_items * per;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t it = e / per;
    int64_t o = e - it * per;
    const int bb = (int)(o % kc); o /= kc;     // output order [u1][a][d2][b]
    const int d2 = (int)(o % Dv); o /= Dv;
    const int a = (int)(o % kc); o /= kc;
    const int u1 = (int)o;
    const int64_t item = item0 + it, b = item / N, t = item - b * N;
    const int j = (int)(t / Lx), x = (int)(t - (int64_t)j * Lx);
    const double ln1 = lns[item];
    double v = 0.0;
    if (ln1 != -INFINITY) {
      const double* UR = U + (item * ks + bb) * n;
      const double* qr = Q + it * qper + ((int64_t)a * Dv + u1) * n * Dv + d2;
      double acc = 0.0;
      for (int r = 0; r < n; ++r) acc = fma(qr[(int64_t)r * Dv], UR[r], acc);
      v = acc * exp(-ln1);
    }
    const int64_t tout = per;
    out[(b * N + (int64_t)x * Lj + j) * tout + (((int64_t)u1 * kc + a) * Dv + d2) * kc + bb] = v;
  }
}

// Z~ = sum_{l,u} T[l,u,l,u] of each trajectory's last tensor, with its log scale.
__global__ void k_hotrg_trace(const double* tens, int Dh, int Dv, int64_t B, const double* lnacc, double* lnabs,
                              int8_t* sign) {
  const int64_t b = blockIdx.x;
  if (b >= B) return;
  const int64_t tq = (int64_t)Dh * Dv * Dh * Dv;
  const double* T = tens + b * tq;
  double s = 0.0;
  for (int e = threadIdx.x; e < Dh * Dv; e += 32) {
    const int l = e / Dv, u = e - l * Dv;
    s += T[(((int64_t)l * Dv + u) * Dh + l) * Dv + u];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) {
    const double la = lnacc[b];
    if (s == 0.0 || !(la > -INFINITY)) { lnabs[b] = -INFINITY; sign[b] = 0; }
    else { lnabs[b] = la + log(fabs(s)); sign[b] = s > 0 ? 1 : -1; }
  }
}

// Broadcast the site tensor to every site of every trajectory of a chunk.
__global__ void k_hotrg_fill(const double* T0, int64_t tq, int64_t count, double* out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count * tq; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = T0[e % tq];
}

unsigned grid_for(int64_t total) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 64));
}

}  // namespace

extern "C" int mctrg_hotrg_run(const mctrg_options* opt, double beta, double h, const double* T0h, int D, int L,
                               int chi, int64_t n, uint64_t seed, uint64_t first_traj, double* lnabs_out,
                               int8_t* sign_out, uint8_t* flags_out, mctrg_estimate* est) {
  if (!opt || !est || n < 1 || first_traj + (uint64_t)n > (1ull << 32)) return MCTRG_EINVAL;
  if (L < 2 || (L & (L - 1)) || L > 4096 || chi < 2 || chi > 32) return MCTRG_EINVAL;
  if (T0h ? (D < 2 || D > 8) : (!(beta >= 0.0) || !std::isfinite(beta) || !std::isfinite(h))) return MCTRG_EINVAL;
  const int D0 = T0h ? D : 2;
  int ndev = 0;
  HCK(cudaGetDeviceCount(&ndev));
  if (opt->device < 0 || opt->device >= ndev) return MCTRG_EINVAL;
  HCK(cudaSetDevice(opt->device));
  cudaStream_t st = (cudaStream_t)opt->cuda_stream;
  const std::vector<Step> steps = schedule(L, D0, chi);
  const int ks = kept_stride(chi);

  // memory plan: per trajectory, two lattice buffers and the per-bond
  // projector factors; per item, the Gram stage and the contraction scratch
  size_t per_traj = 0, per_item = 0, shared = 0;
  for (const Step& a : steps) {
    const size_t lat = (size_t)a.Lx * a.Ly * a.tin + (size_t)a.N * a.tout;
    const size_t bonds = (size_t)a.N * (ks * (size_t)a.n + 1) * sizeof(double) + a.N * sizeof(uint32_t);
    per_traj = std::max(per_traj, lat * sizeof(double) + bonds);
    const size_t q2 = (size_t)a.Dh * a.Dv * a.Dh * a.Dv;
    const size_t gram = (2 * q2 + (size_t)a.n * a.n + (size_t)a.n_pad * a.n + 3 * (size_t)a.n + 2 * (size_t)a.n_pad +
                         ks) * sizeof(double) + ((size_t)a.n_pad + 2 + ks) * sizeof(int);
    const size_t contr = 2 * (size_t)a.kc * a.Dv * a.Dh * a.Dh * a.Dv * sizeof(double);
    per_item = std::max(per_item, std::max(gram, contr));
    shared = std::max(shared, (sample_scratch_doubles(a.n, chi, sample_grid(a.n, chi)) +
                               bd_vectors_scratch_doubles(a.n, 1 << 14, a.kc)) * sizeof(double));
  }
  per_traj += 2 * sizeof(double) + 2 * sizeof(uint32_t) + 16;
  size_t fr = 0, tot = 0;
  HCK(cudaMemGetInfo(&fr, &tot));
  size_t budget = opt->hbm_budget_bytes ? opt->hbm_budget_bytes : (size_t)(0.7 * (double)fr);
  budget = std::min(budget, (size_t)(0.9 * (double)fr));
  if (budget <= shared) return MCTRG_ENOMEM;
  const size_t work = std::max<size_t>((budget - shared) / 4, per_item);
  int64_t B = (int64_t)((budget - shared - work) / std::max<size_t>(per_traj, 1));
  if (opt->max_chunk > 0) B = std::min<int64_t>(B, opt->max_chunk);
  B = std::min<int64_t>(B, n);
  if (B < 1) return MCTRG_ENOMEM;
  int64_t maxN = 1;
  for (const Step& a : steps) maxN = std::max<int64_t>(maxN, a.N);
  const int64_t S = std::max<int64_t>(1, std::min<int64_t>({(int64_t)(work / per_item), B * maxN, 1 << 14}));

  Buf T0d, lat0, lat1, Uall, lnb, ifl, A1, A2, G, W, bd, sig, sroot, perm, nnz, kept, sigt, nk, smp, vscr, P, Q;
  Buf lnacc, tflags, o_lnabs, o_sign, o_flags, stats;
  size_t lat_max = 0, bonds_max = 0, a_max = 0, g_max = 0, w_max = 0, np_max = 0, pq_max = 0, n_max = 0;
  for (const Step& a : steps) {
    lat_max = std::max(lat_max, (size_t)std::max<int64_t>((int64_t)a.Lx * a.Ly * a.tin, a.N * a.tout));
    bonds_max = std::max(bonds_max, (size_t)a.N);
    a_max = std::max(a_max, (size_t)a.Dh * a.Dv * a.Dh * a.Dv);
    g_max = std::max(g_max, (size_t)a.n * a.n);
    w_max = std::max(w_max, (size_t)a.n_pad * a.n);
    np_max = std::max(np_max, (size_t)a.n_pad);
    n_max = std::max(n_max, (size_t)a.n);
    pq_max = std::max(pq_max, (size_t)a.kc * a.Dv * a.Dh * a.Dh * a.Dv);
  }
  const size_t Bs = (size_t)B, Ss = (size_t)S;
  HCK(T0d.ensure(sizeof(double) * (size_t)D0 * D0 * D0 * D0));
  HCK(lat0.ensure(sizeof(double) * Bs * lat_max));
  HCK(lat1.ensure(sizeof(double) * Bs * lat_max));
  HCK(Uall.ensure(sizeof(double) * Bs * bonds_max * ks * n_max));
  HCK(lnb.ensure(sizeof(double) * Bs * bonds_max));
  HCK(ifl.ensure(sizeof(uint32_t) * Bs * bonds_max));
  HCK(A1.ensure(sizeof(double) * Ss * a_max));
  HCK(A2.ensure(sizeof(double) * Ss * a_max));
  HCK(G.ensure(sizeof(double) * Ss * g_max));
  HCK(W.ensure(sizeof(double) * Ss * w_max));
  HCK(bd.ensure(sizeof(double) * Ss * 3 * n_max));
  HCK(sig.ensure(sizeof(double) * Ss * np_max));
  HCK(sroot.ensure(sizeof(double) * Ss * np_max));
  HCK(perm.ensure(sizeof(int) * Ss * np_max));
  HCK(nnz.ensure(sizeof(int) * Ss));
  HCK(kept.ensure(sizeof(int) * Ss * ks));
  HCK(sigt.ensure(sizeof(double) * Ss * ks));
  HCK(nk.ensure(sizeof(int) * Ss));
  HCK(P.ensure(sizeof(double) * Ss * pq_max));
  HCK(Q.ensure(sizeof(double) * Ss * pq_max));
  size_t smp_max = 0, vscr_max = 0;
  for (const Step& a : steps) {
    smp_max = std::max(smp_max, sample_scratch_doubles(a.n, chi, sample_grid(a.n, chi)));
    vscr_max = std::max(vscr_max, bd_vectors_scratch_doubles(a.n, (int)S, a.kc));
  }
  HCK(smp.ensure(sizeof(double) * smp_max));
  HCK(vscr.ensure(sizeof(double) * vscr_max));
  HCK(lnacc.ensure(sizeof(double) * Bs));
  HCK(tflags.ensure(sizeof(uint32_t) * Bs));
  HCK(o_lnabs.ensure(sizeof(double) * (size_t)n));
  HCK(o_sign.ensure((size_t)n));
  HCK(o_flags.ensure((size_t)n));
  HCK(stats.ensure(sizeof(double) * 8));
  if (T0h) HCK(cudaMemcpyAsync(T0d.p, T0h, sizeof(double) * (size_t)D0 * D0 * D0 * D0, cudaMemcpyHostToDevice, st));
  else HCK(launch_site_tensor(beta, h, T0d.as<double>(), st));

  for (int64_t c0 = 0; c0 < n; c0 += B) {
    const int64_t Bc = std::min<int64_t>(B, n - c0);
    double* cur = lat0.as<double>();
    double* nxt = lat1.as<double>();
    const int64_t tq0 = (int64_t)D0 * D0 * D0 * D0;
    k_hotrg_fill<<<grid_for(Bc * L * L * tq0), 256, 0, st>>>(T0d.as<double>(), tq0, Bc * (int64_t)L * L, cur);
    HCK(cudaGetLastError());
    HCK(cudaMemsetAsync(lnacc.p, 0, sizeof(double) * Bc, st));
    HCK(cudaMemsetAsync(tflags.p, 0, sizeof(uint32_t) * Bc, st));
    for (size_t si = 0; si < steps.size(); ++si) {
      const Step& a = steps[si];
      const int64_t items = Bc * a.N, ntens = (int64_t)a.Lx * a.Ly;
      HCK(cudaMemsetAsync(ifl.p, 0, sizeof(uint32_t) * items, st));
      // stage A: every bond's projector factor
      for (int64_t i0 = 0; i0 < items; i0 += S) {
        const int64_t Si = std::min<int64_t>(S, items - i0);
        const int64_t q2 = (int64_t)a.Dh * a.Dv * a.Dh * a.Dv;
        k_hotrg_pair_gram<<<grid_for(Si * 2 * q2), 256, 0, st>>>(cur, i0, Si, a.N, a.Lx, a.Dh, a.Dv, ntens,
                                                                 A1.as<double>(), A2.as<double>());
        HCK(cudaGetLastError());
        k_hotrg_gram<<<grid_for(Si * (int64_t)a.n * a.n), 256, 0, st>>>(A1.as<double>(), A2.as<double>(), Si, a.Dh,
                                                                         a.Dv, G.as<double>());
        HCK(cudaGetLastError());
        BidiagArgs ba{};
        ba.M = G.as<double>(); ba.W = W.as<double>(); ba.bd = bd.as<double>(); ba.n = a.n; ba.S = (int)Si;
        HCK(launch_bidiag(ba, st));
        double* lnb_i = lnb.as<double>() + i0;
        HCK(launch_bd_bisect(bd.as<double>(), a.n, a.n_pad, (int)Si, sig.as<double>(), perm.as<int>(), nnz.as<int>(),
                             lnb_i, 0.0, st));
        k_hotrg_roots<<<grid_for(Si * a.n_pad), 256, 0, st>>>(sig.as<double>(), sroot.as<double>(), lnb_i, Si,
                                                              a.n_pad);
        HCK(cudaGetLastError());
        SampleArgs sa{};
        sa.M = G.as<double>(); sa.W = nullptr; sa.sig = sroot.as<double>(); sa.perm = perm.as<int>();
        sa.nnz = nnz.as<int>(); sa.Urows = nullptr; sa.n = a.n; sa.n_pad = a.n_pad; sa.chi = chi; sa.kc = a.kc;
        sa.stochastic = 1; sa.shared_svd = 0; sa.item0 = i0; sa.n_items = Si; sa.N = a.N; sa.L = L;
        sa.level = (int)si; sa.seed = seed; sa.traj0 = first_traj + (uint64_t)c0; sa.H = nullptr; sa.h_item0 = 0;
        sa.iflags = ifl.as<uint32_t>(); sa.scratch = smp.as<double>(); sa.mode = 1; sa.kept = kept.as<int>();
        sa.sigt = sigt.as<double>(); sa.nk = nk.as<int>(); sa.vrows = nullptr; sa.kstride = ks;
        HCK(launch_sample_split(sa, st, sample_grid(a.n, chi)));
        BdVecArgs va{};
        double* Ui = Uall.as<double>() + (size_t)i0 * ks * a.n;
        va.bd = bd.as<double>(); va.R = W.as<double>(); va.sig = sig.as<double>(); va.kept = kept.as<int>();
        va.nk = nk.as<int>(); va.vrows = Ui; va.scratch = vscr.as<double>(); va.n = a.n; va.n_pad = a.n_pad;
        va.S = (int)Si; va.unit_rows = 1; va.kmax = a.kc; va.kstride = ks;
        HCK(launch_bd_vectors(va, st));
        k_hotrg_scale<<<grid_for(Si * a.kc * (int64_t)a.n), 256, 0, st>>>(Ui, sroot.as<double>(), sigt.as<double>(),
                                                                           kept.as<int>(), nk.as<int>(), Si, a.n,
                                                                           a.n_pad, a.kc, ks);
        HCK(cudaGetLastError());
      }
      // stage B: the new tensors, written reflected into the other buffer
      for (int64_t i0 = 0; i0 < items; i0 += S) {
        const int64_t Si = std::min<int64_t>(S, items - i0);
        const int64_t pq = (int64_t)a.kc * a.Dv * a.Dh * a.Dh * a.Dv;
        k_hotrg_p<<<grid_for(Si * pq), 256, 0, st>>>(cur, Uall.as<double>(), i0, Si, a.N, a.Lx, a.Dh, a.Dv, a.kc, ks,
                                                    ntens, P.as<double>());
        HCK(cudaGetLastError());
        k_hotrg_q<<<grid_for(Si * pq), 256, 0, st>>>(cur, P.as<double>(), i0, Si, a.N, a.Lx, a.Dh, a.Dv, a.kc, ntens,
                                                    Q.as<double>());
        HCK(cudaGetLastError());
        k_hotrg_t<<<grid_for(Si * a.tout), 256, 0, st>>>(Q.as<double>(), Uall.as<double>(), lnb.as<double>(), i0,
                                                         Si, a.N, a.Lx, a.Lj, a.Dh, a.Dv, a.kc, ks, nxt);
        HCK(cudaGetLastError());
      }
      HCK(launch_traj_accum(lnb.as<double>(), ifl.as<uint32_t>(), a.N, Bc, lnacc.as<double>(),
                            tflags.as<uint32_t>(), st));
      std::swap(cur, nxt);
    }
    const Step& last = steps.back();
    k_hotrg_trace<<<(unsigned)Bc, 32, 0, st>>>(cur, last.Dv, last.kc, Bc, lnacc.as<double>(),
                                              o_lnabs.as<double>() + c0, o_sign.as<int8_t>() + c0);
    HCK(cudaGetLastError());
    HCK(launch_flags_to_u8(tflags.as<uint32_t>(), o_flags.as<uint8_t>() + c0, Bc, 0u, st));
  }
  HCK(launch_estimate(o_lnabs.as<double>(), o_sign.as<int8_t>(), o_flags.as<uint8_t>(), n, stats.as<double>(), st));
  double hs[6];
  HCK(cudaMemcpyAsync(hs, stats.p, sizeof(hs), cudaMemcpyDeviceToHost, st));
  if (lnabs_out) HCK(cudaMemcpyAsync(lnabs_out, o_lnabs.p, sizeof(double) * n, cudaMemcpyDefault, st));
  if (sign_out) HCK(cudaMemcpyAsync(sign_out, o_sign.p, (size_t)n, cudaMemcpyDefault, st));
  if (flags_out) HCK(cudaMemcpyAsync(flags_out, o_flags.p, (size_t)n, cudaMemcpyDefault, st));
  HCK(cudaStreamSynchronize(st));
  std::memset(est, 0, sizeof(*est));
  est->n = n;
  est->ln_scale = hs[0];
  est->sum_x = hs[1];
  est->m2_x = hs[2];
  est->n_negative = (int64_t)hs[3];
  est->n_flagged = (int64_t)hs[4];
  finish_estimate(est);
  return est->status;
}
