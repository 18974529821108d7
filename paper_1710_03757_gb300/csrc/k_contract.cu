// K5: plaquette contraction (Sec. III, Levin-Nave TRG step), its FP64 GEMM
// with the next level's matricization fused into the epilogue; K6: final
// trace; K7 helpers: per-trajectory accumulation and the estimator sums.
//
// New tensor at the plaquette whose top-left corner p is an A tensor:
//   T'[al,be,de,ga] = sum_{i,j,k,m} F3(p)[al,i,j] F4(p+a1)[be,k,i]
//                                   F2(p+a2)[j,m,ga] F1(p+a1+a2)[m,k,de]
// with legs (l,u,r,d) = (al,be,de,ga).  It is evaluated as
//   X [(al,be)][(j,k)] = sum_i F3[al,i,j] F4[be,k,i]
//   Yt[(de,ga)][(j,k)] = sum_m F2[j,m,ga] F1[m,k,de]
//   T' = X Yt^T  (a GEMM with M = N = D^2, K = d^2).
// Parent halves come from the level-k layout of the sampler: left [d^2][D]
// (F1 of an A tensor, F2 of a B tensor), right [D][d^2] (F3 / F4).
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace mctrg {

// ---- X and Yt ----------------------------------------------------------------
// grid (n_items, D, 2): z = 0 builds row block al of X, z = 1 row block de of Yt.
__global__ void k_form_xy(XYArgs a) {
  extern __shared__ double sm[];
  const int d = a.d, D = a.D, d2 = d * d;
  double* s_a = sm;          // [d2]
  double* s_b = sm + d2;     // [d2]
  const int64_t it = blockIdx.x;
  const int64_t item = a.c0 + it;
  const int64_t b = item / a.Nnew, c = item % a.Nnew;
  int64_t par[4];
  if (a.fixed_parents) { par[0] = 0; par[1] = 1; par[2] = 1; par[3] = 0; }
  else tensor_parents(a.L, a.level_old, c, par);
  const int64_t stride = (int64_t)2 * d2 * D;
  auto half_left = [&](int q) { return a.H + (b * a.Nold + par[q] - a.h_item0) * stride; };
  auto half_right = [&](int q) { return half_left(q) + (int64_t)d2 * D; };
  const int sel = blockIdx.y;
  if (blockIdx.z == 0) {
    // X[(al,be)][(j,k)] = sum_i F3[al][i*d+j] * F4[be][k*d+i]
    const double* F3 = half_right(0) + (int64_t)sel * d2;
    const double* F4 = half_right(1);
    for (int e = threadIdx.x; e < d2; e += blockDim.x) s_a[e] = F3[e];
    double* Xo = a.X + ((int64_t)it * D * D + (int64_t)sel * D) * d2;
    for (int be = 0; be < D; ++be) {
      __syncthreads();
      for (int e = threadIdx.x; e < d2; e += blockDim.x) s_b[e] = F4[(int64_t)be * d2 + e];
      __syncthreads();
      for (int e = threadIdx.x; e < d2; e += blockDim.x) {
        const int j = e / d, k = e - j * d;
        double acc = 0.0;
        for (int i = 0; i < d; ++i) acc = fma(s_a[i * d + j], s_b[k * d + i], acc);
        Xo[(int64_t)be * d2 + e] = acc;
      }
    }
  } else {
    // Yt[(de,ga)][(j,k)] = sum_m F2[(j*d+m)][ga] * F1[(m*d+k)][de]
    const double* F1 = half_left(3);
    const double* F2 = half_left(2);
    for (int e = threadIdx.x; e < d2; e += blockDim.x) s_a[e] = F1[(int64_t)e * D + sel];
    double* Yo = a.Yt + ((int64_t)it * D * D + (int64_t)sel * D) * d2;
    for (int ga = 0; ga < D; ++ga) {
      __syncthreads();
      for (int e = threadIdx.x; e < d2; e += blockDim.x) s_b[e] = F2[(int64_t)e * D + ga];
      __syncthreads();
      for (int e = threadIdx.x; e < d2; e += blockDim.x) {
        const int j = e / d, k = e - j * d;
        double acc = 0.0;
        for (int m = 0; m < d; ++m) acc = fma(s_b[j * d + m], s_a[m * d + k], acc);
        Yo[(int64_t)ga * d2 + e] = acc;
      }
    }
  }
}

cudaError_t launch_form_xy(const XYArgs& a, cudaStream_t st) {
  if (a.n_items <= 0) return cudaSuccess;
  dim3 grid((unsigned)a.n_items, a.D, 2);
  const int d2 = a.d * a.d;
  const int threads = d2 >= 256 ? 256 : (d2 >= 64 ? 64 : 32);
  k_form_xy<<<grid, threads, 2 * d2 * sizeof(double), st>>>(a);
  return cudaGetLastError();
}

// ---- FP64 GEMM with the matricization epilogue -------------------------------
// 64 x 64 output tile per CTA, K step 16, 256 threads with 4 x 4 outputs each.
namespace {
constexpr int TM = 64, TK = 16;
}

__global__ void __launch_bounds__(256) k_gemm_f64(GemmArgs a) {
  __shared__ double sX[TK][TM + 1];
  __shared__ double sY[TK][TM + 1];
  const int D = a.D, n = D * D, K = a.K;
  const int tiles_c = (n + TM - 1) / TM;
  const int tr = blockIdx.y / tiles_c, tcol = blockIdx.y % tiles_c;
  const int64_t it = blockIdx.x;
  const double* X = a.X + (int64_t)it * n * K;
  const double* Y = a.Yt + (int64_t)it * n * K;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int r0 = tr * TM, c0 = tcol * TM;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int e = threadIdx.x; e < TM * TK; e += 256) {
      const int rr = e / TK, kk = e - rr * TK;
      const int gr = r0 + rr, gc = c0 + rr, gk = k0 + kk;
      sX[kk][rr] = (gr < n && gk < K) ? X[(int64_t)gr * K + gk] : 0.0;
      sY[kk][rr] = (gc < n && gk < K) ? Y[(int64_t)gc * K + gk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double xr[4], yc[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { xr[q] = sX[kk][ty + 16 * q]; yc[q] = sY[kk][tx + 16 * q]; }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(xr[p], yc[q], acc[p][q]);
    }
    __syncthreads();
  }
  const int64_t item = a.c0 + it;
  int par = a.fixed_parity;
  if (par < 0) par = tensor_parity(a.L, a.level_new, item % a.Nnew);
  double* Mo = a.M + (int64_t)it * n * n;
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int r = r0 + ty + 16 * p;
    if (r >= n) continue;
    const int al = r / D, be = r - al * D;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int cc = c0 + tx + 16 * q;
      if (cc >= n) continue;
      const int de = cc / D, ga = cc - de * D;
      int64_t off;
      if (par == 0) off = (int64_t)r * n + cc;                                   // (l,u),(r,d)
      else off = (int64_t)(be * D + de) * n + (ga * D + al);                      // (u,r),(d,l)
      Mo[off] = acc[p][q];
    }
  }
}

cudaError_t launch_gemm_f64(const GemmArgs& a, cudaStream_t st) {
  if (a.n_items <= 0) return cudaSuccess;
  const int n = a.D * a.D;
  const int tiles = (n + TM - 1) / TM;
  dim3 grid((unsigned)a.n_items, tiles * tiles);
  k_gemm_f64<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

// ---- K6: final trace ------------------------------------------------------------
__global__ void k_trace(const double* X, const double* Yt, int64_t K2, double lnacc0,
                        const double* lnacc, double* lnabs, int8_t* sign) {
  __shared__ double red[256];
  const int64_t it = blockIdx.x;
  const double* x = X + it * K2;
  const double* y = Yt + it * K2;
  double acc = 0.0;
  for (int64_t e = threadIdx.x; e < K2; e += blockDim.x) acc = fma(x[e], y[e], acc);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double tr = red[0];
    const double base = lnacc0 + (lnacc ? lnacc[it] : 0.0);
    if (tr == 0.0 || !(base > -INFINITY)) { lnabs[it] = -INFINITY; sign[it] = 0; }
    else { lnabs[it] = base + log(fabs(tr)); sign[it] = tr > 0 ? 1 : -1; }
  }
}

cudaError_t launch_trace(const double* X, const double* Yt, int64_t K2, int64_t n_items,
                         double lnacc0, const double* lnacc, double* lnabs, int8_t* sign,
                         cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  k_trace<<<(unsigned)n_items, 256, 0, st>>>(X, Yt, K2, lnacc0, lnacc, lnabs, sign);
  return cudaGetLastError();
}

// ---- site tensor and matricizations -------------------------------------------
// T[l,u,r,d] = sum_s e^{beta h s} W[s,l] W[s,u] W[s,r] W[s,d],
// W[s,0] = sqrt(cosh beta), W[s,1] = s sqrt(sinh beta); s = +1 (index 0), -1.
__global__ void k_site_tensor(double beta, double h, double* T) {
  const int e = threadIdx.x;
  if (e >= 16) return;
  const int l = (e >> 3) & 1, u = (e >> 2) & 1, r = (e >> 1) & 1, d = e & 1;
  const double c = sqrt(cosh(beta)), s = sqrt(sinh(beta));
  double v = 0.0;
  for (int k = 0; k < 2; ++k) {
    const double spin = k == 0 ? 1.0 : -1.0;
    const double w1 = spin * s;
    const double wl = l ? w1 : c, wu = u ? w1 : c, wr = r ? w1 : c, wd = d ? w1 : c;
    v += exp(beta * h * spin) * (wl * wu * wr * wd);
  }
  T[e] = v;
}

cudaError_t launch_site_tensor(double beta, double h, double* T, cudaStream_t st) {
  k_site_tensor<<<1, 32, 0, st>>>(beta, h, T);
  return cudaGetLastError();
}

// The site tensor with the site's spin inserted (an impurity: the network's
// trace becomes sum_sigma sigma_i e^{-beta H}, a partial trace of Sec. III):
// T_imp[l,u,r,d] = sum_s s e^{beta h s} W[s,l] W[s,u] W[s,r] W[s,d].
__global__ void k_impurity_tensor(double beta, double h, double* T) {
  const int e = threadIdx.x;
  if (e >= 16) return;
  const int l = (e >> 3) & 1, u = (e >> 2) & 1, r = (e >> 1) & 1, d = e & 1;
  const double c = sqrt(cosh(beta)), s = sqrt(sinh(beta));
  double v = 0.0;
  for (int k = 0; k < 2; ++k) {
    const double spin = k == 0 ? 1.0 : -1.0;
    const double w1 = spin * s;
    const double wl = l ? w1 : c, wu = u ? w1 : c, wr = r ? w1 : c, wd = d ? w1 : c;
    v += spin * exp(beta * h * spin) * (wl * wu * wr * wd);
  }
  T[e] = v;
}

cudaError_t launch_impurity_tensor(double beta, double h, double* T, cudaStream_t st) {
  k_impurity_tensor<<<1, 32, 0, st>>>(beta, h, T);
  return cudaGetLastError();
}

// Level-0 matrices of a network that is not translation invariant: item
// item0 + it = b N0 + t takes site t's tensor (the impurity at sites imp0 /
// imp1, the plain one elsewhere; D = 2), matricized by t's sublattice.
__global__ void k_level0_matrices(const double* T0, const double* Timp, int imp0, int imp1, int L,
                                  int64_t item0, int64_t n_items, int64_t N0, double* M) {
  const int64_t tot = n_items * 16;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t it = e >> 4;
    const int q = (int)(e & 15);
    const int64_t t = (item0 + it) % N0;
    const double* T = (t == imp0 || t == imp1) ? Timp : T0;
    const int l = (q >> 3) & 1, u = (q >> 2) & 1, r = (q >> 1) & 1, d = q & 1;
    const int par = tensor_parity(L, 0, t);
    double* Mo = M + it * 16;
    if (par == 0) Mo[(l * 2 + u) * 4 + (r * 2 + d)] = T[q];      // A: (l,u),(r,d)
    else Mo[(u * 2 + r) * 4 + (d * 2 + l)] = T[q];               // B: (u,r),(d,l)
  }
}

cudaError_t launch_level0_matrices(const double* T0, const double* Timp, int imp0, int imp1, int L, int64_t item0,
                                   int64_t n_items, int64_t N0, double* M, cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  const int64_t tot = n_items * 16;
  const int64_t blocks = std::min<int64_t>((tot + 255) / 256, 4096);
  k_level0_matrices<<<(unsigned)blocks, 256, 0, st>>>(T0, Timp, imp0, imp1, L, item0, n_items, N0, M);
  return cudaGetLastError();
}

// Spins-on-bonds network (Sec. IV, Fig. 1): the legs carry the spins, and the
// four spins around a tensor form a plaquette whose four bonds it holds:
// T[l,u,r,d] = exp(beta (s_l s_u + s_u s_r + s_r s_d + s_d s_l)
//                  + beta h (s_l + s_u + s_r + s_d) / 2)   (a spin is on two legs).
__global__ void k_bond_tensor(double beta, double h, double* T) {
  const int e = threadIdx.x;
  if (e >= 16) return;
  const double sl = (e >> 3) & 1 ? -1.0 : 1.0, su = (e >> 2) & 1 ? -1.0 : 1.0;
  const double sr = (e >> 1) & 1 ? -1.0 : 1.0, sd = e & 1 ? -1.0 : 1.0;
  T[e] = exp(beta * (sl * su + su * sr + sr * sd + sd * sl) + 0.5 * beta * h * (sl + su + sr + sd));
}

cudaError_t launch_bond_tensor(double beta, double h, double* T, cudaStream_t st) {
  k_bond_tensor<<<1, 32, 0, st>>>(beta, h, T);
  return cudaGetLastError();
}

__global__ void k_matricize2(const double* T, int D, double* out) {
  const int n = D * D;
  const int64_t tot = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(e / ((int64_t)D * D * D)), u = (int)((e / (D * D)) % D),
              r = (int)((e / D) % D), d = (int)(e % D);
    const double v = T[e];
    out[(int64_t)(l * D + u) * n + (r * D + d)] = v;              // A: (l,u),(r,d)
    out[tot + (int64_t)(u * D + r) * n + (d * D + l)] = v;        // B: (u,r),(d,l)
  }
}

cudaError_t launch_matricize2(const double* T, int D, double* out, cudaStream_t st) {
  const int64_t tot = (int64_t)D * D * D * D;
  const int blocks = (int)((tot + 255) / 256);
  k_matricize2<<<blocks < 1024 ? blocks : 1024, 256, 0, st>>>(T, D, out);
  return cudaGetLastError();
}

// ---- per-trajectory accumulation -------------------------------------------------
__global__ void k_traj_accum(const double* ilns1, const uint32_t* iflags, int64_t N, int64_t B,
                             double* lnacc, uint32_t* tflags) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= B) return;
  double s = 0.0;
  uint32_t f = 0;
  for (int64_t t = 0; t < N; ++t) {
    if (ilns1) s += ilns1[b * N + t];
    if (iflags) f |= iflags[b * N + t];
  }
  if (ilns1) lnacc[b] += s;
  tflags[b] |= f;
}

cudaError_t launch_traj_accum(const double* ilns1, const uint32_t* iflags, int64_t N, int64_t B,
                              double* lnacc, uint32_t* tflags, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  k_traj_accum<<<(unsigned)((B + 127) / 128), 128, 0, st>>>(ilns1, iflags, N, B, lnacc, tflags);
  return cudaGetLastError();
}

// ---- estimator sums (one block, fixed reduction order) ------------------------
// stats = {m, sum x, sum (x - mean)^2, n_negative, n_flagged, n_zero} with
// x_i = sign_i exp(lnabs_i - m), m = max lnabs over nonzero samples.
__device__ double block_sum_1024(double v, double* red) {
  const int tid = threadIdx.x;
  __syncthreads();
  red[tid] = v;
  __syncthreads();
  for (int s = 512; s > 0; s >>= 1) {
    if (tid < s) red[tid] += red[tid + s];
    __syncthreads();
  }
  return red[0];
}

__global__ void __launch_bounds__(1024) k_estimate(const double* lnabs, const int8_t* sign,
                                                   const uint8_t* flags, int64_t n, double* stats) {
  __shared__ double red[1024];
  const int tid = threadIdx.x;
  double m = -INFINITY;
  for (int64_t i = tid; i < n; i += 1024)
    if (sign[i] != 0) m = fmax(m, lnabs[i]);
  red[tid] = m;
  __syncthreads();
  for (int s = 512; s > 0; s >>= 1) {
    if (tid < s) red[tid] = fmax(red[tid], red[tid + s]);
    __syncthreads();
  }
  const double mm = red[0] > -INFINITY ? red[0] : 0.0;
  double s1 = 0.0, cneg = 0.0, cflag = 0.0, czero = 0.0;
  for (int64_t i = tid; i < n; i += 1024) {
    const int sg = sign[i];
    if (sg != 0) { const double x = exp(lnabs[i] - mm); s1 += sg > 0 ? x : -x; }
    cneg += sg < 0;
    czero += sg == 0;
    cflag += (flags && flags[i]) ? 1.0 : 0.0;
  }
  const double S1 = block_sum_1024(s1, red);
  const double mean = S1 / (double)n;
  double d2 = 0.0;
  for (int64_t i = tid; i < n; i += 1024) {
    const int sg = sign[i];
    double x = 0.0;
    if (sg != 0) { x = exp(lnabs[i] - mm); if (sg < 0) x = -x; }
    d2 = fma(x - mean, x - mean, d2);
  }
  const double M2 = block_sum_1024(d2, red);
  const double NN = block_sum_1024(cneg, red);
  const double NF = block_sum_1024(cflag, red);
  const double NZ = block_sum_1024(czero, red);
  if (tid == 0) {
    stats[0] = mm; stats[1] = S1; stats[2] = M2; stats[3] = NN; stats[4] = NF; stats[5] = NZ;
  }
}

cudaError_t launch_estimate(const double* lnabs, const int8_t* sign, const uint8_t* flags,
                            int64_t n, double* stats, cudaStream_t st) {
  k_estimate<<<1, 1024, 0, st>>>(lnabs, sign, flags, n, stats);
  return cudaGetLastError();
}

__global__ void k_flags_to_u8(const uint32_t* f, uint8_t* out, int64_t n, uint32_t extra) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (uint8_t)((f ? f[i] : 0u) | extra);
}

cudaError_t launch_flags_to_u8(const uint32_t* f, uint8_t* out, int64_t n, uint32_t extra, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_flags_to_u8<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(f, out, n, extra);
  return cudaGetLastError();
}

}  // namespace mctrg
