// K3 + K4: stochastic truncation of each tensor's SVD and the split into the
// two three-leg halves (Sec. II and Sec. III).
//
// For a spectrum s_1 >= ... >= s_n' > 0 (values at or below n 2^-52 s_1 are
// zeros) and a sample size chi < n', a chi-subset e is drawn with
// p(e) ~ prod_{j in e} s_j^2 (Sec. II, Eqs. w and p) and each kept value is
// divided by its inclusion rate r_i = sum_{e contains i} p(e) (Sec. II, Eq. r),
// so that the average of the truncated spectra is the full one (Eq. Ssum).
// The paper defers the O(chi n') sampler to Ferris (2015); this is a
// fixed-size product-weight design built on normalized elementary symmetric
// polynomials of w_i = (s_i / s_1)^2:
//   E[i][j] = e_j(w_1..w_i) / (w_1 ... w_j)
//           = E[i-1][j] + (w_i / w_j) E[i-1][j-1],   values in [1, C(i,j)];
//   G[i][b] = e_b(w_{i+1}..w_n') / (w_{i+1} ... w_{i+b})
//           = G[i+1][b] (w_{i+b+1} / w_{i+1}) + G[i+1][b-1].
// Draw: the largest kept index first; with j picks left among {1..b} the
// running sum over i of P(largest = i) is E[i][j], so the pick is the
// smallest i in [j, b] with E[i][j] > u E[b][j] (u from Philox step t).
// Rates: r_i = sum_a E[i-1][a] G[i][chi-1-a] R(i,a) / E[n'][chi] with
// R(i,a) = prod_{t < chi-a} w_{i+t} / w_{a+1+t}  (each factor <= 1).
//
// One CTA of 128 threads per item (trajectory, tensor): warp 0 builds E while
// warp 1 builds G (the row recurrences run along i with one lane per column,
// and a second column per lane past 32, neighbouring columns exchanged by warp
// shuffles); warp 0 then draws with a ballot search per step and computes the
// chi rates; all warps write halves
//   left[row][a]  = sqrt(s~_a) u_a[row],   right[a][col] = sqrt(s~_a) v_a[col],
// s~ = (s / s_1) / r, u = M v / s computed here for the kept indices only.
#include <cmath>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "kernels_bd.h"

namespace mctrg {

namespace {
constexpr int kThreads = 128;

// Sum of KV (16 or 8) per-lane values over the warp, all at once: halving
// exchanges (each lane keeps the half of its values its partner does not) and
// last butterflies; on return lane l holds the total of value l / (32 / KV).
template <int KV>
__device__ __forceinline__ double warp_sum_k(double (&v)[KV], int lane) {
#pragma unroll
  for (int h = KV / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {
    const bool hi = lane & o;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const double keep = hi ? v[j + h] : v[j];
      const double send = hi ? v[j] : v[j + h];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  double t = v[0];
#pragma unroll
  for (int o = 16 / KV; o >= 1; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
}  // namespace

size_t sample_scratch_doubles(int n, int chi, int grid) {
  return (size_t)grid * (size_t)(n + 1) * (size_t)(2 * chi + 1);
}

int sample_grid(int n, int chi) {
  const size_t per = sample_scratch_doubles(n, chi, 1) * sizeof(double);
  const size_t cap = ((size_t)256 << 20) / per;
  return (int)std::max<size_t>(152, std::min<size_t>(1024, cap));
}

// KV kept vectors are staged per pass of the M v product (16, or 8 for sides
// whose 16 staged rows would not fit in shared memory).
template <int KV>
__global__ void __launch_bounds__(kThreads) k_sample_split(SampleArgs a) {
  extern __shared__ double dsm[];
  const int n = a.n, np = a.n_pad, chi = a.chi, kc = a.kc, ks = a.kstride;
  double* w = dsm;                                  // [np] normalized weights
  double* wn = w + np;                              // [np] s_i / s_1
  double* vbuf = wn + np;                           // [KV][n]
  unsigned char* inset = (unsigned char*)(vbuf + (size_t)KV * n);   // [np]
  __shared__ int s_kept[kKeptMax];
  __shared__ double s_sigt[kKeptMax];
  __shared__ int s_nk;
  __shared__ uint32_t s_flags;

  double* tabE = a.scratch + (size_t)blockIdx.x * (size_t)(n + 1) * (2 * chi + 1);
  double* tabG = tabE + (size_t)(n + 1) * (chi + 1);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int64_t it = blockIdx.x; it < a.n_items; it += gridDim.x) {
    const int64_t item = a.item0 + it;
    const int64_t b = item / a.N, t = item % a.N;
    int64_t slot = it;
    if (a.shared_svd) slot = tensor_parity(a.L, a.level, t);
    const double* sg = a.sig + (size_t)slot * np;
    const double s1 = sg[0];
    const int nz = (s1 > 0.0) ? a.nnz[slot] : 0;
    const bool sample = a.stochastic && nz > chi;

    if (a.mode == 2) {                         // choices made earlier (split form)
      if (tid < ks) { s_kept[tid] = a.kept[it * ks + tid]; s_sigt[tid] = a.sigt[it * ks + tid]; }
      if (tid == 0) { s_nk = a.nk[it]; s_flags = 0; }
      __syncthreads();
    } else {
    for (int i = tid; i < np; i += kThreads) {
      const double v = (i < nz) ? sg[i] / s1 : 0.0;
      wn[i] = v;
      w[i] = v * v;
      inset[i] = 0;
    }
    // without sampling the kc largest nonzero values are kept (all of them on
    // an exact level, nz <= kc; the top kc on a deterministic one, Eq. approxSVD)
    if (tid == 0) { s_flags = 0; s_nk = sample ? chi : min(nz, kc); }
    __syncthreads();

    if (sample) {
      const bool two = chi > 32;             // a second column per lane (32 + lane + 1)
      if (warp == 0) {                       // forward table E, lane l <-> columns l+1, l+33
        const int j = lane + 1, j2 = lane + 33;
        const double wj = (j <= chi) ? w[j - 1] : 1.0;
        const double wj2 = (j2 <= chi) ? w[j2 - 1] : 1.0;
        double Ej = 0.0, Ej2 = 0.0;
        if (lane == 0) tabE[0] = 1.0;
        if (j <= chi) tabE[j] = 0.0;
        if (j2 <= chi) tabE[j2] = 0.0;
        for (int i = 1; i <= nz; ++i) {
          const double wi = w[i - 1];
          double prev = __shfl_up_sync(0xffffffffu, Ej, 1);
          if (lane == 0) prev = 1.0;
          double* row = tabE + (size_t)i * (chi + 1);
          if (two) {                         // column 33's left neighbour is lane 31's column 32
            const double top = __shfl_sync(0xffffffffu, Ej, 31);
            double prev2 = __shfl_up_sync(0xffffffffu, Ej2, 1);
            if (lane == 0) prev2 = top;
            Ej2 = Ej2 + (wi / wj2) * prev2;
            if (j2 <= chi) row[j2] = Ej2;
          }
          Ej = Ej + (wi / wj) * prev;
          if (lane == 0) row[0] = 1.0;
          if (j <= chi) row[j] = Ej;
        }
      } else if (warp == 1) {                // backward table G, lane l <-> columns l+1, l+33
        const int bb = lane + 1, bb2 = lane + 33;
        double Gb = 0.0, Gb2 = 0.0;
        if (lane == 0) tabG[(size_t)nz * chi] = 1.0;
        if (bb < chi) tabG[(size_t)nz * chi + bb] = 0.0;
        if (bb2 < chi) tabG[(size_t)nz * chi + bb2] = 0.0;
        for (int i = nz - 1; i >= 0; --i) {
          double prev = __shfl_up_sync(0xffffffffu, Gb, 1);
          if (lane == 0) prev = 1.0;
          double* row = tabG + (size_t)i * chi;
          if (two) {
            const double top = __shfl_sync(0xffffffffu, Gb, 31);
            double prev2 = __shfl_up_sync(0xffffffffu, Gb2, 1);
            if (lane == 0) prev2 = top;
            if (bb2 <= nz - i) {
              const double first = (i + bb2 + 1 <= nz) ? Gb2 * (w[i + bb2] / w[i]) : 0.0;
              Gb2 = first + prev2;
            } else {
              Gb2 = 0.0;
            }
            if (bb2 < chi) row[bb2] = Gb2;
          }
          if (bb <= nz - i) {
            const double first = (i + bb + 1 <= nz) ? Gb * (w[i + bb] / w[i]) : 0.0;
            Gb = first + prev;
          } else {
            Gb = 0.0;
          }
          if (lane == 0) row[0] = 1.0;
          if (bb < chi) row[bb] = Gb;
        }
      }
      __syncthreads();
      if (warp == 0) {                       // draw, largest index first
        uint32_t fl = 0;
        int bcur = nz;
        const uint32_t traj = (uint32_t)(a.traj0 + b);
        for (int st = 0; st < chi; ++st) {
          const int j = chi - st;
          const double total = tabE[(size_t)bcur * (chi + 1) + j];
          const double u = philox_uniform(a.seed, traj, (uint32_t)a.level, (uint32_t)t, (uint32_t)st);
          const double x = u * total;
          int found = -1;
          for (int i0 = j; i0 <= bcur && found < 0; i0 += 32) {
            const int i = i0 + lane;
            const bool p = (i <= bcur) && (tabE[(size_t)i * (chi + 1) + j] > x);
            const unsigned m = __ballot_sync(0xffffffffu, p);
            if (m) found = i0 + __ffs(m) - 1;
          }
          if (found < 0) { found = bcur; fl |= FLAG_DRAW_TIE; }   // only if the table holds NaN
          const double lo = tabE[(size_t)(found - 1) * (chi + 1) + j];
          const double hi = tabE[(size_t)found * (chi + 1) + j];
          if ((x - lo) <= TIE_TOL * total || (hi - x) <= TIE_TOL * total) fl |= FLAG_DRAW_TIE;
          if (lane == 0) s_kept[st] = found - 1;
          bcur = found - 1;
        }
        __syncwarp();
        // inclusion rate of each kept index (lane a <-> picks a and a + 32)
        for (int pk = lane; pk < chi; pk += 32) {
          const int I = s_kept[pk] + 1;                         // 1-based
          const int alo = max(0, chi - 1 - (nz - I)), ahi = min(chi - 1, I - 1);
          double R = 1.0;
          for (int q = 0; q < chi - ahi; ++q) R *= w[I - 1 + q] / w[ahi + q];
          double acc = 0.0;
          for (int aa = ahi; aa >= alo; --aa) {
            acc += tabE[(size_t)(I - 1) * (chi + 1) + aa] * tabG[(size_t)I * chi + (chi - 1 - aa)] * R;
            if (aa > alo) R *= w[I + chi - aa - 1] / w[aa - 1];
          }
          const double r = acc / tabE[(size_t)nz * (chi + 1) + chi];
          s_sigt[pk] = wn[I - 1] / r;
        }
        __syncwarp();
        // ascending order of the kept indices (distinct, so ranks are unique)
        const int pk2 = lane + 32;
        const int mine = lane < chi ? s_kept[lane] : 0, mine2 = pk2 < chi ? s_kept[pk2] : 0;
        const double mys = lane < chi ? s_sigt[lane] : 0.0, mys2 = pk2 < chi ? s_sigt[pk2] : 0.0;
        int rank = 0, rank2 = 0;
        for (int q = 0; q < chi; ++q) {
          rank += s_kept[q] < mine;
          rank2 += s_kept[q] < mine2;
        }
        __syncwarp();
        if (lane < chi) { s_kept[rank] = mine; s_sigt[rank] = mys; inset[mine] = 1; }
        if (pk2 < chi) { s_kept[rank2] = mine2; s_sigt[rank2] = mys2; inset[mine2] = 1; }
        if (lane == 0 && fl) atomicOr(&s_flags, fl);
      }
    } else {
      const int nkeep = min(nz, kc);
      for (int i = tid; i < nkeep; i += kThreads) inset[i] = 1;
      if (tid < nkeep) { s_kept[tid] = tid; s_sigt[tid] = wn[tid]; }
    }
    __syncthreads();

    const int nk0 = s_nk;
    if (sample) {                              // near-tie flags
      uint32_t fl = 0;
      for (int i = tid; i + 1 < nz; i += kThreads)
        if (inset[i] != inset[i + 1] && (wn[i] - wn[i + 1]) <= GAP_TOL) fl |= FLAG_SPLIT_CLUSTER;
      if (tid < nk0 && wn[s_kept[tid]] < TINY_TOL) fl |= FLAG_TINY_KEPT;
      if (fl) atomicOr(&s_flags, fl);
    }
    if (a.mode == 1) {                         // split form: hand the choices on
      __syncthreads();
      if (tid < ks) {
        a.kept[it * ks + tid] = tid < nk0 ? s_kept[tid] : 0;
        a.sigt[it * ks + tid] = tid < nk0 ? s_sigt[tid] : 0.0;
      }
      if (tid == 0) {
        a.nk[it] = nk0;
        if (a.iflags && s_flags) a.iflags[item - a.h_item0] |= s_flags;
      }
      __syncthreads();
      continue;
    }
    }
    const int nk = s_nk;

    // ---- halves ----
    double* Hl = a.H + (size_t)(item - a.h_item0) * 2 * n * kc;
    double* Hr = Hl + (size_t)n * kc;
    const double* Wm = a.W + (size_t)slot * np * n;
    const int* pm = a.perm + (size_t)slot * np;
    for (int idx = tid; idx < kc * n; idx += kThreads) {
      const int al = idx / n, col = idx - al * n;
      double v = 0.0;
      if (al < nk) {
        const int r = s_kept[al];
        const double* brow = a.mode == 2 ? a.vrows + ((size_t)it * ks + al) * n : Wm + (size_t)pm[r] * n;
        v = sqrt(s_sigt[al]) * brow[col] / sg[r];
      }
      Hr[idx] = v;
    }
    if (a.Urows) {
      const double* Ur = a.Urows + (size_t)slot * np * n;
      for (int idx = tid; idx < n * kc; idx += kThreads) {
        const int row = idx / kc, al = idx - row * kc;
        double v = 0.0;
        if (al < nk) v = sqrt(s_sigt[al]) * Ur[(size_t)s_kept[al] * n + row];
        Hl[idx] = v;
      }
    } else {
      const double* Mm = a.M + (size_t)slot * n * n;
      for (int idx = tid; idx < n * kc; idx += kThreads) {
        const int al = idx - (idx / kc) * kc;
        if (al >= nk) Hl[idx] = 0.0;
      }
      for (int a0 = 0; a0 < nk; a0 += KV) {
        const int nv = min(KV, nk - a0);
        __syncthreads();
        for (int idx = tid; idx < nv * n; idx += kThreads) {
          const int q = idx / n, col = idx - q * n;
          vbuf[idx] = a.mode == 2 ? a.vrows[((size_t)it * ks + a0 + q) * n + col]
                                  : Wm[(size_t)pm[s_kept[a0 + q]] * n + col];
        }
        __syncthreads();
        for (int row = warp; row < n; row += kThreads / 32) {
          double acc[KV];
#pragma unroll
          for (int q = 0; q < KV; ++q) acc[q] = 0.0;
          const double* mr = Mm + (size_t)row * n;
          for (int col = lane; col < n; col += 32) {
            const double mv = mr[col];
#pragma unroll
            for (int q = 0; q < KV; ++q)
              if (q < nv) acc[q] = fma(mv, vbuf[q * n + col], acc[q]);
          }
          const double sum = warp_sum_k<KV>(acc, lane);
          const int q = lane / (32 / KV);
          if (lane % (32 / KV) == 0 && q < nv) {
            const int r = s_kept[a0 + q];
            const double sr = sg[r];
            Hl[(size_t)row * kc + a0 + q] = sqrt(s_sigt[a0 + q]) * sum / (sr * sr);
          }
        }
      }
    }
    __syncthreads();
    if (tid == 0 && a.iflags && s_flags && a.mode == 0) a.iflags[item - a.h_item0] |= s_flags;
    __syncthreads();
  }
}

cudaError_t launch_sample_split(const SampleArgs& a, cudaStream_t st, int grid) {
  if (a.n_items <= 0) return cudaSuccess;
  if (a.chi > kKeptMax || a.kc > kKeptMax || (a.mode != 0 && a.kstride < std::max(a.chi, a.kc)))
    return cudaErrorInvalidValue;
  const auto smem_for = [&](int kv) {
    return (size_t)a.n_pad * 2 * sizeof(double) + (size_t)kv * a.n * sizeof(double) + (size_t)a.n_pad + 16;
  };
  if (grid > a.n_items) grid = (int)a.n_items;
  constexpr size_t kSmemCap = 227 * 1024;
  if (smem_for(16) <= 160 * 1024) {
    static std::atomic<uint64_t> attr{0};
    cudaError_t e = raise_smem_limit(k_sample_split<16>, kSmemCap, attr);
    if (e != cudaSuccess) return e;
    k_sample_split<16><<<grid, kThreads, smem_for(16), st>>>(a);
  } else {
    if (smem_for(8) > kSmemCap) return cudaErrorInvalidValue;
    static std::atomic<uint64_t> attr{0};
    cudaError_t e = raise_smem_limit(k_sample_split<8>, kSmemCap, attr);
    if (e != cudaSuccess) return e;
    k_sample_split<8><<<grid, kThreads, smem_for(8), st>>>(a);
  }
  return cudaGetLastError();
}

// u_r = M v_r / s_r = M b_r / s_r^2 for every rank r < nnz of S matrices,
// stored by rank as rows: Urows[slot][r][row].  One CTA per (slot, r).
__global__ void k_u_rows(const double* M, const double* W, const double* sig, const int* perm,
                         const int* nnz, double* Urows, int n, int n_pad) {
  const int slot = blockIdx.y, r = blockIdx.x;
  double* out = Urows + ((size_t)slot * n_pad + r) * n;
  if (r >= nnz[slot]) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = 0.0;
    return;
  }
  const double s = sig[(size_t)slot * n_pad + r];
  const double* b = W + ((size_t)slot * n_pad + perm[(size_t)slot * n_pad + r]) * n;
  const double* Mm = M + (size_t)slot * n * n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int row = warp; row < n; row += nw) {
    double acc = 0.0;
    for (int c = lane; c < n; c += 32) acc = fma(Mm[(size_t)row * n + c], b[c], acc);
    acc = warp_sum(acc);
    if (lane == 0) out[row] = acc / (s * s);
  }
}

cudaError_t launch_u_rows(const double* M, const double* W, const double* sig, const int* perm,
                          const int* nnz, double* Urows, int n, int n_pad, int S, cudaStream_t st) {
  dim3 grid(n_pad, S);
  k_u_rows<<<grid, 128, 0, st>>>(M, W, sig, perm, nnz, Urows, n, n_pad);
  return cudaGetLastError();
}

}  // namespace mctrg
