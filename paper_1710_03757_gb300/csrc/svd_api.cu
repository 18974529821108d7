// C-ABI access to the batched SVD (K2) on its own: the Jacobi route, the
// bidiagonalization route and the two-stage (band) route.
#include <algorithm>
#include <vector>

#include "../../include/mctrg.h"
#include "common.cuh"
#include "kernels.h"
#include "kernels_band.h"
#include "kernels_bd.h"
#include "mctrg_internal.h"

namespace mctrg {

// sigma[b][r] = s_r (r < n, descending); vt[b][r][:] = unit right vector of s_r.
__global__ void k_svd_finalize(const double* W, const double* sig, const int* perm, int n, int n_pad,
                               double* sigma, double* vt) {
  const int64_t b = blockIdx.x;
  const double* sg = sig + b * n_pad;
  const int* pm = perm + b * n_pad;
  for (int r = threadIdx.x; r < n; r += blockDim.x) sigma[b * n + r] = sg[r];
  if (!vt) return;
  for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) {
    const int r = (int)(e / n), c = (int)(e - (int64_t)r * n);
    const double s = sg[r];
    vt[b * n * n + e] = s > 0.0 ? W[(b * n_pad + pm[r]) * n + c] / s : 0.0;
  }
}

cudaError_t svd_chunk(const double* M, int n, int64_t count, double* sigma, double* vt, int max_sweeps,
                      double* W, double* sig, int* perm, int* nnz, uint32_t* flags, cudaStream_t st) {
  const int np = n + (n & 1);
  JacobiArgs ja{};
  ja.M = M; ja.W = W; ja.sig = sig; ja.perm = perm; ja.lns1 = nullptr; ja.nnz = nnz; ja.mflags = flags;
  ja.n = n; ja.n_pad = np; ja.S = (int)count; ja.max_sweeps = max_sweeps;
  cudaError_t e = launch_jacobi(ja, st);
  if (e != cudaSuccess) return e;
  k_svd_finalize<<<(unsigned)count, 256, 0, st>>>(W, sig, perm, n, np, sigma, vt);
  return cudaGetLastError();
}

// Kept ranks 0 .. nv-1 for every matrix (the leading right vectors), stride ks.
__global__ void k_kept_leading(int* kept, int* nk, const int* nnz, int nv, int S, int ks) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  for (int q = 0; q < ks; ++q) kept[(size_t)s * ks + q] = q < nv ? q : 0;
  nk[s] = nv;
}

__global__ void k_bd_finalize(const double* sig, int n, int n_pad, int nv, const double* vrows, double* sigma,
                              double* vt, int ks) {
  const int64_t b = blockIdx.x;
  for (int r = threadIdx.x; r < n; r += blockDim.x) sigma[b * n + r] = sig[b * n_pad + r];
  if (!vt) return;
  for (int64_t e = threadIdx.x; e < (int64_t)nv * n; e += blockDim.x) vt[b * nv * n + e] = vrows[b * ks * n + e];
}

}  // namespace mctrg

using namespace mctrg;

extern "C" int mctrg_svd_bidiag_batched(const double* M, int n, int64_t batch, double* sigma, int n_vec,
                                        double* vt, void* stream) {
  if (!M || !sigma || n < 2 || n > 2304 || batch < 1 || batch > (1 << 30)) return MCTRG_EINVAL;
  if (n_vec < 0 || n_vec > kKeptMax || n_vec > n || (n_vec > 0 && !vt)) return MCTRG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int np = n + (n & 1);
  const int ks = kept_stride(n_vec);
  const size_t per = ((size_t)n * n + 3 * (size_t)n + np + (size_t)ks * n) * sizeof(double) +
                     ((size_t)np + 1 + ks + 1) * sizeof(int);
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return MCTRG_ECUDA;
  const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>({batch, (int64_t)(fr / 4 / per), 1 << 16}));
  const size_t scr = bd_vectors_scratch_doubles(n, (int)chunk, std::max(1, n_vec)) * sizeof(double);
  void* buf = nullptr;
  if (cudaMalloc(&buf, per * (size_t)chunk + scr) != cudaSuccess) return MCTRG_ENOMEM;
  double* W = (double*)buf;
  double* bd = W + (size_t)chunk * n * n;
  double* sig = bd + (size_t)chunk * 3 * n;
  double* vrows = sig + (size_t)chunk * np;
  double* scratch = vrows + (size_t)chunk * ks * n;
  int* perm = (int*)(scratch + scr / sizeof(double));
  int* nnz = perm + (size_t)chunk * np;
  int* kept = nnz + chunk;
  int* nk = kept + (size_t)chunk * ks;
  int status = MCTRG_OK;
  for (int64_t b0 = 0; b0 < batch; b0 += chunk) {
    const int cnt = (int)std::min(chunk, batch - b0);
    BidiagArgs ba{};
    ba.M = M + (size_t)b0 * n * n; ba.W = W; ba.bd = bd; ba.n = n; ba.S = cnt;
    cudaError_t e = launch_bidiag(ba, st);
    if (e == cudaSuccess) e = launch_bd_bisect(bd, n, np, cnt, sig, perm, nnz, nullptr, 0.0, st);
    if (e == cudaSuccess && n_vec > 0) {
      k_kept_leading<<<(cnt + 127) / 128, 128, 0, st>>>(kept, nk, nnz, n_vec, cnt, ks);
      BdVecArgs va{};
      va.bd = bd; va.R = W; va.sig = sig; va.kept = kept; va.nk = nk; va.vrows = vrows; va.scratch = scratch;
      va.n = n; va.n_pad = np; va.S = cnt; va.unit_rows = 1; va.kmax = n_vec; va.kstride = ks;
      e = launch_bd_vectors(va, st);
    }
    if (e == cudaSuccess) {
      k_bd_finalize<<<cnt, 256, 0, st>>>(sig, n, np, n_vec, vrows, sigma + (size_t)b0 * n,
                                          n_vec > 0 ? vt + (size_t)b0 * n_vec * n : nullptr, ks);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) { status = MCTRG_ECUDA; break; }
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) status = MCTRG_ECUDA;
  cudaFree(buf);
  return status;
}

// Device buffers of the band route for `chunk` matrices of side n, carved
// from one allocation: Wk (n x n), bd (3n), then band_carve's.
static size_t band_bytes(int n, int64_t chunk) {
  // rounded up to 256 bytes: the buffers that follow hold doubles
  const size_t b = (size_t)chunk * (sizeof(double) * ((size_t)n * n + 3 * (size_t)n) + band_item_bytes(n)) + 256;
  return (b + 255) & ~(size_t)255;
}
static void band_all(void* buf, int n, int64_t chunk, BandArgs& a) {
  double* p = (double*)buf;
  a.Wk = (int64_t*)p; p += (size_t)chunk * n * n;
  a.bd = p; p += (size_t)chunk * 3 * n;
  band_carve(p, n, chunk, a);
}

extern "C" int mctrg_band_reduce_batched(const double* M, int n, int64_t batch, double* band, double* bd,
                                         void* stream) {
  if (!M || !band || !band_supported(n) || batch < 1 || batch > (1 << 30)) return MCTRG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return MCTRG_ECUDA;
  const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>({batch, (int64_t)(fr / 4 / band_bytes(n, 1)), 1 << 14}));
  void* buf = nullptr;
  if (cudaMalloc(&buf, band_bytes(n, chunk)) != cudaSuccess) return MCTRG_ENOMEM;
  BandArgs a{};
  band_all(buf, n, chunk, a);
  int status = cudaMemsetAsync(a.err, 0, sizeof(uint32_t), st) == cudaSuccess ? MCTRG_OK : MCTRG_ECUDA;
  for (int64_t b0 = 0; b0 < batch && status == MCTRG_OK; b0 += chunk) {
    const int cnt = (int)std::min(chunk, batch - b0);
    a.M = M + (size_t)b0 * n * n; a.S = cnt;
    cudaError_t e = launch_band_reduce(a, bd != nullptr, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(band + (size_t)b0 * n * (kBandW + 1), a.band, sizeof(double) * cnt * n * (kBandW + 1),
                          cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && bd)
      e = cudaMemcpyAsync(bd + (size_t)b0 * 3 * n, a.bd, sizeof(double) * cnt * 3 * n, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) status = MCTRG_ECUDA;
  }
  uint32_t err = 0;
  if (cudaMemcpyAsync(&err, a.err, sizeof(err), cudaMemcpyDeviceToHost, st) != cudaSuccess) status = MCTRG_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) status = MCTRG_ECUDA;
  if (status == MCTRG_OK && err) status = MCTRG_ECUDA;
  cudaFree(buf);
  return status;
}

extern "C" int mctrg_svd_band_batched(const double* M, int n, int64_t batch, double* sigma, int n_vec,
                                      double* vt, void* stream) {
  if (!M || !sigma || !band_supported(n) || batch < 1 || batch > (1 << 30)) return MCTRG_EINVAL;
  if (n_vec < 0 || n_vec > 16 || n_vec > n || (n_vec > 0 && !vt)) return MCTRG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int np = n + (n & 1);
  const int ks = kept_stride(n_vec);
  const size_t per_extra = ((size_t)np + (size_t)ks * n) * sizeof(double) + ((size_t)np + 1 + ks + 1) * sizeof(int);
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return MCTRG_ECUDA;
  const int64_t chunk = std::max<int64_t>(
      1, std::min<int64_t>({batch, (int64_t)(fr / 4 / (band_bytes(n, 1) + per_extra)), 1 << 14}));
  const size_t scr = bd_vectors_scratch_doubles(n, (int)chunk, std::max(1, n_vec)) * sizeof(double);
  const size_t bb = band_bytes(n, chunk);
  void* buf = nullptr;
  if (cudaMalloc(&buf, bb + per_extra * (size_t)chunk + scr) != cudaSuccess) return MCTRG_ENOMEM;
  BandArgs a{};
  band_all(buf, n, chunk, a);
  double* sig = (double*)((char*)buf + bb);
  double* vrows = sig + (size_t)chunk * np;
  double* scratch = vrows + (size_t)chunk * ks * n;
  int* perm = (int*)(scratch + scr / sizeof(double));
  int* nnz = perm + (size_t)chunk * np;
  int* kept = nnz + chunk;
  int* nk = kept + (size_t)chunk * ks;
  int status = cudaMemsetAsync(a.err, 0, sizeof(uint32_t), st) == cudaSuccess ? MCTRG_OK : MCTRG_ECUDA;
  for (int64_t b0 = 0; b0 < batch && status == MCTRG_OK; b0 += chunk) {
    const int cnt = (int)std::min(chunk, batch - b0);
    a.M = M + (size_t)b0 * n * n; a.S = cnt;
    cudaError_t e = launch_band_reduce(a, true, st);
    if (e == cudaSuccess) e = launch_bd_bisect(a.bd, n, np, cnt, sig, perm, nnz, nullptr, 0.0, st);
    if (e == cudaSuccess && n_vec > 0) {
      k_kept_leading<<<(cnt + 127) / 128, 128, 0, st>>>(kept, nk, nnz, n_vec, cnt, ks);
      BdVecArgs va{};
      va.bd = a.bd; va.R = nullptr; va.sig = sig; va.kept = kept; va.nk = nk; va.vrows = vrows; va.scratch = scratch;
      va.n = n; va.n_pad = np; va.S = cnt; va.unit_rows = 1; va.kmax = n_vec; va.kstride = ks; va.skip_backtr = 1;
      e = launch_bd_vectors(va, st);
      if (e == cudaSuccess) {
        BandVecArgs bv{};
        bv.band = &a; bv.sig = sig; bv.kept = kept; bv.nk = nk; bv.vrows = vrows; bv.n_pad = np; bv.kstride = ks;
        bv.unit_rows = 1;
        e = launch_band_backtr(bv, st);
      }
    }
    if (e == cudaSuccess) {
      k_bd_finalize<<<cnt, 256, 0, st>>>(sig, n, np, n_vec, vrows, sigma + (size_t)b0 * n,
                                          n_vec > 0 ? vt + (size_t)b0 * n_vec * n : nullptr, ks);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) status = MCTRG_ECUDA;
  }
  uint32_t err = 0;
  if (cudaMemcpyAsync(&err, a.err, sizeof(err), cudaMemcpyDeviceToHost, st) != cudaSuccess) status = MCTRG_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) status = MCTRG_ECUDA;
  if (status == MCTRG_OK && err) status = MCTRG_ECUDA;
  cudaFree(buf);
  return status;
}

extern "C" int mctrg_svd_batched(const double* M, int n, int64_t batch, double* sigma, double* vt,
                                 int max_sweeps, void* stream) {
  if (!M || !sigma || n < 1 || n > 1024 || batch < 1 || batch > (1 << 30)) return MCTRG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (max_sweeps <= 0) max_sweeps = 40;
  const int np = n + (n & 1);
  const size_t per = (size_t)np * n * sizeof(double) + (size_t)np * (sizeof(double) + sizeof(int)) +
                     sizeof(int) + sizeof(uint32_t);
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return MCTRG_ECUDA;
  const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(batch, (int64_t)(fr / 4 / per)));
  void* buf = nullptr;
  if (cudaMalloc(&buf, per * (size_t)chunk) != cudaSuccess) return MCTRG_ENOMEM;
  double* W = (double*)buf;
  double* sig = W + (size_t)chunk * np * n;
  int* perm = (int*)(sig + (size_t)chunk * np);
  int* nnz = perm + (size_t)chunk * np;
  uint32_t* flags = (uint32_t*)(nnz + chunk);
  int status = MCTRG_OK;
  bool noconv = false;
  std::vector<uint32_t> hf;
  for (int64_t b0 = 0; b0 < batch && status == MCTRG_OK; b0 += chunk) {
    const int64_t cnt = std::min(chunk, batch - b0);
    if (cudaMemsetAsync(flags, 0, sizeof(uint32_t) * cnt, st) != cudaSuccess ||
        svd_chunk(M + (size_t)b0 * n * n, n, cnt, sigma + (size_t)b0 * n, vt ? vt + (size_t)b0 * n * n : nullptr,
                  max_sweeps, W, sig, perm, nnz, flags, st) != cudaSuccess) {
      status = MCTRG_ECUDA;
      break;
    }
    hf.resize((size_t)cnt);
    if (cudaMemcpyAsync(hf.data(), flags, sizeof(uint32_t) * cnt, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      status = MCTRG_ECUDA;
      break;
    }
    for (uint32_t f : hf) noconv |= (f & FLAG_NOCONV) != 0;
  }
  cudaStreamSynchronize(st);
  cudaFree(buf);
  if (status == MCTRG_OK && noconv) status = MCTRG_ENOCONV;
  return status;
}
