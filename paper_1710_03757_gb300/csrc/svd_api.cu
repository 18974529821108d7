// C-ABI access to the batched Jacobi SVD (K2) on its own.
#include <algorithm>
#include <vector>

#include "../../include/mctrg.h"
#include "common.cuh"
#include "kernels.h"
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

}  // namespace mctrg

using namespace mctrg;

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
