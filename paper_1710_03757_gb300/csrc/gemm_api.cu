// The plaquette GEMM through the C ABI on its own: M[b] = X[b] Yt[b]^T,
// plain row-major output (the matricization epilogue with parity A is the
// identity map), on the CUDA cores in FP64 or at FP64 accuracy on the tensor
// cores (BF16 slices).
#include <cstdint>

#include "../../include/mctrg.h"
#include "common.cuh"
#include "kernels.h"
#include "kernels_tc.h"

extern "C" int mctrg_contract_batched(const double* X, const double* Yt, int D, int K, int64_t batch, double* M,
                                      int precision, void* stream) {
  if (!X || !Yt || !M || D < 1 || D > 32 || K < 1 || batch < 1 || batch > (1 << 30)) return MCTRG_EINVAL;
  const int n = D * D;
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == MCTRG_FP64) {
    mctrg::GemmArgs gm{};
    gm.X = X; gm.Yt = Yt; gm.M = M; gm.D = D; gm.K = K; gm.c0 = 0; gm.n_items = batch; gm.Nnew = 1;
    gm.L = 2; gm.level_new = 0; gm.fixed_parity = 0;
    if (mctrg::launch_gemm_f64(gm, st) != cudaSuccess) return MCTRG_ECUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? MCTRG_OK : MCTRG_ECUDA;
  }
  if (precision != MCTRG_FP64TC || !mctrg::gemm_ozaki_supported(n, K)) return MCTRG_EINVAL;
  int bits = 0, slices = 0;
  mctrg::ozaki_params(K, &bits, &slices);
  const size_t elems = (size_t)batch * n * K;
  void *xs = nullptr, *ys = nullptr;
  int* ex = nullptr;
  uint32_t* err = nullptr;
  int status = MCTRG_ENOMEM;
  if (cudaMalloc(&xs, 2 * slices * elems) != cudaSuccess || cudaMalloc(&ys, 2 * slices * elems) != cudaSuccess ||
      cudaMalloc(&ex, sizeof(int) * 2 * (size_t)batch * n) != cudaSuccess ||
      cudaMalloc(&err, sizeof(uint32_t)) != cudaSuccess)
    goto out;
  status = MCTRG_ECUDA;
  {
    const int64_t rows = batch * n;
    uint32_t herr = 0;
    mctrg::GemmOzArgs ga{};
    ga.M = M; ga.D = D; ga.n = n; ga.K = K; ga.c0 = 0; ga.n_items = batch; ga.Nnew = 1; ga.L = 2;
    ga.level_new = 0; ga.fixed_parity = 0; ga.expX = ex; ga.expY = ex + rows; ga.slices = slices;
    ga.bits = bits; ga.err = err;
    if (cudaMemsetAsync(err, 0, sizeof(uint32_t), st) != cudaSuccess ||
        mctrg::launch_ozaki_split(X, rows, K, xs, ex, st) != cudaSuccess ||
        mctrg::launch_ozaki_split(Yt, rows, K, ys, ex + rows, st) != cudaSuccess ||
        mctrg::launch_gemm_ozaki(ga, xs, ys, st) != cudaSuccess ||
        cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      goto out;
    status = herr ? MCTRG_ECUDA : MCTRG_OK;
  }
out:
  cudaStreamSynchronize(st);
  cudaFree(xs);
  cudaFree(ys);
  cudaFree(ex);
  cudaFree(err);
  return status;
}
