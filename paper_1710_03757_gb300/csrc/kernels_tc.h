// Launch interface of the tensor-core (tcgen05) plaquette GEMM.
#pragma once
#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

namespace mctrg {

constexpr int kTcMaxStages = 4;

struct GemmTcArgs {
  double* M;              // [n_items][n][n] FP64 output, matricized like k_gemm_f64
  int D, n, K;            // n = D*D output rows/cols, K = d*d
  int64_t c0, n_items, Nnew;
  int L, level_new;
  int fixed_parity;       // >= 0 overrides the geometry
  const double* scaleX;   // [n_items] scale of X (max |X|)
  const double* scaleY;   // [n_items] scale of Yt
  int passes;             // 1: hi*hi; 3: hi*hi + hi*lo + lo*hi
  uint32_t* err;          // set to 1 when a bounded wait expired
};

// X or Yt (n_items x per_item FP64) -> scaled TF32-in-FP32 (kind 0) or BF16
// (kind 1) hi part and optional residual lo part; scale[i] = max |block i|.
cudaError_t launch_convert_scaled(const double* src, int64_t per_item, int64_t n_items, int kind, void* hi,
                                  void* lo, double* scale, cudaStream_t st);
bool gemm_tc_supported(int n, int K, int kind);
cudaError_t launch_gemm_tc(const GemmTcArgs& a, int kind, const void* Xh, const void* Yh, const void* Xl,
                           const void* Yl, cudaStream_t st);

// ---- FP64-accurate GEMM on the tensor cores (BF16 slices, Ozaki scheme) ----
struct GemmOzArgs {
  double* M;              // [n_items][n][n] FP64 output, matricized like k_gemm_f64
  int D, n, K;            // n = D*D output rows/cols, K = d*d (multiple of 64, <= 1024)
  int64_t c0, n_items, Nnew;
  int L, level_new;
  int fixed_parity;       // >= 0 overrides the geometry
  const int* expX;        // [n_items][n] row exponents of X (every |x| < 2^e)
  const int* expY;        // [n_items][n] row exponents of Yt
  int slices, bits;       // slice planes per operand and bits per slice (ozaki_params)
  uint32_t* err;          // set to 1 when a bounded wait expired
};
// Slice width b (bits) and slice count s for inner dimension K.
void ozaki_params(int K, int* bits, int* slices);
bool gemm_ozaki_supported(int n, int K);
// rows x K FP64 (row-major) -> s BF16 slice planes [s][rows][K] and row exponents.
cudaError_t launch_ozaki_split(const double* src, int64_t rows, int K, void* dst, int* expo, cudaStream_t st);
cudaError_t launch_gemm_ozaki(const GemmOzArgs& a, const void* Xs, const void* Ys, cudaStream_t st);

}  // namespace mctrg
