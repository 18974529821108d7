// FP64 throughput probe: the denominator of the FP64-pipe roofline.
//
// Every thread runs CH independent DFMA recurrences x <- x b + c for a fixed
// number of steps, so the FP64 pipe sees CH independent instructions per
// thread between dependences and the warps of an SM keep it busy; the grid is
// a whole number of CTAs per SM.  Several shapes (chains per thread, threads
// per CTA) run the same work, and a 4 x 4 outer product of changing operands
// (the instruction pattern of a GEMM, which the FP64 pipe sustains better
// than dependent chains of one operand); the best rate is the peak.  The recurrence contracts
// toward c / (1 - b), so every value stays finite and normal, and the final
// values are summed into one word that the host reads (nothing is dead code).
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/mctrg.h"

namespace {

// CH independent chains per thread, unrolled U steps per loop trip.
template <int CH, int U>
__global__ void k_dfma_probe(int64_t steps, double b, double c, double* sink) {
  double x[CH];
#pragma unroll
  for (int j = 0; j < CH; ++j) x[j] = 1.0 + 1e-3 * (threadIdx.x + j);
  for (int64_t s = 0; s < steps; s += U) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int j = 0; j < CH; ++j) x[j] = fma(x[j], b, c);
    }
  }
  double t = 0.0;
#pragma unroll
  for (int j = 0; j < CH; ++j) t += x[j];
  if (t == 12345.678) sink[0] = t;   // never true; keeps the chains live
  if (threadIdx.x == 0 && blockIdx.x == 0) sink[1] = t;
}

// A 4 x 4 outer product per step (the FP64 GEMM's instruction pattern): 16
// independent accumulators fed by 8 operands, each FMA with distinct inputs.
template <int CH, int U>
__global__ void k_dfma_outer(int64_t steps, double b, double c, double* sink) {
  double acc[4][4], x[4], y[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    x[p] = b * (1.0 + 1e-3 * (threadIdx.x + p));
    y[p] = c * (1.0 - 1e-3 * (threadIdx.x + p));
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = 0.0;
  }
  for (int64_t s = 0; s < steps; s += U) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(x[p], y[q], acc[p][q]);
    }
  }
  double t = 0.0;
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) t += acc[p][q];
  if (t == 12345.678) sink[0] = t;
  if (threadIdx.x == 0 && blockIdx.x == 0) sink[1] = t;
}

// Best of three timed launches of one variant (after one untimed launch);
// returns the rate in TFLOP/s (0 on failure) and its launch time in *ms.
template <int CH, int U>
double time_variant(void (*kern)(int64_t, double, double, double*), int sms, int threads, int64_t steps,
                    double* sink, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0) != cudaSuccess || per_sm < 1)
    return 0.0;
  const int grid = sms * per_sm;
  const int64_t st = (steps / U) * U;
  kern<<<grid, threads>>>(st / 4 < U ? U : (st / 4 / U) * U, 0.9999999, 1e-7, sink);
  if (cudaGetLastError() != cudaSuccess) return 0.0;
  float best = 0.f;
  for (int r = 0; r < 3; ++r) {
    float t = 0.f;
    if (cudaEventRecord(e0) != cudaSuccess) return 0.0;
    kern<<<grid, threads>>>(st, 0.9999999, 1e-7, sink);
    if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1) != cudaSuccess ||
        cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
      return 0.0;
    if (r == 0 || t < best) best = t;
  }
  *ms = best;
  return 2.0 * CH * (double)st * grid * threads / (best * 1e-3) / 1e12;
}

}  // namespace

extern "C" int mctrg_measure_fp64_peak(int device, int64_t steps, double* tflops, double* ms) {
  if (!tflops || steps < 16) return MCTRG_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return MCTRG_ECUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return MCTRG_ECUDA;
  double* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMalloc(&sink, 2 * sizeof(double)) != cudaSuccess) return MCTRG_ECUDA;
  double best = 0.0;
  float best_ms = 0.f;
  if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    // a few shapes of the same work: the pipe's rate is the best of them
    const int threads[3] = {128, 256, 512};
    for (int ti = 0; ti < 3; ++ti) {
      float t = 0.f;
      double r;
      r = time_variant<4, 8>(k_dfma_probe<4, 8>, sms, threads[ti], steps, sink, e0, e1, &t);
      if (r > best) { best = r; best_ms = t; }
      r = time_variant<8, 4>(k_dfma_probe<8, 4>, sms, threads[ti], steps, sink, e0, e1, &t);
      if (r > best) { best = r; best_ms = t; }
      r = time_variant<16, 2>(k_dfma_probe<16, 2>, sms, threads[ti], steps, sink, e0, e1, &t);
      if (r > best) { best = r; best_ms = t; }
      r = time_variant<16, 2>(k_dfma_outer<16, 2>, sms, threads[ti], steps, sink, e0, e1, &t);
      if (r > best) { best = r; best_ms = t; }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  if (!(best > 0.0)) return MCTRG_ECUDA;
  *tflops = best;
  if (ms) *ms = best_ms;
  return MCTRG_OK;
}
