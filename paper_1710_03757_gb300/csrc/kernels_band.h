// Launch interfaces of the two-stage (band) route of the batched SVD (K2):
// dense -> band reduction with its trailing updates on the tensor cores,
// band -> bidiagonal by bulge chasing, and the back-transformation of the
// kept right vectors through both stages.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mctrg {

constexpr int kBandW = 8;   // band width b: stage-1 panels of b columns, b superdiagonals

// Sides the band route takes: multiples of b from 64 to 256 (the inner
// dimension of the tensor-core products stays <= 256, where their FP32 group
// sums are exact).
bool band_supported(int n);

// Right reflectors of the bulge chase of one n x n band.
int band_nref(int n);

// Per-matrix device buffers of the route (S matrices of side n).
struct BandArgs {
  const double* M;    // [S][n][n] input, read only
  int64_t* Wk;        // [S][n][n] working matrix (the bidiagonalization route's W buffer):
                      //   fixed point during stage 1; on return rows k..k+b-1 of each panel
                      //   hold its right reflectors U (columns k+b..) and their T factor
                      //   (columns k..k+b-1), as doubles
  double* band;       // [S][n][b+1] band[i][o] = B(i, i+o)
  double* bd;         // [S][3n] d, e of the bidiagonal (third part zero)
  double* refl;       // [S][nref][b] chase reflectors, sweep by sweep: tau, v_1 .. v_{b-1}
                      //   (step t of sweep i acts on columns i+1+8t ..)
  double* work;       // per-matrix panel scratch: band_work_doubles(n) doubles each
  int* eA;            // [S] fixed-point exponent of each matrix
  uint32_t* err;      // set to 1 when a bounded wait of a tensor-core kernel expired
  int n, S;
};
size_t band_work_doubles(int n);
// Bytes per matrix of band, work, refl and eA (Wk and bd are the
// caller's); band_carve lays them out for S matrices from `base` (which must
// hold S * band_item_bytes(n) + 256 bytes) and puts err after them.
size_t band_item_bytes(int n);
void band_carve(void* base, int n, int64_t S, BandArgs& a);

// Stage 1 and 2: M -> band (Wk, band) -> bidiagonal (bd).  Stage 1 alone when
// chase == false (band filled, bd untouched).
cudaError_t launch_band_reduce(const BandArgs& a, bool chase, cudaStream_t st);
// Stage 2 alone (after launch_band_reduce(a, false, st)).
cudaError_t launch_band_chase(const BandArgs& a, cudaStream_t st);

// v = P1 P2 v_B for the kept vectors: vrows[s][a][:] holds v_B on entry
// (unit vectors of the bidiagonal, from the inverse iteration) and s_r v_r on
// return (v_r with unit_rows).  kmax <= 16.
struct BandVecArgs {
  const BandArgs* band;   // the reduction's buffers (host copy of the struct)
  const double* sig;      // [S][n_pad]
  const int* kept;        // [S][kstride]
  const int* nk;          // [S]
  double* vrows;          // [S][kstride][n]
  int n_pad, kstride, unit_rows;
};
cudaError_t launch_band_backtr(const BandVecArgs& a, cudaStream_t st);

}  // namespace mctrg
