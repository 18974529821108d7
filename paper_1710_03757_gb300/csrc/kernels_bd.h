// Launch interfaces of the bidiagonalization route of the batched SVD (K2).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mctrg {

// Stride of the per-matrix kept-index arrays (kept ranks, reweighted values,
// kept vectors) for a kept count kc <= 64: 32 up to 32 kept values, else 64.
inline int kept_stride(int kc) { return kc <= 32 ? 32 : 64; }
constexpr int kKeptMax = 64;

// One matrix of a ragged launch: matrices of different sizes (and owners) in
// one launch of the bidiagonalization route, each with its own buffers.
struct SvdItem {
  const double* M;    // n x n input
  double* W;          // n x n working copy; right reflectors on return
  double* bd;         // 3n: d, e, tauR
  double* sig;        // n_pad singular values, descending
  int* perm;          // n_pad
  int* nnz;           // 1
  double* lns1;       // 1 (may be null)
  const int* kept;    // kept ranks (ascending), up to 64
  const int* nk;      // 1
  double* vrows;      // nk x n: s_r v_r of the kept ranks
  double zero_rel;    // zero threshold (<= 0: n 2^-52)
  int n, n_pad;
};

// 1. Householder bidiagonalization  Q_L^T M Q_R = B  (upper bidiagonal) of S
//    row-major n x n matrices.  bd[s] = [d (n) | e (n, e[n-1] = 0) | tauR (n)];
//    the right reflector of step k, u_k = (1, R[k][k+2], ..., R[k][n-1]) on
//    columns k+1.., stays in row k of the working copy R = W[s] (n x n).
//    Sides up to 1024 keep a row's columns in registers; larger sides (up to
//    2304) stream them in two passes per row group.
struct BidiagArgs {
  const double* M;   // [S][n][n] read only
  double* W;         // [S][n][n] (any row stride >= n is not supported: n x n)
  double* bd;        // [S][3n]
  int n, S;
  const SvdItem* items = nullptr;   // ragged: S matrices described here (n = the largest)
};
cudaError_t launch_bidiag(const BidiagArgs& a, cudaStream_t st);
// The same over a ragged set of S matrices (device table; n_max the largest
// side; smem the largest bidiag_smem_bytes of their sides).
size_t bidiag_smem_bytes(int n);
cudaError_t launch_bidiag_items(const SvdItem* items, int S, int n_max, size_t smem, cudaStream_t st);

// 2. All singular values of each B by bisection on Sturm counts of the
//    Golub-Kahan tridiagonal; written descending into sig[S][n_pad] with
//    perm[r] = r, nnz = #{s > zero_rel s_1} (zero_rel <= 0: n 2^-52) and
//    lns1 = ln s_1 (may be null).  Values surely below the zero threshold are
//    written as 0.
cudaError_t launch_bd_bisect(const double* bd, int n, int n_pad, int S, double* sig, int* perm, int* nnz,
                             double* lns1, double zero_rel, cudaStream_t st);
// The same over a ragged set of matrices (n_max = the largest n; device table).
cudaError_t launch_bd_bisect_items(const SvdItem* items, int S, int n_max, cudaStream_t st);

// 3. Right singular vectors of the kept indices: kept[s][0..nk[s]-1] are
//    ranks (ascending, so singular values descending).  vrows[s][a][0..n-1]
//    receives s_r v_r for r = kept[s][a] (the scaling of a Jacobi row),
//    computed by inverse iteration on the Golub-Kahan tridiagonal
//    (reorthogonalized within clusters of close kept values) and the right
//    reflectors.  scratch: bd_vectors_scratch_doubles(n, S, kmax) doubles.
struct BdVecArgs {
  const double* bd;     // [S][3n]
  const double* R;      // [S][n][n] reflectors (row k holds u_k)
  const double* sig;    // [S][n_pad]
  const int* kept;      // [S][kstride]
  const int* nk;        // [S]
  double* vrows;        // [S][kstride][n]
  double* scratch;
  int n, n_pad, S;
  int unit_rows;        // 1: write v_r itself instead of s_r v_r
  int kmax;             // largest nk of the batch (<= 64)
  int kstride;          // kept_stride of the largest kept count (non-ragged layout)
  const SvdItem* items = nullptr;   // ragged: S matrices described here (n = the largest)
  int skip_backtr = 0;  // 1: leave the unit vectors of the bidiagonal in vrows
};
cudaError_t launch_bd_vectors(const BdVecArgs& a, cudaStream_t st);
size_t bd_vectors_scratch_doubles(int n, int S, int kmax);

}  // namespace mctrg
