// Launch interfaces of the bidiagonalization route of the batched SVD (K2).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mctrg {

// 1. Householder bidiagonalization  Q_L^T M Q_R = B  (upper bidiagonal) of S
//    row-major n x n matrices.  bd[s] = [d (n) | e (n, e[n-1] = 0) | tauR (n)];
//    the right reflector of step k, u_k = (1, R[k][k+2], ..., R[k][n-1]) on
//    columns k+1.., stays in row k of the working copy R = W[s] (n x n).
struct BidiagArgs {
  const double* M;   // [S][n][n] read only
  double* W;         // [S][n][n] (any row stride >= n is not supported: n x n)
  double* bd;        // [S][3n]
  int n, S;
};
cudaError_t launch_bidiag(const BidiagArgs& a, cudaStream_t st);

// 2. All singular values of each B by bisection on Sturm counts of the
//    Golub-Kahan tridiagonal; written descending into sig[S][n_pad] with
//    perm[r] = r, nnz = #{s > zero_rel s_1} (zero_rel <= 0: n 2^-52) and
//    lns1 = ln s_1 (may be null).  Values surely below the zero threshold are
//    written as 0.
cudaError_t launch_bd_bisect(const double* bd, int n, int n_pad, int S, double* sig, int* perm, int* nnz,
                             double* lns1, double zero_rel, cudaStream_t st);

// 3. Right singular vectors of the kept indices: kept[s][0..nk[s]-1] are
//    ranks (ascending, so singular values descending).  vrows[s][a][0..n-1]
//    receives s_r v_r for r = kept[s][a] (the scaling of a Jacobi row),
//    computed by inverse iteration on the Golub-Kahan tridiagonal
//    (reorthogonalized within clusters of close kept values) and the right
//    reflectors.  scratch: bd_vectors_scratch_doubles(n, S) doubles.
struct BdVecArgs {
  const double* bd;     // [S][3n]
  const double* R;      // [S][n][n] reflectors (row k holds u_k)
  const double* sig;    // [S][n_pad]
  const int* kept;      // [S][32]
  const int* nk;        // [S]
  double* vrows;        // [S][32][n]
  double* scratch;
  int n, n_pad, S;
  int unit_rows;        // 1: write v_r itself instead of s_r v_r
  int kmax;             // largest nk of the batch (<= 32)
};
cudaError_t launch_bd_vectors(const BdVecArgs& a, cudaStream_t st);
size_t bd_vectors_scratch_doubles(int n, int S);

}  // namespace mctrg
