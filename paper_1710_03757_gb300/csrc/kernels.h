// Launch interfaces of the MC-TRG device kernels (host-callable).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mctrg {

// ---- K2: batched one-sided Jacobi SVD (FP64) -------------------------------
// For S row-major n x n matrices M, orthogonalizes the rows by plane
// rotations from the left (Hestenes' one-sided Jacobi): J M = B with
// mutually orthogonal rows b_i, so M = sum_i u_i s_i v_i^T with
// s_i = |b_i|, v_i = b_i / s_i, u_i = M v_i / s_i.
struct JacobiArgs {
  const double* M;     // [S][n][n] input (read only)
  double* W;           // [S][n_pad][n] output rows b_i (unsorted)
  double* sig;         // [S][n_pad] singular values, descending
  int* perm;           // [S][n_pad] perm[r] = row of W holding the r-th largest
  double* lns1;        // [S] ln s_1 (-inf for a zero matrix); may be null
  int* nnz;            // [S] #{s_i > n 2^-52 s_1}
  uint32_t* mflags;    // [S] |= FLAG_NOCONV when the sweep cap was hit; may be null
  int n, n_pad, S;
  int max_sweeps;
  // Noise level of the arithmetic that produced M: singular values at or
  // below zero_rel * s_1 count as zeros (nnz), and rows below
  // (noise_u / 2) |M|_F are left out of the sweeps.  0 means FP64:
  // zero_rel = n 2^-52, noise_u = 2^-52.
  double zero_rel, noise_u;
};
cudaError_t launch_jacobi(const JacobiArgs& a, cudaStream_t st);

// ---- K3 + K4: stochastic truncation and split into halves -------------------
// Per item (trajectory b, tensor t of one level): choose the kept singular
// indices (all nonzero ones when there are at most chi, else a Philox-driven
// draw with p(e) ~ prod s^2), reweight by the inclusion rates, and write the
// two halves  left[row][a] = sqrt(s~_a) u_a[row],  right[a][col] = sqrt(s~_a) v_a[col]
// (zero-padded to kc columns / rows), s~ = (s / s_1) / r.
struct SampleArgs {
  const double* M;      // [slots][n][n] the matrices (distinct mode)
  const double* W;      // [slots][n_pad][n] Jacobi rows
  const double* sig;    // [slots][n_pad]
  const int* perm;      // [slots][n_pad]
  const int* nnz;       // [slots]
  const double* Urows;  // shared mode: [2][n_pad][n] unit left vectors by rank; else null
  int n, n_pad, chi, kc;
  int stochastic;       // 0: keep all nonzero values (exact level)
  int shared_svd;       // 1: slot = parity of tensor t; 0: slot = item - item0
  int64_t item0, n_items, N;   // items are b * N + t
  int L, level;
  uint64_t seed, traj0;        // trajectory counter = traj0 + b
  double* H;            // halves, item-major, stride 2 n kc: [left n x kc | right kc x n]
  int64_t h_item0;      // item index of H[0] (items below it are not stored)
  uint32_t* iflags;     // [items] |= truncation flags (indexed item - h_item0); may be null
  double* scratch;      // tables: gridDim * (n + 1) * (2 chi + 1) doubles
  // Split form (bidiagonalization route, whose vectors exist only for the kept
  // indices): mode 1 chooses and writes kept[it][kstride] (ranks, ascending),
  // sigt[it][kstride] (reweighted values s~) and nk[it], without halves; mode 2
  // reads them back and writes the halves from vrows[it][a][col] = s_r v_r[col]
  // (r = kept[it][a]) instead of W / perm.  it = item - item0.  mode 0: both.
  // kstride = kept_stride(chi) (32, or 64 above 32 kept values).
  int mode;
  int* kept;
  double* sigt;
  int* nk;
  const double* vrows;
  int kstride;
};
// chi and kc at most 64 (kKeptMax).
cudaError_t launch_sample_split(const SampleArgs& a, cudaStream_t st, int grid);
size_t sample_scratch_doubles(int n, int chi, int grid);
// CTAs of a sampler launch over n x n spectra: up to 1024, fewer when the
// tables of that many would pass 256 MB (at least 152, one per SM).
int sample_grid(int n, int chi);

// Shared mode helper: unit left vectors u_r = M v_r / s_r for r < nnz by rank.
cudaError_t launch_u_rows(const double* M, const double* W, const double* sig, const int* perm,
                          const int* nnz, double* Urows, int n, int n_pad, int S, cudaStream_t st);

// ---- K5: plaquette contraction ----------------------------------------------
// New tensor T'[al,be,de,ga] = sum_{i,j,k,m} F3[al,i,j] F4[be,k,i] F2[j,m,ga] F1[m,k,de]
// from the four parent halves, as X[(al,be)][(j,k)] = sum_i F3 F4 and
// Yt[(de,ga)][(j,k)] = sum_m F2 F1, then T' = X Yt^T.
struct XYArgs {
  const double* H;       // parent halves (level k-1), stride 2 d^2 D per item
  int64_t h_item0;       // item index of H[0]
  int d, D;              // parent leg dim, parent kept dim (= new leg dim)
  int64_t c0, n_items;   // new items c0 .. c0+n_items-1 (b * Nnew + c)
  int64_t Nnew, Nold;    // tensors per trajectory at the new / parent level
  int L, level_old;      // geometry of the parent level
  int fixed_parents;     // 1: parents are items (0,1,1,0) (shared plaquette)
  double* X;             // [n_items][D*D][d*d]
  double* Yt;            // [n_items][D*D][d*d]
};
cudaError_t launch_form_xy(const XYArgs& a, cudaStream_t st);

// M[item] = X Yt^T written in the matricized layout of the new tensor:
// parity A: M[(al,be)][(de,ga)];  B: M[(be,de)][(ga,al)];  raw = A layout.
struct GemmArgs {
  const double* X; const double* Yt;
  double* M;             // [n_items][D*D][D*D]
  int D, K;              // K = d*d
  int64_t c0, n_items, Nnew;
  int L, level_new;      // geometry for the parity of the new tensors
  int fixed_parity;      // >= 0 overrides the geometry (0 = A / raw)
};
cudaError_t launch_gemm_f64(const GemmArgs& a, cudaStream_t st);

// Final level: Tr T' = sum_{al,be} T'[al,be,al,be] = <X, Yt>; per item b:
// lnabs[b] = lnacc0 + lnacc[b] + ln|Tr|, sign[b] = sign(Tr).
cudaError_t launch_trace(const double* X, const double* Yt, int64_t K2, int64_t n_items,
                         double lnacc0, const double* lnacc, double* lnabs, int8_t* sign,
                         cudaStream_t st);

// ---- small kernels -----------------------------------------------------------
cudaError_t launch_site_tensor(double beta, double h, double* T, cudaStream_t st);
// The spins-on-bonds tensor of the paper's Fig. 1 network (D = 2).
cudaError_t launch_bond_tensor(double beta, double h, double* T, cudaStream_t st);
// A and B matricizations of a raw tensor T[l][u][r][d] (D^4): out[0] = A, out[1] = B.
// The impurity tensor (site tensor with the site's spin inserted), D = 2.
cudaError_t launch_impurity_tensor(double beta, double h, double* T, cudaStream_t st);
// Level-0 matrices [n_items][4][4] of items item0.. (b N0 + t): site t's tensor
// (Timp at imp0 / imp1, T0 elsewhere) matricized by its sublattice.
cudaError_t launch_level0_matrices(const double* T0, const double* Timp, int imp0, int imp1, int L, int64_t item0,
                                   int64_t n_items, int64_t N0, double* M, cudaStream_t st);
cudaError_t launch_matricize2(const double* T, int D, double* out, cudaStream_t st);
// lnacc[b] += sum_t ilns1[b*N+t] (if ilns1), tflags[b] |= OR_t iflags[b*N+t].
cudaError_t launch_traj_accum(const double* ilns1, const uint32_t* iflags, int64_t N, int64_t B,
                              double* lnacc, uint32_t* tflags, cudaStream_t st);
// stats = {m, sum x, sum (x - mean)^2, n_neg, n_flag, n_zero} over n results (single block).
cudaError_t launch_estimate(const double* lnabs, const int8_t* sign, const uint8_t* flags,
                            int64_t n, double* stats, cudaStream_t st);
// out[i] = f[i] | extra (f may be null: extra alone)
cudaError_t launch_flags_to_u8(const uint32_t* f, uint8_t* out, int64_t n, uint32_t extra, cudaStream_t st);

}  // namespace mctrg
