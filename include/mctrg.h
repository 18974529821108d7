/*
 * mctrg.h - C ABI of the GB300 Monte Carlo TRG library.
 *
 * The library estimates Z = Tr(N), the trace of the partition-function
 * tensor network of the 2D Ising model (Sec. IV, Eq. ising_model, extended by
 * a uniform field h), by Monte Carlo tensor-network renormalization:
 * Levin-Nave TRG (Sec. III) in which every truncated SVD keeps a random
 * subset of chi singular values drawn with probability proportional to the
 * product of their squares and reweighted by their inclusion probabilities
 * (Sec. II, Eqs. Ssum, r, w, p).  Each independent trajectory coarse-grains
 * the whole lattice, sampling every tensor independently (Sec. III), and
 * yields an unbiased sample Z~ of Z (Sec. III, Eq. infiniteEnsemble); the
 * sample mean and its standard error form the estimate (Sec. V, Eq.
 * shrunkDev).
 *
 * Conventions shared by every call:
 *  - Every function returns an int status: MCTRG_OK (0) or a negative
 *    MCTRG_E* code; mctrg_strerror() names it.  No C++ exception crosses
 *    this boundary.
 *  - A context owns its device memory (tensors, plans, scratch) and is not
 *    thread-safe: one host thread at a time per context.  A server is
 *    thread-safe.
 *  - All device work of a context runs on the stream given in
 *    mctrg_options.cuda_stream (NULL = the legacy default stream).
 *  - Trajectory i of (lattice, seed) draws its uniforms from a Philox4x32-10
 *    counter that contains first_traj + i, so it is identical whatever the
 *    batch, chunking or co-scheduled work.
 */
#ifndef MCTRG_H
#define MCTRG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define MCTRG_OK            0
#define MCTRG_EINVAL      (-1)   /* bad argument: L, chi, beta, shape, pointer */
#define MCTRG_ENOMEM      (-2)   /* footprint exceeds the HBM budget even for one trajectory, or allocation failed */
#define MCTRG_ENOCONV     (-3)   /* a Jacobi SVD hit the sweep cap; results returned, trajectories flagged */
#define MCTRG_EDOMAIN     (-4)   /* sample mean of Z~ <= 0: ln Z undefined, mean_Z_scaled still valid */
#define MCTRG_ECUDA       (-5)   /* a CUDA runtime call failed */
#define MCTRG_ESTATE      (-6)   /* call out of order (e.g. run before init) */
#define MCTRG_ETIMEDOUT   (-7)   /* server wait expired */
#define MCTRG_EAGAIN      (-8)   /* server job not finished yet */
#define MCTRG_EUNREACHABLE (-9)  /* server: target error cannot be met within max_samples */
#define MCTRG_ENOTFOUND  (-10)   /* server: unknown job id */

/* ---- per-trajectory flag bits (uint8 per trajectory) ------------------ *
 * They mark trajectories whose kept index sets can legitimately differ
 * between two correct implementations (near-ties).  They do not bias the
 * estimate; they only exclude a trajectory from per-trajectory comparisons. */
#define MCTRG_FLAG_SPLIT_CLUSTER 1u  /* kept and dropped singular values closer than 1e-8 * s_1 */
#define MCTRG_FLAG_DRAW_TIE      2u  /* a sampler uniform fell within 1e-9 (relative) of a CDF step */
#define MCTRG_FLAG_TINY_KEPT     4u  /* a kept singular value below 1e-7 * s_1 */
#define MCTRG_FLAG_NOCONV       16u  /* a Jacobi SVD of this trajectory hit the sweep cap */

/* ---- arithmetic of the contraction ------------------------------------ *
 * FP64: every step in FP64.  TF32 / BF16: the plaquette GEMM runs on the
 * tensor cores (tcgen05) with FP32 accumulation; each tensor's two operands
 * are scaled by their largest magnitude before rounding and the product is
 * scaled back (per-step scaling).  The X3 variants keep the rounding residual
 * of each operand and add the two cross products (three passes), which
 * squares the operand rounding error.  The SVD and the sampling
 * probabilities stay FP64 in every mode; at a level whose matrices come from
 * the tensor cores, singular values below min(sqrt(n) u, 1/64) s_1 (u the
 * operand unit roundoff of the mode) are that arithmetic's noise and count
 * as zeros.  Levels whose GEMM shape the tensor-core kernel does not cover
 * (matrix side not a multiple of 256, or above 1024) use the FP64 GEMM and
 * the FP64 threshold. */
/* FP64TC: the plaquette GEMM at FP64 accuracy on the tensor cores: each row
 * of X and Yt is scaled by a power of two and split exactly into s BF16
 * slices of b bits (b = 8, s = 7 for inner dimension K <= 256; b = 7, s = 8
 * up to 1024), the s(s+1)/2 leading slice products are formed exactly by
 * tcgen05 (one FP32 accumulator per slice-sum group, exact below 2^24) and
 * summed in FP64 (Ozaki, Ogita, Oishi and Rump 2012).  The result carries an
 * error below 2^-43 K |row max| |column max|, the order of an FP64 dot
 * product's, so the FP64 zero threshold applies.  Levels whose inner
 * dimension is not a multiple of 64 up to 1024 use the FP64 GEMM. */
typedef enum { MCTRG_FP64 = 0, MCTRG_TF32 = 1, MCTRG_BF16 = 2, MCTRG_TF32X3 = 3, MCTRG_BF16X3 = 4,
               MCTRG_FP64TC = 5 } mctrg_precision;

typedef struct {
    int device;               /* CUDA device ordinal                                   */
    void* cuda_stream;        /* cudaStream_t for all work of the context; NULL = default */
    int precision;            /* mctrg_precision                                       */
    size_t hbm_budget_bytes;  /* device memory the context may hold; 0 = 80% of free   */
    int max_sweeps;           /* Jacobi sweep cap; 0 = 40                              */
    int max_chunk;            /* max trajectories per device chunk; 0 = automatic      */
    int profile;              /* 1: time every kernel launch with CUDA events on the
                                 context's stream (see mctrg_kernel_stats)             */
    int svd;                  /* mctrg_svd_route of the per-trajectory SVDs            */
    double zero_tol_scale;    /* multiplies the zero threshold of every SVD: singular
                                 values at or below scale * tau count as zeros
                                 (Sec. II samples among the nonzero values; tau is
                                 n 2^-52 s_1 in FP64, see mctrg_precision for the
                                 mixed modes); 0 = 1, negative or non-finite: EINVAL */
    int deterministic_levels; /* levels 0 .. deterministic_levels-1 keep the chi largest
                                 singular values with weight 1 instead of sampling
                                 (Sec. II, Eq. approxSVD: plain TRG); sampling starts
                                 at the next level whose spectrum has more than chi
                                 nonzero values.  While the network is translation
                                 invariant these levels cost one split per
                                 sublattice (Sec. III).  0 = Monte Carlo TRG from
                                 the start; a value >= 2 log2 L runs deterministic
                                 TRG, every trajectory identical; in between, the
                                 hybrid of Sec. V (deterministic coarse-graining
                                 steps, then Monte Carlo), whose trajectories are
                                 unbiased samples of the trace of the network after
                                 those levels.  A kept and a dropped value closer
                                 than 1e-8 s_1 set MCTRG_FLAG_SPLIT_CLUSTER in every
                                 trajectory.  Negative: EINVAL */
    const char* autotune_cache; /* mctrg_batch_run: file of the launch geometry chosen
                                 per matrix shape (read, and written when new shapes
                                 were timed); NULL = choose every run, keep nothing */
} mctrg_options;

/* Route of the per-trajectory SVDs (Sec. II, Eq. exactSVD), all with the
 * absolute accuracy of a backward-stable FP64 SVD (a few eps |M|):
 *   JACOBI  QR with column pivoting, then one-sided Jacobi on the rows; its
 *           cost follows the numerical rank.
 *   BIDIAG  Householder bidiagonalization, every singular value by bisection
 *           on Sturm counts of the Golub-Kahan tridiagonal, and right vectors
 *           of the kept indices only (inverse iteration, back-transformation);
 *           (8/3) n^3 + O(n^2) flops whatever the rank.
 *   AUTO    BIDIAG where the matrices can have full rank (n >= 64 and the
 *           plaquette's inner dimension d^2 >= n / 2), JACOBI elsewhere.
 *   BAND    AUTO's choice, with the two-stage route in place of BIDIAG where
 *           n is a multiple of 8 from 64 to 256 (chi <= 16): the reduction's
 *           (8/3) n^3 flops as exact integer products of 8-bit digit slices
 *           on the tensor cores, O(n^2) FP64 work per matrix beside them
 *           (mctrg_svd_band_batched).  Not taken by mctrg_batch_run (EINVAL).
 * JACOBI covers n <= 1024: levels with larger matrices (n up to 2304, chi up
 * to 48) take BIDIAG whatever the option. */
typedef enum { MCTRG_SVD_AUTO = 0, MCTRG_SVD_JACOBI = 1, MCTRG_SVD_BIDIAG = 2, MCTRG_SVD_BAND = 3 } mctrg_svd_route;

/* Estimate of Z from n trajectories (Sec. III Eq. infiniteEnsemble, Sec. V Eq.
 * shrunkDev).  With m = ln_scale = max_i ln|Z~_i| and x_i = sign_i e^{ln|Z~_i| - m}:
 *   mean_Z_scaled = mean(x),  se_Z_scaled = std(x) / sqrt(n)   (Z^ = e^m mean(x)),
 *   ln_mean_Z = m + ln mean(x),  se_ln_Z = se_Z_scaled / mean_Z_scaled,
 *   ess = (sum x)^2 / sum x^2.
 * sum_x = sum_i x_i and m2_x = sum_i (x_i - mean(x))^2, both at scale m,
 * are the sufficient statistics that mctrg_merge_estimates combines
 * (pairwise update of Chan, Golub and LeVeque). */
typedef struct {
    int64_t n;
    double ln_mean_Z;
    double se_ln_Z;
    double mean_Z_scaled;
    double se_Z_scaled;
    double ln_scale;
    double ess;
    int64_t n_negative;
    int64_t n_flagged;
    double sum_x;
    double m2_x;
    int status;               /* MCTRG_OK, MCTRG_EDOMAIN or MCTRG_ENOCONV */
} mctrg_estimate;

typedef struct mctrg_ctx* mctrg_ctx_t;

/* Fill *opt with defaults (device 0, default stream, FP64, automatic budget). */
int mctrg_options_default(mctrg_options* opt);

/* Create a context on opt->device.  *out receives the handle.  Errors:
 * EINVAL (NULL pointer, bad precision), ECUDA (device unusable). */
int mctrg_create(const mctrg_options* opt, mctrg_ctx_t* out);

/* Set up an L x L periodic Ising lattice at inverse temperature beta >= 0 and
 * field h (Sec. IV), truncating every SVD to chi kept singular values
 * (Sec. II).  L must be a power of two, 2 <= L <= 65536; 1 <= chi <= 48.
 * The site tensor is T[l,u,r,d] = sum_s e^{beta h s} W[s,l] W[s,u] W[s,r] W[s,d]
 * with W[s,0] = sqrt(cosh beta), W[s,1] = s sqrt(sinh beta).  Runs the shared
 * deterministic prefix (levels where nothing is sampled, and the one SVD of
 * the first sampled level) on the device; blocks until it is done.
 * Errors: EINVAL, ENOMEM, ECUDA. */
int mctrg_init_lattice(mctrg_ctx_t ctx, double beta, double h, int L, int chi);

/* The paper's own lattice (Sec. IV, Fig. 1): the Ising spins live on the
 * bonds of the L x L tensor network (2 L^2 spins on a 45-degree rotated
 * periodic square lattice; L = 8 is the paper's 128-spin network, six
 * coarse-graining steps).  The tensor holds the four bonds around a plaquette:
 * T[l,u,r,d] = exp(beta (s_l s_u + s_u s_r + s_r s_d + s_d s_l)
 *                  + beta h (s_l + s_u + s_r + s_d) / 2), index 0 = spin +1.
 * Arguments, limits and errors as mctrg_init_lattice. */
int mctrg_init_bond_lattice(mctrg_ctx_t ctx, double beta, double h, int L, int chi);

/* Observables by impurity tensors (Sec. III: the method applies to partial
 * traces as to Z).  The lattice of mctrg_init_lattice with the tensor of site
 * (0, 0) -- and of its right neighbour (1, 0) when n_imp = 2 -- replaced by
 * the site tensor with the site's spin inserted,
 *   T_imp[l,u,r,d] = sum_s s e^{beta h s} W[s,l] W[s,u] W[s,r] W[s,d],
 * so that every trajectory is an unbiased sample of Z <sigma_00> (n_imp = 1)
 * or of Z <sigma_00 sigma_10> (n_imp = 2, the bond energy); signs are tracked
 * as for Z.  The network is not translation invariant, so every level is
 * split tensor by tensor from level 0 (leg dimensions min(chi, D^2) from
 * D = 2, no shared prefix).  Divide by an estimate of Z with
 * mctrg_ratio_estimate.  n_imp is 1 or 2; deterministic_levels must be 0.
 * Errors: EINVAL, ECUDA. */
int mctrg_init_impurity(mctrg_ctx_t ctx, double beta, double h, int L, int chi, int n_imp);

/* Ratio of the means of two estimates from independent trajectory sets
 * (e.g. Z <sigma> over Z), and its standard error by first-order error
 * propagation (sum of the squared relative errors; an exactly zero numerator
 * mean takes its own spread).  Host only.  Errors: EINVAL (n < 2), EDOMAIN
 * (denominator mean <= 0). */
int mctrg_ratio_estimate(const mctrg_estimate* num, const mctrg_estimate* den, double* ratio, double* se);

/* Monte Carlo HOTRG: the stochastic truncation of Sec. II on the higher-order
 * TRG (Xie et al. 2012), one of the other SVD-based coarse-graining schemes
 * to which Secs. III and V say the method extends.  A step merges pairs of
 * rows: T(x,2j) over T(x,2j+1), contracted over their vertical bond, gives
 * M(x,j) with horizontal legs of dimension Dh^2.  Every merged horizontal
 * bond gets its own random projector P~ = sum_{i in e} u_i u_i^T / r_i from
 * the eigenpairs (u_i, lambda_i) of the Gram matrix of M(x,j)'s right
 * unfolding: e is a chi-subset of the nonzero eigenvalues (above n 2^-52
 * lambda_1) drawn with p(e) ~ prod lambda_i, r_i its inclusion rates, so
 * E[P~] is the identity on all that M(x,j) sees and every trajectory is an
 * unbiased sample of Z (sign tracked).  The new tensor is
 * U~_left^T M U~_right (U~ = [u_i / sqrt(r_i)]) divided by sqrt(lambda_1) of
 * its right bond; the lattice is then reflected across its diagonal, so after
 * 2 log2 L steps one tensor is left and traced.  Trajectory i draws its
 * uniforms from Philox4x32-10 under seed with counter (t >> 1, bond, step,
 * first_traj + i), bond = j Lx + x.
 * T0: NULL for the Ising site tensor at (beta, h) (that of mctrg_init_lattice),
 * else a host pointer to D^4 doubles [l][u][r][d], 2 <= D <= 8 (beta, h
 * ignored).  L a power of two, 2 <= L <= 4096; 2 <= chi <= 32.  opt: device,
 * cuda_stream, hbm_budget_bytes (0: 70% of the free memory), max_chunk (> 0:
 * at most that many trajectories at once).  Outputs as mctrg_run (each host
 * or device memory, NULL to skip; est required).  Allocates its working
 * memory and frees it before returning; blocks until done.  Returns OK,
 * EDOMAIN (mean <= 0), EINVAL, ENOMEM, ECUDA. */
int mctrg_hotrg_run(const mctrg_options* opt, double beta, double h, const double* T0, int D, int L, int chi,
                    int64_t n_samples, uint64_t seed, uint64_t first_traj, double* lnabsZ, int8_t* sign,
                    uint8_t* flags, mctrg_estimate* est);

/* Same as mctrg_init_lattice with an arbitrary site tensor T0 (host pointer,
 * D^4 doubles, index order [l][u][r][d], row-major), 1 <= D <= 8, copied. */
int mctrg_init_tensor(mctrg_ctx_t ctx, const double* T0, int D, int L, int chi);

/* Run n_samples >= 1 trajectories with counters first_traj .. first_traj+n-1
 * (first_traj + n_samples <= 2^32) under a 64-bit seed.
 * Outputs (caller-owned, each host or device memory, detected per pointer;
 * NULL to skip): lnabsZ[n] = ln|Z~_i| (-inf when Z~_i = 0), sign[n] in
 * {-1, 0, +1}, flags[n] = MCTRG_FLAG_* bits.  est (required, host) receives
 * the estimate.  Blocks until the results are written.  Returns OK,
 * EDOMAIN (mean <= 0), ENOCONV (some SVD hit the sweep cap), or an error. */
int mctrg_run(mctrg_ctx_t ctx, int64_t n_samples, uint64_t seed, uint64_t first_traj,
              double* lnabsZ, int8_t* sign, uint8_t* flags, mctrg_estimate* est);

/* Device bytes the context would hold to run n_samples trajectories in the
 * chunking it would choose (*bytes), after init.  Errors: ESTATE, EINVAL. */
int mctrg_footprint(mctrg_ctx_t ctx, int64_t n_samples, size_t* bytes);

/* Combine k >= 1 estimates of disjoint trajectory ranges of one lattice and
 * seed into *out by rescaling their sufficient statistics to a common scale
 * (host only; the replicas-only multi-GPU merge). */
int mctrg_merge_estimates(const mctrg_estimate* parts, int k, mctrg_estimate* out);

/* ---- per-kernel statistics (profiling option) -------------------------- *
 * With mctrg_options.profile = 1, every launch of the hot-path kernels is
 * bracketed by CUDA events on the context's stream and accumulated per
 * kernel class since the last reset.  flops_alg is the algorithmic work of
 * the launches (not the instructions executed):
 *   JACOBI   (8/3) n^3 + 4 n^2 kc per matrix (SVD floor: bidiagonal reduction
 *            for all singular values plus the kept singular vectors)
 *   GEMM     2 n^2 d^2 per tensor (n = D^2 rows/cols, d^2 inner)
 *   FORM_XY  4 D^2 d^3 per tensor
 *   SAMPLE   4 n kc + 2 n^2 kc per tensor (tables and draws; left halves M v)
 *   TRACE    2 D^2 d^2 per trajectory
 *   BIDIAG   (8/3) n^3 per matrix (Householder bidiagonalization)
 *   BISECT   no flop count is recorded: each nonzero value takes ~20 FP32 and
 *            ~6 FP64 Sturm counts of 2n steps (2 FP64 operations per step)
 *   VECTORS  2 n^2 kc + 20 (2n) kc per matrix (back-transformation and
 *            inverse iteration of the kept vectors; 4 n^2 kc on the BAND route,
 *            whose vectors pass back through both stages)
 *   BAND     (8/3) n^3 per matrix (the dense -> band reduction of the BAND
 *            route: tensor-core products and FP64 panel factorizations)
 *   CHASE    6 b n^2 per matrix, b = 8 (band -> bidiagonal bulge chase)
 * bytes_alg counts each kernel's compulsory global-memory traffic
 * (inputs read once, outputs written once). */
enum { MCTRG_K_FORM_XY = 0, MCTRG_K_GEMM = 1, MCTRG_K_JACOBI = 2, MCTRG_K_SAMPLE = 3,
       MCTRG_K_TRACE = 4, MCTRG_K_OTHER = 5, MCTRG_K_BIDIAG = 6, MCTRG_K_BISECT = 7,
       MCTRG_K_VECTORS = 8, MCTRG_K_BAND = 9, MCTRG_K_CHASE = 10, MCTRG_K_COUNT = 11 };
typedef struct {
    int64_t launches;
    double ms;          /* summed event-timed duration */
    int64_t items;      /* matrices / tensors / trajectories processed */
    double flops_alg;
    double bytes_alg;
} mctrg_kernel_stat;

/* Statistics of kernel class `kernel` (MCTRG_K_*) since the last reset.
 * Errors: EINVAL (bad class), ESTATE (profiling off). */
int mctrg_kernel_stats(mctrg_ctx_t ctx, int kernel, mctrg_kernel_stat* out);
int mctrg_reset_kernel_stats(mctrg_ctx_t ctx);

/* ---- batching: uneven jobs in one run ----------------------------------- *
 * A job of a batch: lattice (Sec. IV, the site tensor of mctrg_init_lattice),
 * bond dimension, n_samples trajectories with counters first_traj ..
 * first_traj + n_samples - 1 under seed. */
typedef struct {
    double beta, h;
    int L, chi;
    int64_t n_samples;
    uint64_t seed;
    uint64_t first_traj;
} mctrg_job;

/* Run n_jobs >= 1 jobs of uneven L and chi together on opt->device and
 * opt->cuda_stream (precision MCTRG_FP64 or MCTRG_FP64TC; the other options
 * as for mctrg_create).  The jobs' levels advance together in sub-batches:
 * per job the geometry-dependent kernels (plaquette operands, contraction,
 * choice of the kept indices, halves), and one launch per stage of the
 * bidiagonalization-route SVD (Householder reduction, bisection, kept
 * vectors) over the matrices of every job, of whatever size.  The number of
 * matrices per SVD launch for each matrix shape and the sampler's CTA count
 * are launch geometry with identical arithmetic, chosen by timing
 * candidates on the device and kept in opt->autotune_cache.  Job j's
 * results are those of mctrg_run with the same lattice, seed and counters,
 * bit for bit.  Outputs: est[j] (host, required); lnabsZ, sign, flags
 * (nullable, host or device) receive the jobs' per-trajectory results one
 * after the other (job 0's n_samples first).  The paper has no counterpart
 * (it runs one lattice at a time).  Blocks until done.  Errors: EINVAL,
 * ENOMEM (the jobs' own buffers and one item of the largest shape do not
 * fit), ECUDA; a job's estimate carries EDOMAIN or ENOCONV in its status. */
int mctrg_batch_run(const mctrg_options* opt, const mctrg_job* jobs, int n_jobs, mctrg_estimate* est,
                    double* lnabsZ, int8_t* sign, uint8_t* flags);

/* ---- the batched SVD on its own ------------------------------------------ *
 * Singular values, and optionally right singular vectors, of `batch` row-major
 * n x n FP64 matrices by the library's batched one-sided Jacobi SVD (the full
 * SVD of Sec. II, Eq. exactSVD, that every tensor of a trajectory goes
 * through).  M (device, batch*n*n) is read only.  sigma (device, batch*n)
 * receives the singular values in descending order; vt (device, batch*n*n,
 * may be NULL) receives the right singular vectors as rows in the same order
 * (zero rows for singular values that are exactly zero).  1 <= n <= 1024,
 * batch >= 1, max_sweeps <= 0 means 40.  Allocates its working rows on the
 * device for the call and frees them; runs on `stream` (cudaStream_t, NULL =
 * default) and returns once the stream has completed.
 * Errors: EINVAL, ENOMEM, ECUDA, ENOCONV (a matrix hit the sweep cap; results
 * still written). */
int mctrg_svd_batched(const double* M, int n, int64_t batch, double* sigma, double* vt,
                      int max_sweeps, void* stream);

/* The same batched SVD for callers that cannot allocate device memory.
 * There is no counterpart in the paper: it exists for callers such as a
 * program whose device memory belongs to another allocator (for example a
 * framework's caching allocator holding nearly all of it), a loop that must
 * never stall the device (cudaFree, which mctrg_svd_batched calls, waits for
 * the whole device), or code that may not call an allocator at all.
 * Arguments and results are those of mctrg_svd_batched; the caller still
 * provides M, sigma and vt.  The working memory is one fixed 16 MiB array
 * compiled into the library, which every device that loads the library holds
 * until the process exits; no allocation or free of any kind happens.
 * n may be at most MCTRG_SVD_NOALLOC_MAX_N (larger n returns MCTRG_EINVAL);
 * any batch size works (the batch is processed in pieces that fit).
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.  Every call
 * reuses the same array and its flag word is cleared at the start of each
 * call; two calls whose work overlapped on the device would race, so calls
 * from one process are serialized and each returns only after `stream` has
 * completed, also when it fails after queueing work.  The array and that
 * serialization are per process and per device: another process (or another
 * loaded copy of the library) has its own array and is not serialized
 * against this one.  `stream` must belong to the current device.
 * Errors: EINVAL, ECUDA, ENOCONV. */
#define MCTRG_SVD_NOALLOC_MAX_N 1024
int mctrg_svd_batched_noalloc(const double* M, int n, int64_t batch, double* sigma, double* vt,
                              int max_sweeps, void* stream);

/* ---- the plaquette contraction on its own ------------------------------ *
 * The coarse-graining step's contraction (Sec. III; Levin-Nave plaquette)
 * ends in one matrix product per new tensor, M = X Yt^T; this runs it for a
 * batch: X, Yt (device, batch x n x K, row-major, n = D^2) and M (device,
 * batch x n x n, row-major; written, not accumulated).  precision:
 * MCTRG_FP64 (FP64 on the CUDA cores) or MCTRG_FP64TC (BF16 slices on the
 * tensor cores, FP64-accurate; K a multiple of 64, at most 1024).  1 <= D,
 * n <= 1024, K >= 1, batch >= 1.  Allocates its working memory (FP64TC: the
 * slice planes and row exponents) for the call and frees it; runs on
 * `stream` and returns once the stream has completed.  Errors: EINVAL,
 * ENOMEM, ECUDA. */
int mctrg_contract_batched(const double* X, const double* Yt, int D, int K, int64_t batch, double* M,
                           int precision, void* stream);

/* The bidiagonalization route of the same SVD on its own (the route
 * MCTRG_SVD_BIDIAG of the contexts): Householder bidiagonalization, every
 * singular value by bisection on Sturm counts of the Golub-Kahan tridiagonal,
 * and the right vectors of the n_vec largest singular values by inverse
 * iteration and back-transformation.  M (device, batch*n*n, row-major) is read
 * only; sigma (device, batch*n) receives the singular values in descending
 * order (values below n 2^-52 max_ij |B_ij|, B the bidiagonal, are 0);
 * vt (device, batch*n_vec*n; NULL when n_vec = 0) receives unit right vectors
 * as rows.  Each value carries an absolute error of a few 2^-52 |M|; vectors
 * of values closer than 1e-3 |M| to another are an orthonormal basis of their
 * cluster's subspace; vectors of values at the noise level (a few 2^-52 n |M|
 * and below: the numerical null space) are not determined and carry no
 * guarantee.  Allocates and frees its working memory.
 * 2 <= n <= 2304, 0 <= n_vec <= min(64, n).  Errors: EINVAL, ENOMEM, ECUDA. */
int mctrg_svd_bidiag_batched(const double* M, int n, int64_t batch, double* sigma, int n_vec,
                             double* vt, void* stream);

/* The two-stage (band) route of the same SVD on its own (the route
 * MCTRG_SVD_BAND of the contexts).  Sec. II asks only for the SVD of each
 * matricization; this route computes it with the reduction's flops on the
 * tensor cores: M is reduced to an upper band with 8 superdiagonals in
 * panels of 8 columns (QR of each column panel and LQ of its row panel in
 * FP64; the products with the trailing matrix, and its two-sided update, as
 * exact integer products of 8-bit digit slices on the tensor cores, the
 * trailing matrix held in 59-bit fixed point relative to |M|_F), the band is
 * reduced to bidiagonal form by bulge chasing (FP64), and the singular values
 * and right vectors follow as in mctrg_svd_bidiag_batched (bisection,
 * inverse iteration, and the two stages' right reflectors applied back).
 * Arguments, layouts, accuracy and ownership as mctrg_svd_bidiag_batched;
 * n a multiple of 8 with 64 <= n <= 256, 0 <= n_vec <= 16.  The fixed point
 * is set from |M|_F computed in FP64, so the entries must keep their squares
 * in range: a matrix whose squared entries all underflow (every |M_ij| below
 * about 1e-154) is treated as zero, and one with entries above about 1e154
 * is not supported; the level matrices of a context are normalized and never
 * come near either.
 * Errors: EINVAL, ENOMEM, ECUDA (also when a tensor-core kernel's bounded
 * wait expired). */
int mctrg_svd_band_batched(const double* M, int n, int64_t batch, double* sigma, int n_vec,
                           double* vt, void* stream);

/* The band route's reductions alone, for inspection: band (device,
 * batch*n*9) receives the upper band B(i, i+o), o = 0..8 (entries beyond
 * column n-1 undefined), an orthogonal two-sided transformation of M; bd
 * (device, batch*3n, or NULL to stop after the band) the diagonal d (n) and
 * superdiagonal e (n, e[n-1] = 0) of the bidiagonal the bulge chase reaches,
 * then n zeros.  The paper has no counterpart (the steps of an SVD).  n and
 * batch as mctrg_svd_band_batched.  Allocates and frees its working memory.
 * Errors: EINVAL, ENOMEM, ECUDA. */
int mctrg_band_reduce_batched(const double* M, int n, int64_t batch, double* band, double* bd, void* stream);

/* ---- measurement ------------------------------------------------------ *
 * FP64 arithmetic rate of a device, the peak against which the FP64 kernels
 * (the SVD routes, the FP64 contraction) are quoted: a probe kernel runs, in
 * every thread of a whole number of CTAs per SM, 4, 8 or 16 independent
 * chains of about `steps` fused multiply-adds (x <- x b + c), or a 4 x 4
 * outer product of changing operands per step (16 fused multiply-adds), at
 * 128, 256 and 512 threads per CTA; for each shape one untimed launch, then three launches
 * timed with CUDA events on the legacy default stream.  *tflops = the best
 * rate (2 flops per step and chain); *ms (may be NULL) receives that launch's
 * duration.  The paper has no counterpart (it reports no timings).
 * steps >= 16.  Errors: EINVAL, ECUDA. */
int mctrg_measure_fp64_peak(int device, int64_t steps, double* tflops, double* ms);

/* Release every resource of the context (NULL is a no-op). */
void mctrg_destroy(mctrg_ctx_t ctx);

/* Static string naming a status code. */
const char* mctrg_strerror(int status);

/* ---- serving: continuous batching of estimate jobs -------------------- *
 * A server owns one device, a device-memory budget (hbm_budget_bytes of the
 * options; 0 = 80% of the free memory) and 16 workers (slots), each with its
 * own stream and a persistent context.  Jobs (beta, h, L, chi, target
 * standard error of ln Z) arrive with mctrg_server_submit at any time and
 * are admitted by HBM footprint: a free worker takes the oldest queued job
 * whose footprint (the memory plan of its largest round of trajectories,
 * bounded from the largest leg dimensions the lattice can have; see
 * mctrg_server_footprint) fits the budget that running and idle workers do
 * not hold; a job passed over 32 times for later, smaller ones blocks the
 * queue until memory frees.  Workers keep their buffers between jobs and
 * give them back only when a queued job is blocked on memory.  A job
 * advances in rounds of trajectories (the first about half a second of SVD
 * work, from the n^3 of the lattice's levels: 2 to 256 trajectories;
 * doubling up to 8192); after each round it stops when its standard error
 * of ln Z reaches the target, or when that error projected to max_samples by
 * the 1/sqrt(N) law (Sec. V, Eq. shrunkDev) exceeds twice the target
 * (EUNREACHABLE; a merged mean Z~ <= 0 or a non-finite error counts as
 * unbounded), or when max_samples is spent.
 * The kernels of all running jobs share the device on their streams.
 * Trajectory i of a job uses counter i under the job's seed, so its result
 * is the same alone and in any mix. */
typedef struct mctrg_server* mctrg_server_t;

int mctrg_server_create(const mctrg_options* opt, mctrg_server_t* out);
/* Non-blocking.  target_se_lnZ >= 0 (0: a fixed-sample job that runs exactly
 * max_samples trajectories, no early stop); max_samples >= 1.  Returns
 * EUNREACHABLE at once when even one trajectory of the job cannot fit the
 * server's budget. */
int mctrg_server_submit(mctrg_server_t srv, double beta, double h, int L, int chi,
                        double target_se_lnZ, int64_t max_samples, uint64_t seed,
                        uint64_t* job_id);
/* EAGAIN until the job is done; then fills *est and *latency_s (submit to
 * completion, seconds) and forgets the job.  Returns OK when the target error
 * was reached, EUNREACHABLE (est still filled) when it was projected out of
 * reach or max_samples ran out first. */
int mctrg_server_poll(mctrg_server_t srv, uint64_t job_id, mctrg_estimate* est, double* latency_s);
/* Blocks up to timeout_s; ETIMEDOUT if the job is still running. */
int mctrg_server_wait(mctrg_server_t srv, uint64_t job_id, double timeout_s,
                      mctrg_estimate* est, double* latency_s);
/* Device bytes a job (L, chi, max_samples) would be admitted with (*bytes);
 * EUNREACHABLE when not even one trajectory fits the budget. */
int mctrg_server_footprint(mctrg_server_t srv, int L, int chi, int64_t max_samples, size_t* bytes);
/* The server's budget and the bytes its workers hold now (either may be NULL). */
int mctrg_server_memory(mctrg_server_t srv, size_t* budget, size_t* reserved);
void mctrg_server_destroy(mctrg_server_t srv);

#ifdef __cplusplus
}
#endif
#endif /* MCTRG_H */
