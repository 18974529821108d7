// K2, two-stage route: the SVD of a level matrix (Sec. II, Eq. exactSVD) with
// most of its reduction on the tensor cores.  GB300 issues FP64 at 2 lanes
// per clock per SM; the one-stage bidiagonalization spends (8/3) n^3 flops
// there.  This route splits the reduction in two (the successive band
// reduction of Bischof, Lang and Sun, 2000):
//
//  1. dense -> upper band with b = 8 superdiagonals, in panels of b columns.
//     Panel k: Householder QR of the column panel (FP64, k_band_qr), the
//     product W = V^T A of its reflectors with the trailing matrix
//     (k_band_gemm_w), the row panel updated and reduced by an LQ
//     factorization (k_band_lq), the product X = A U^T with the LQ reflectors
//     (k_band_gemm_x), and the two-sided trailing update
//     A <- A - [V | Y] [Z ; U], Z = T^T W, Y = (X - V Z U^T) T_U (k_band_update).
//     The three products carry the (8/3) n^3 flops.  They run as exact
//     integer products on the tensor cores: the trailing matrix is held in
//     59-bit fixed point (int64 relative to 2^e > |A|_F; orthogonal updates
//     keep every entry below |A|_F), the FP64 operands (V, U, Y, Z) in 62-bit
//     fixed point relative to their own row or column exponent, each operand
//     split into eight signed 8-bit digits stored as BF16 (exact), and the
//     digit products with i + j <= 7 accumulated by tcgen05.mma in tensor
//     memory, one FP32 accumulator per digit group g = i + j (Ozaki, Ogita,
//     Oishi and Rump 2012; sums of up to 256 products of 8-bit digits are
//     integers below 2^24 for the leading groups, so FP32 holds them
//     exactly).  The update is applied in integer arithmetic, so apart from
//     the panel factorizations stage 1 issues no FP64 instruction per
//     trailing element.
//  2. band -> bidiagonal by bulge chasing (k_band_chase, one warp per matrix,
//     the band in shared memory): per sweep i a right reflector clears row i
//     beyond the superdiagonal, and alternating left and right reflectors of
//     length <= b chase the bulge it creates down the band (LAPACK's dgbbrd
//     does this with Givens rotations; Householder reflectors here).
//     O(n^2 b) FP64 flops.
//  Then the bisection of the bidiagonalization route gives the singular
//  values, its inverse iteration the kept right vectors of the bidiagonal,
//  and k_band_backtr applies the chase's and the panels' right reflectors to
//  them, v = P1 P2 v_B.
//
// Every mbarrier wait is bounded; on expiry a kernel records an error word
// and skips its output, and frees its tensor memory.
#include <cuda_bf16.h>

#include <cstdint>

#include "common.cuh"
#include "kernels_band.h"
#include "tc_ptx.cuh"

namespace mctrg {

using namespace tcptx;

namespace {
constexpr int B = kBandW;        // band width / panel width
constexpr int kSl = 8;           // digit slices per operand
constexpr int kFixBits = 59;     // fixed-point fraction bits of the trailing matrix
constexpr int kFloatP = 62;      // fixed-point bits of an FP64 operand below 2^e
constexpr int kZeroExp = -1100;  // exponent of an all-zero row or column
constexpr int kWin = 24;         // chase window: offsets c - r in [-7, 15] (+1 pad)
constexpr int kTileM = 128;      // rows of an MMA tile (tensor-memory lanes)
constexpr uint32_t kTileBytes = 128u * 128u;   // 128 rows x 128 bytes (4 slices x 16 K)

// Doubles of one matrix's panel scratch.
__host__ __device__ __forceinline__ size_t work_stride(int n) { return (size_t)26 * n + 128; }

// Per-matrix panel scratch, in doubles.
struct Work {
  double* V;    // [n][8]  reflectors of the column panel, rows relative to k
  double* T;    // [64]    their T factor (upper triangular)
  double* Z;    // [8][n]  W = V^T A, then Z = T^T W (columns relative to k+b)
  double* ZU;   // [64]    Z U^T
  double* Y;    // [n][8]  rows relative to k+b
  int* el;      // [n]     row exponents of [V | Y]
  int* er;      // [n]     column exponents of [Z ; U]
};
__device__ __forceinline__ Work work_of(double* base, int n) {
  Work w;
  w.V = base;
  w.T = w.V + (size_t)n * 8;
  w.Z = w.T + 64;
  w.ZU = w.Z + (size_t)8 * n;
  w.Y = w.ZU + 64;
  w.el = (int*)(w.Y + (size_t)n * 8);
  w.er = (int*)(w.Y + (size_t)n * 9);
  return w;
}

// 2^p as a double, from exponent bits (beyond the normal range a product of
// two powers, which underflows or overflows as the scaling would).
__device__ __forceinline__ double p2(int p) {
  if (p >= -1022 && p <= 1023) return __hiloint2double((1023 + p) << 20, 0);
  p = max(-2044, min(2046, p));
  const int h = p / 2;
  return __hiloint2double((1023 + h) << 20, 0) * __hiloint2double((1023 + (p - h)) << 20, 0);
}

// round(x 2^sh) as an integer from the bits of x (no FP64 instruction); the
// caller keeps the result below 2^62.
__device__ __forceinline__ long long fix_of(double x, int sh_total) {
  const long long b = __double_as_longlong(x);
  const int be = (int)((b >> 52) & 0x7ff);
  const long long q = (b & 0xFFFFFFFFFFFFFll) | (be ? (1ll << 52) : 0ll);
  const int sh = (be ? be - 1075 : -1074) + sh_total;
  long long F;
  if (sh >= 0) F = q << sh;
  else if (sh > -62) F = (q + (1ll << (-sh - 1))) >> (-sh);
  else F = 0;
  return b < 0 ? -F : F;
}

// Exponent e with |x| < 2^e for the largest magnitude x (kZeroExp for 0).
__device__ __forceinline__ int exp_above(double amax) {
  const int be = (__double2hiint(amax) >> 20) & 0x7ff;
  if (amax == 0.0) return kZeroExp;
  return be ? be - 1022 : -1022;
}

// The eight balanced 8-bit digits of each of eight integers (|x| < 2^63 -
// 2^62), as BF16 (exact), packed per slice: out[s] holds slice s (s = 0 the
// top digit) of x[0..7].  Adding 0x80 to every byte turns the balanced digits
// into the plain bytes of one 64-bit sum, so each digit costs a byte permute
// and an FP32 subtraction.
__device__ __forceinline__ void digits8(const long long (&x)[8], uint4 (&out)[kSl]) {
  uint32_t lo[8], hi[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const unsigned long long y = (unsigned long long)x[e] + 0x8080808080808080ull;
    lo[e] = (uint32_t)y;
    hi[e] = (uint32_t)(y >> 32);
  }
#pragma unroll
  for (int s = 0; s < kSl; ++s) {
    const int bi = 7 - s;                       // byte of the digit, 7 = top
    uint32_t f[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const uint32_t w = bi >= 4 ? hi[e] : lo[e];
      const float v = __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7440u | (uint32_t)(bi & 3))) - 8388736.0f;
      f[e] = __float_as_uint(v);
    }
    out[s].x = __byte_perm(f[0], f[1], 0x7632);
    out[s].y = __byte_perm(f[2], f[3], 0x7632);
    out[s].z = __byte_perm(f[4], f[5], 0x7632);
    out[s].w = __byte_perm(f[6], f[7], 0x7632);
  }
}

// Store the slices of eight consecutive K values (k-step q, half kh = K/8 & 1)
// of row rho into the slice tiles at `tiles` (per k-step two 16 KB tiles of
// 128 rows x 128 bytes, 4 slices side by side in the 128-byte swizzle).
__device__ __forceinline__ void store_slices(uint8_t* tiles, uint32_t tile_bytes, int q, int kh, int rho,
                                             const uint4 (&d)[kSl]) {
#pragma unroll
  for (int s = 0; s < kSl; ++s) {
    uint8_t* t = tiles + (size_t)(q * 2 + (s >> 2)) * tile_bytes;
    const int chunk = (((s & 3) << 1) | kh) ^ (rho & 7);
    *(uint4*)(t + rho * 128 + chunk * 16) = d[s];
  }
}

// The 36 products of a k-step: accumulator g = i + j at columns g * N.  Two
// descriptors are formed per call; each product's start addresses differ from
// them by compile-time offsets (the 14-bit start field holds address / 16).
__device__ __forceinline__ void issue_products(uint32_t tmem, const uint8_t* A, uint32_t abytes, const uint8_t* Bt,
                                               uint32_t bbytes, int q, int N, uint32_t idesc, bool first) {
  const uint64_t a0 = umma_desc(smem_u32(A + (size_t)q * 2 * abytes));
  const uint64_t b0 = umma_desc(smem_u32(Bt + (size_t)q * 2 * bbytes));
#pragma unroll
  for (int g = 0; g < kSl; ++g)
#pragma unroll
    for (int i = 0; i <= g; ++i) {
      const int j = g - i;
      const uint64_t ad = a0 + (uint64_t)((((i >> 2) * abytes) + (i & 3) * 32) >> 4);
      const uint64_t bd = b0 + (uint64_t)((((j >> 2) * bbytes) + (j & 3) * 32) >> 4);
      umma<1>(tmem + (uint32_t)(g * N), ad, bd, idesc, (first && i == 0) ? 0u : 1u);
    }
}

static __device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

static __device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(cols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_free(uint32_t tmem, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
}

// round(v 2^p) for an integer v (p of either sign).
__device__ __forceinline__ long long shift_round(long long v, int p) {
  if (p >= 0) return p < 63 ? v << p : 0;
  if (p <= -63) return 0;
  return (v + (1ll << (-p - 1))) >> (-p);
}

// Warp sum (every lane receives it).
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sums of nd dots over the first m entries of smem vectors: dot d pairs
// vectors xa[d] and xb[d]; warp w takes dots w, w + nw, ...  Every thread
// reads the results from out[] after the call's final barrier.
template <class FA, class FB>
__device__ __forceinline__ void block_dots(int nd, int m, FA xa, FB xb, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int d = warp; d < nd; d += nw) {
    double p = 0.0;
    for (int t = lane; t < m; t += 32) p = fma(xa(d, t), xb(d, t), p);
    p = warp_sum(p);
    if (lane == 0) out[d] = p;
  }
  __syncthreads();
}

// Gram values G[a][c] = x_a . x_c for a < c (the 28 that T needs) of b
// shared-memory vectors of length m, into G[a * b + c].
template <class FX>
__device__ __forceinline__ void gram_upper(int m, FX x, double* G) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int d = warp; d < B * (B - 1) / 2; d += nw) {
    int a = 0, rem = d;
    while (rem >= B - 1 - a) { rem -= B - 1 - a; ++a; }
    const int c = a + 1 + rem;
    double p = 0.0;
    for (int t = lane; t < m; t += 32) p = fma(x(a, t), x(c, t), p);
    p = warp_sum(p);
    if (lane == 0) G[a * B + c] = p;
  }
  __syncthreads();
}

// T of Q = H_0 ... H_{b-1} = I - Y T Y^T (forward, columnwise, as LAPACK's
// dlarft) from the Gram values G[a][c] = y_a . y_c (a < c) and the taus; by
// one thread.
__device__ void form_t(const double* G, const double* tau, double* T) {
  for (int j = 0; j < B; ++j) {
    for (int i = 0; i < B; ++i) T[i * B + j] = 0.0;
    T[j * B + j] = tau[j];
    for (int i = 0; i < j; ++i) {
      double s = 0.0;
      for (int l = i; l < j; ++l) s = fma(T[i * B + l], G[l * B + j], s);
      T[i * B + j] = -tau[j] * s;
    }
  }
}

// Householder reflector (dlarfg) of a vector with first entry alpha and
// squared norm sq of the rest: H = I - tau v v^T, v_0 = 1, v_i = x_i scl,
// H x = beta e_1.
__device__ __forceinline__ void reflector(double alpha, double sq, double& beta, double& tau, double& scl) {
  if (sq == 0.0) { beta = alpha; tau = 0.0; scl = 0.0; return; }
  beta = -copysign(sqrt(fma(alpha, alpha, sq)), alpha);
  tau = (beta - alpha) / beta;
  scl = 1.0 / (alpha - beta);
}
}  // namespace

bool band_supported(int n) { return n >= 64 && n <= 256 && n % B == 0; }

int band_nref(int n) {
  int c = 0;
  for (int i = 0; i + 1 < n; ++i) {
    int c0 = i + 1, c1 = std::min(i + B, n - 1);
    while (c1 > c0) { ++c; c0 += B; c1 = std::min(c1 + B, n - 1); }
  }
  return c;
}

size_t band_work_doubles(int n) { return work_stride(n); }

size_t band_item_bytes(int n) {
  return sizeof(double) * ((size_t)n * (B + 1) + band_work_doubles(n) + (size_t)band_nref(n) * B) + sizeof(int);
}

void band_carve(void* base, int n, int64_t S, BandArgs& a) {
  double* p = (double*)base;
  const size_t nref = (size_t)band_nref(n);
  a.band = p; p += (size_t)S * n * (B + 1);
  a.work = p; p += (size_t)S * band_work_doubles(n);
  a.refl = p; p += (size_t)S * nref * B;
  a.eA = (int*)p;
  a.err = (uint32_t*)(a.eA + S);
  a.n = n;
}

// ---------------------------------------------------------------------------
// Fixed-point copy of each matrix: e with |M|_F < 2^(e-1), Wk = round(M 2^(59-e)).
__global__ void __launch_bounds__(256) k_band_init(BandArgs a) {
  __shared__ double red[8];
  const int s = blockIdx.x, n = a.n;
  const double* M = a.M + (size_t)s * n * n;
  long long* A = (long long*)a.Wk + (size_t)s * n * n;
  double ss = 0.0;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) ss = fma(M[i], M[i], ss);
  ss = warp_sum(ss);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  ss = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) ss += red[w];
  const int e = ss > 0.0 ? exp_above(sqrt(ss)) + 1 : 0;
  if (threadIdx.x == 0) a.eA[s] = e;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) A[i] = fix_of(M[i], kFixBits - e);
}

// ---------------------------------------------------------------------------
// Panel k, QR of the column panel A[k:n][k:k+b] (m = n - k rows, one thread
// per row, the panel in shared memory column by column).  Writes R into the
// band, V (unit lower trapezoidal) and T into the scratch.
__global__ void __launch_bounds__(256) k_band_qr(BandArgs a, int k) {
  __shared__ double P[B][256];
  __shared__ double red[64], s_tau[B], s_sc[3];
  const int s = blockIdx.x, n = a.n, m = n - k, t = threadIdx.x;
  const long long* A = (const long long*)a.Wk + (size_t)s * n * n;
  const double unit = p2(a.eA[s] - kFixBits);
  Work w = work_of(a.work + (size_t)s * work_stride(n), n);
  if (t < m) {
#pragma unroll
    for (int j = 0; j < B; ++j) P[j][t] = (double)A[(size_t)(k + t) * n + k + j] * unit;
  } else if (t < 256) {
#pragma unroll
    for (int j = 0; j < B; ++j) P[j][t] = 0.0;
  }
  __syncthreads();
  double v[B];
  for (int j = 0; j < B; ++j) {
    // squared norm of column j below row j, and alpha = P[j][j]
    block_dots(1, m, [&](int, int r) { return r > j ? P[j][r] : 0.0; },
               [&](int, int r) { return P[j][r]; }, red);
    // the reflector's scalars once (sqrt and divisions cost tens of FP64
    // instructions), read by every thread
    if (t == 0) reflector(P[j][j], red[0], s_sc[0], s_sc[1], s_sc[2]);
    __syncthreads();
    const double beta = s_sc[0], tau = s_sc[1], scl = s_sc[2];
    const double vt = t == j ? 1.0 : ((t > j && t < m) ? P[j][t] * scl : 0.0);
    v[j] = vt;
    // R[t][j] (t < j) is final: column j is not touched by later reflectors
    if (t < j) a.band[((size_t)s * n + k + t) * (B + 1) + (j - t)] = P[j][t];
    if (t == j) a.band[((size_t)s * n + k + j) * (B + 1)] = beta;
    __syncthreads();                                   // every thread read P[j][*] before it changes
    P[j][t] = vt;                                      // column j now holds v
    __syncthreads();
    // w_c = sum_r v_r P[c][r] for c > j
    block_dots(B - 1 - j, m, [&](int d, int r) { return P[j][r]; },
               [&](int d, int r) { return P[j + 1 + d][r]; }, red);
    if (t >= j && t < m) {
      for (int c = j + 1; c < B; ++c) P[c][t] = fma(-tau * red[c - j - 1], vt, P[c][t]);
    }
    if (t == 0) s_tau[j] = tau;
    __syncthreads();
  }
  if (t < m) {
#pragma unroll
    for (int j = 0; j < B; ++j) w.V[(size_t)t * 8 + j] = v[j];
  }
  // Gram of the reflectors for T, then T
  __syncthreads();
  for (int j = 0; j < B; ++j) P[j][t] = (t < m) ? v[j] : 0.0;
  __syncthreads();
  gram_upper(m, [&](int i, int r) { return P[i][r]; }, red);
  if (t == 0) form_t(red, s_tau, w.T);
}

// ---------------------------------------------------------------------------
// Tensor-core products.  One CTA of 128 threads per (matrix, 128-row tile):
// the threads split the operands into digit slices in shared memory, thread 0
// issues the 36 products per k-step and commits them to an mbarrier that the
// next chunk's split waits on.  Operand A is 128 rows x K; operand B is N
// rows x K; K runs in chunks of 32 (two k-steps of 16).
namespace {
constexpr int kChunkK = 32;
constexpr uint32_t kABytes = 4 * kTileBytes;   // 2 k-steps x 2 slice halves
}

// W^T = A^T V over the rows k..n-1 (K) for the trailing columns k+b.. of one
// 128-column tile (the MMA's rows), N = 16 (V's b columns, zero padded).
__global__ void __launch_bounds__(256) k_band_gemm_w(BandArgs a, int k) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* As = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int N = 16;
  constexpr uint32_t bt = N * 128;                 // one B tile
  uint8_t* Bs = As + kABytes;
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  const int s = blockIdx.x, n = a.n, t = threadIdx.x, warp = t >> 5;
  const int rho = t & 127, hk = t >> 7;             // MMA row, and which 16 of a chunk's 32 K values
  const int c = k + B + blockIdx.y * kTileM + rho;  // this thread's column (MMA row)
  const int m = n - k;
  const long long* A = (const long long*)a.Wk + (size_t)s * n * n;
  Work w = work_of(a.work + (size_t)s * work_stride(n), n);
  if (t == 0) {
    s_fail = 0;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // B rows b..15 stay zero
  for (int i = t; i < (int)(4 * bt / 16); i += blockDim.x) ((uint4*)Bs)[i] = make_uint4(0, 0, 0, 0);
  if (warp == 0) tmem_alloc(&tmem_slot, 128);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = umma_idesc(1, kTileM, N);
  const int nchunk = (m + kChunkK - 1) / kChunkK;
  // the next chunk's 16 values of this thread, loaded while the products of
  // the current chunk run
  long long x[16];
  auto load = [&](int ch) {
    const int rb = k + ch * kChunkK + hk * 16;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int r = rb + e;
      x[e] = (c < n && r < n) ? A[(size_t)r * n + c] : 0ll;
    }
  };
  load(0);
  int committed = 0;                                 // commits thread 0 issued (the same count in every thread)
  for (int ch = 0; ch < nchunk; ++ch) {
    if (ch > 0 && !mbar_wait(&bar, (ch - 1) & 1)) atomicOr(&s_fail, 1);
    __syncthreads();
    if (s_fail) break;
    const int r0 = k + ch * kChunkK;
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      long long y[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) y[e] = x[g * 8 + e];
      uint4 d[kSl];
      digits8(y, d);
      store_slices(As, kTileBytes, hk, g, rho, d);
    }
    if (t < 32) {                                    // V: row j = t & 7 of B, 8 K values per thread
      const int j = t & 7, g8 = t >> 3;
      long long y[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int r = r0 + g8 * 8 + e;
        y[e] = r < n ? fix_of(w.V[(size_t)(r - k) * 8 + j], kFloatP - 1) : 0ll;
      }
      uint4 d[kSl];
      digits8(y, d);
      store_slices(Bs, bt, g8 >> 1, g8 & 1, j, d);
    }
    fence_async_smem();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
      issue_products(tmem, As, kTileBytes, Bs, bt, 0, N, idesc, ch == 0);
      issue_products(tmem, As, kTileBytes, Bs, bt, 1, N, idesc, false);
      umma_commit(&bar);
    }
    ++committed;
    if (ch + 1 < nchunk) load(ch + 1);
  }
  if (!s_fail && !mbar_wait(&bar, (nchunk - 1) & 1)) atomicOr(&s_fail, 1);
  tc_fence_after();
  __syncthreads();
  if (!s_fail && warp < 4) {
    // row c of W^T: value = (hi 2^32 + lo) 2^(eA - 64)
    long long hi[8], lo[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) { hi[j] = 0; lo[j] = 0; }
#pragma unroll
    for (int g = 0; g < kSl; ++g) {
      uint32_t v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(g * N), v);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const long long G = __float2ll_rn(__uint_as_float(v[j]));
        if (g < 4) hi[j] = (hi[j] << 8) + G;
        else lo[j] = (lo[j] << 8) + G;
      }
    }
    if (c < n) {
      const double sc = p2(a.eA[s] - 64);
#pragma unroll
      for (int j = 0; j < 8; ++j)
        w.Z[(size_t)j * n + (c - k - B)] = fma((double)hi[j], 4294967296.0 * sc, (double)lo[j] * sc);
    }
  } else if (s_fail && t == 0) {
    atomicOr(a.err, 1u);
  }
  // after an expired wait, give the products in flight another bounded wait
  // before their tensor memory is freed
  if (s_fail && committed > 0) mbar_wait(&bar, (committed - 1) & 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_free(tmem, 128);
}

// ---------------------------------------------------------------------------
// Panel k, row panel: Z = T^T W, RP = A[k:k+b][k+b:] - V[0:b] Z, LQ of RP (one
// thread per column), T_U, Z U^T, the column exponents of [Z ; U].  U and T_U
// go into the working matrix (rows k..k+b-1), L into the band.
__global__ void __launch_bounds__(256) k_band_lq(BandArgs a, int k) {
  __shared__ double R[B][256];
  __shared__ double red[64], s_tau[B], Ts[64], Vt[64], s_sc[3];
  const int s = blockIdx.x, n = a.n, t = threadIdx.x;
  const int mp = n - k - B;                          // columns k+b .. n-1
  long long* A = (long long*)a.Wk + (size_t)s * n * n;
  double* Ad = (double*)A;
  const double unit = p2(a.eA[s] - kFixBits);
  Work w = work_of(a.work + (size_t)s * work_stride(n), n);
  if (t < 64) { Ts[t] = w.T[t]; Vt[t] = w.V[t]; }    // T and the top b x b block of V
  __syncthreads();
  const bool act = t < mp;
  const int c = k + B + t;
  double z[B], rp[B];
  if (act) {
    double wv[B];
#pragma unroll
    for (int i = 0; i < B; ++i) wv[i] = w.Z[(size_t)i * n + t];
#pragma unroll
    for (int j = 0; j < B; ++j) {
      double acc = 0.0;
#pragma unroll
      for (int i = 0; i <= j; ++i) acc = fma(Ts[i * B + j], wv[i], acc);
      z[j] = acc;
    }
    // the top b x b block of V is unit lower triangular
#pragma unroll
    for (int i = 0; i < B; ++i) {
      double acc = fma((double)A[(size_t)(k + i) * n + c], unit, -z[i]);
#pragma unroll
      for (int j = 0; j < i; ++j) acc = fma(-Vt[i * B + j], z[j], acc);
      rp[i] = acc;
    }
#pragma unroll
    for (int j = 0; j < B; ++j) w.Z[(size_t)j * n + t] = z[j];
  } else {
#pragma unroll
    for (int j = 0; j < B; ++j) { z[j] = 0.0; rp[j] = 0.0; }
  }
#pragma unroll
  for (int i = 0; i < B; ++i) R[i][t] = rp[i];
  __syncthreads();
  double u[B];
  for (int j = 0; j < B; ++j) {
    block_dots(1, mp, [&](int, int q) { return q > j ? R[j][q] : 0.0; },
               [&](int, int q) { return R[j][q]; }, red);
    if (t == 0) reflector(R[j][j], red[0], s_sc[0], s_sc[1], s_sc[2]);
    __syncthreads();
    const double beta = s_sc[0], tau = s_sc[1], scl = s_sc[2];
    const double ut = t == j ? 1.0 : ((t > j && act) ? R[j][t] * scl : 0.0);
    u[j] = ut;
    // L[j][t] (t < j) is final: column t is not touched by later reflectors;
    // L[j][j] = beta.  Row k+j, column k+b+t: band offset b + t - j
    if (t < j) a.band[((size_t)s * n + k + j) * (B + 1) + (B + t - j)] = R[j][t];
    if (t == j) a.band[((size_t)s * n + k + j) * (B + 1) + B] = beta;
    __syncthreads();
    R[j][t] = ut;                                    // row j now holds u
    __syncthreads();
    block_dots(B - 1 - j, mp, [&](int d, int q) { return R[j][q]; },
               [&](int d, int q) { return R[j + 1 + d][q]; }, red);
    if (t >= j && act) {
      for (int i = j + 1; i < B; ++i) R[i][t] = fma(-tau * red[i - j - 1], ut, R[i][t]);
    }
    if (t == 0) s_tau[j] = tau;
    __syncthreads();
  }
  // rows of U (u[j] for this column) and the Gram for T_U
#pragma unroll
  for (int j = 0; j < B; ++j) R[j][t] = act ? u[j] : 0.0;
  __syncthreads();
  gram_upper(mp, [&](int i, int q) { return R[i][q]; }, red);
  if (t == 0) form_t(red, s_tau, Ts);                // T_U (Ts no longer needed as T)
  __syncthreads();
  // Z U^T (64 dots), z in smem for the reductions
  __shared__ double Zs[B][256];
#pragma unroll
  for (int j = 0; j < B; ++j) Zs[j][t] = z[j];
  __syncthreads();
  block_dots(B * B, mp, [&](int d, int q) { return Zs[d / B][q]; }, [&](int d, int q) { return R[d % B][q]; }, red);
  if (t < 64) w.ZU[t] = red[t];
  // U rows and T_U into the working matrix; the exponent of [Z ; U] per column
  if (act) {
    // exponent of the update's right operand column [Z 2^-eA ; U]
    const double dn = p2(-a.eA[s]);
    double mx = 0.0;
#pragma unroll
    for (int j = 0; j < B; ++j) {
      Ad[(size_t)(k + j) * n + c] = u[j];
      mx = fmax(mx, fmax(fabs(z[j]) * dn, fabs(u[j])));
    }
    w.er[t] = exp_above(mx);
  }
  if (t < 64) Ad[(size_t)(k + t / B) * n + k + (t % B)] = Ts[t];
}

// ---------------------------------------------------------------------------
// X = A U^T over the trailing rows (one 128-row tile, the MMA's rows) and
// columns k+b.. (K); then per row Y = (X - V Z U^T) T_U and the row exponent
// of [V | Y].
__global__ void __launch_bounds__(256) k_band_gemm_x(BandArgs a, int k) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* As = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int N = 16;
  constexpr uint32_t bt = N * 128;
  uint8_t* Bs = As + kABytes;
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  __shared__ double ZUs[64], TUs[64];
  const int s = blockIdx.x, n = a.n, t = threadIdx.x, warp = t >> 5;
  const int rho = t & 127, hk = t >> 7;
  const int r = k + B + blockIdx.y * kTileM + rho;  // this thread's row
  const int mp = n - k - B;                          // K = columns k+b .. n-1
  const long long* A = (const long long*)a.Wk + (size_t)s * n * n;
  const double* Ad = (const double*)A;
  Work w = work_of(a.work + (size_t)s * work_stride(n), n);
  if (t == 0) {
    s_fail = 0;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (t < 64) { ZUs[t] = w.ZU[t]; TUs[t] = Ad[(size_t)(k + t / B) * n + k + (t % B)]; }
  for (int i = t; i < (int)(4 * bt / 16); i += blockDim.x) ((uint4*)Bs)[i] = make_uint4(0, 0, 0, 0);
  if (warp == 0) tmem_alloc(&tmem_slot, 128);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = umma_idesc(1, kTileM, N);
  const int nchunk = (mp + kChunkK - 1) / kChunkK;
  long long x[16];
  auto load = [&](int ch) {
    const int cb = k + B + ch * kChunkK + hk * 16;  // n and cb are multiples of 8
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      if (r < n && cb + 8 * g < n) {
        const longlong2* p = (const longlong2*)(A + (size_t)r * n + cb + 8 * g);
#pragma unroll
        for (int e = 0; e < 4; ++e) { const longlong2 q = p[e]; x[8 * g + 2 * e] = q.x; x[8 * g + 2 * e + 1] = q.y; }
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) x[8 * g + e] = 0ll;
      }
    }
  };
  load(0);
  int committed = 0;                                 // commits thread 0 issued (the same count in every thread)
  for (int ch = 0; ch < nchunk; ++ch) {
    if (ch > 0 && !mbar_wait(&bar, (ch - 1) & 1)) atomicOr(&s_fail, 1);
    __syncthreads();
    if (s_fail) break;
    const int c0 = k + B + ch * kChunkK;
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      long long y[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) y[e] = x[g * 8 + e];
      uint4 d[kSl];
      digits8(y, d);
      store_slices(As, kTileBytes, hk, g, rho, d);
    }
    if (t < 32) {                                    // U: row j of B, 8 K values per thread
      const int j = t & 7, g8 = t >> 3;
      long long y[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int cc = c0 + g8 * 8 + e;
        y[e] = cc < n ? fix_of(Ad[(size_t)(k + j) * n + cc], kFloatP - 1) : 0ll;
      }
      uint4 d[kSl];
      digits8(y, d);
      store_slices(Bs, bt, g8 >> 1, g8 & 1, j, d);
    }
    fence_async_smem();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
      issue_products(tmem, As, kTileBytes, Bs, bt, 0, N, idesc, ch == 0);
      issue_products(tmem, As, kTileBytes, Bs, bt, 1, N, idesc, false);
      umma_commit(&bar);
    }
    ++committed;
    if (ch + 1 < nchunk) load(ch + 1);
  }
  if (!s_fail && !mbar_wait(&bar, (nchunk - 1) & 1)) atomicOr(&s_fail, 1);
  tc_fence_after();
  __syncthreads();
  if (!s_fail && warp < 4) {
    long long hi[8], lo[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) { hi[j] = 0; lo[j] = 0; }
#pragma unroll
    for (int g = 0; g < kSl; ++g) {
      uint32_t v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(g * N), v);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const long long G = __float2ll_rn(__uint_as_float(v[j]));
        if (g < 4) hi[j] = (hi[j] << 8) + G;
        else lo[j] = (lo[j] << 8) + G;
      }
    }
    if (r < n) {
      const double sc = p2(a.eA[s] - 64);
      double vr[B], x[B], y[B];
#pragma unroll
      for (int i = 0; i < B; ++i) vr[i] = w.V[(size_t)(r - k) * 8 + i];
#pragma unroll
      for (int j = 0; j < B; ++j) {
        double acc = fma((double)hi[j], 4294967296.0 * sc, (double)lo[j] * sc);
#pragma unroll
        for (int i = 0; i < B; ++i) acc = fma(-vr[i], ZUs[i * B + j], acc);
        x[j] = acc;
      }
      // exponent of the update's left operand row [V 2^eA | Y] (both parts of
      // the order of |A|; the right operand carries Z 2^-eA)
      const double up = p2(a.eA[s]);
      double mx = 0.0;
#pragma unroll
      for (int j = 0; j < B; ++j) {
        double acc = 0.0;
#pragma unroll
        for (int i = 0; i <= j; ++i) acc = fma(x[i], TUs[i * B + j], acc);
        y[j] = acc;
        mx = fmax(mx, fmax(fabs(acc), fabs(vr[j]) * up));
      }
      const int ro = r - k - B;
#pragma unroll
      for (int j = 0; j < B; ++j) w.Y[(size_t)ro * 8 + j] = y[j];
      w.el[ro] = exp_above(mx);
    }
  } else if (s_fail && t == 0) {
    atomicOr(a.err, 1u);
  }
  // after an expired wait, give the products in flight another bounded wait
  // before their tensor memory is freed
  if (s_fail && committed > 0) mbar_wait(&bar, (committed - 1) & 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_free(tmem, 128);
}

// ---------------------------------------------------------------------------
// Trailing update A[k+b:][k+b:] -= [V | Y] [Z ; U] for one 128-row tile, its
// 32-column tiles in turn: K = 2b = 16 (one k-step), applied in fixed point.
// The operands are [V 2^eA | Y] and [Z 2^-eA ; U] (the same product): V and U
// are of order 1, Y and Z of order |A|.  The row operand shares one exponent
// over the tile's rows, the column operand one over each 32-column tile (both
// the largest of the per-row / per-column exponents: digits keep 62 bits of
// the largest entry), so every element of a tile takes the same shifts.  256
// threads: the row operand is split once (V halves by threads 0-127, Y halves
// by 128-255); per column tile two warps split the column operand, thread 0
// issues the 36 products, and warp w applies the results of rows 32 (w % 4)
// .. +31 (its tensor-memory lanes) and columns 16 (w / 4) .. +15 of the tile,
// the row segment loaded before the products run.
__global__ void __launch_bounds__(256, 2) k_band_update(BandArgs a, int k) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* As = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int N = 32, NH = 16;
  constexpr uint32_t bt = N * 128;
  uint8_t* Bs = As + 2 * kTileBytes;
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail, s_el, s_er;
  const int s = blockIdx.x, n = a.n, t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int r0 = k + B + blockIdx.y * kTileM;       // first row of the tile
  long long* A = (long long*)a.Wk + (size_t)s * n * n;
  const double* Ad = (const double*)A;
  Work w = work_of(a.work + (size_t)s * work_stride(n), n);
  const int eA = a.eA[s];
  if (t == 0) {
    s_fail = 0;
    s_el = kZeroExp;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&tmem_slot, 256);
  __syncthreads();
  {
    // the tile's row exponent: the largest el of its rows
    const int r = r0 + (t & 127);
    int e = (t < 128 && r < n) ? w.el[r - k - B] : kZeroExp;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    if (lane == 0 && t < 128) atomicMax(&s_el, e);
  }
  __syncthreads();
  const int el = s_el;
  {
    // A operand: row rho = [V[r] 2^eA | Y[r]]
    const int rho = t & 127, part = t >> 7, r = r0 + rho;
    long long x[8];
    if (r < n && el != kZeroExp) {
#pragma unroll
      for (int e = 0; e < 8; ++e)
        x[e] = part == 0 ? fix_of(w.V[(size_t)(r - k) * 8 + e], kFloatP - el + eA)
                         : fix_of(w.Y[(size_t)(r - k - B) * 8 + e], kFloatP - el);
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) x[e] = 0;
    }
    uint4 d[kSl];
    digits8(x, d);
    store_slices(As, kTileBytes, 0, part, rho, d);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = umma_idesc(1, kTileM, N);
  const int quad = warp & 3, hc = warp >> 2;
  const int rho = quad * 32 + lane, r = r0 + rho;
  const int ntile = (n - k - B + N - 1) / N;
  int committed = 0;                                 // commits thread 0 issued (the same count in every thread)
  for (int ct = 0; ct < ntile; ++ct) {
    const int cb = k + B + ct * N;                  // first column of the tile
    // this warp's 16 columns of the row, loaded before the products run; n and
    // cw are multiples of 8, so the first 8 exist when cw < n and the second 8
    // when cw + 8 < n
    const int cw = cb + hc * NH;
    const bool rowok = r < n && el != kZeroExp && cw < n;
    const bool half2 = cw + 8 < n;
    longlong2* rowp = (longlong2*)(A + (size_t)r * n + cw);
    longlong2 q[NH / 2];
#pragma unroll
    for (int i = 0; i < NH / 2; ++i) q[i] = make_longlong2(0, 0);
    if (rowok) {
#pragma unroll
      for (int i = 0; i < NH / 4; ++i) q[i] = rowp[i];
      if (half2) {
#pragma unroll
        for (int i = NH / 4; i < NH / 2; ++i) q[i] = rowp[i];
      }
    }
    if (t < 2 * N) {                                 // B operand: column c = [Z[:, c] 2^-eA ; U[:, c]]
      const int cc = t & (N - 1), part = t >> 5, c = cb + cc;
      int er = c < n ? w.er[c - k - B] : kZeroExp;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) er = max(er, __shfl_xor_sync(0xffffffffu, er, o));
      if (t == 0) s_er = er;                         // the tile's column exponent
      long long x[8];
      if (c < n && er != kZeroExp) {
#pragma unroll
        for (int e = 0; e < 8; ++e)
          x[e] = part == 0 ? fix_of(w.Z[(size_t)e * n + (c - k - B)], kFloatP - er - eA)
                           : fix_of(Ad[(size_t)(k + e) * n + c], kFloatP - er);
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) x[e] = 0;
      }
      uint4 d[kSl];
      digits8(x, d);
      store_slices(Bs, bt, 0, part, cc, d);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
      issue_products(tmem, As, kTileBytes, Bs, bt, 0, N, idesc, true);
      umma_commit(&bar);
    }
    ++committed;
    if (!mbar_wait(&bar, ct & 1)) atomicOr(&s_fail, 1);
    tc_fence_after();
    __syncthreads();
    if (s_fail) break;
    const int er = s_er;
    // value of an element: (hi 2^32 + lo) 2^(el + er - 68), in fixed-point
    // units 2^(eA - 59): shifted by sh = el + er - eA - 9, the same for the
    // whole tile.  The tensor-memory loads are warp-collective: every lane
    // issues them; only the arithmetic and the stores depend on the row.
    const bool apply = rowok && er != kZeroExp;
    const int sh = el + er - eA - 9;
#pragma unroll
    for (int part = 0; part < 2; ++part) {           // this warp's 16 columns, 8 at a time
      const int jc = hc * NH + part * 8;
      // group sums here are integers of at most 8 x 16 x 2^14 = 2^21 in
      // magnitude, read back exactly by adding 1.5 2^23 (an FP32 add; the
      // bias 0x4B400000 of each is taken out of the pair sums below) and
      // paired in 32 bits: G0 2^8 + G1 and so on stay below 2^30
      int gb[kSl][8];
#pragma unroll
      for (int g = 0; g < kSl; ++g) {
        uint32_t v[8];
        tmem_ld8(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(g * N + jc), v);
#pragma unroll
        for (int j = 0; j < 8; ++j) gb[g][j] = __float_as_int(__uint_as_float(v[j]) + 12582912.0f);
      }
      if (apply) {
        // (b 2^8 + b) of two biased sums, modulo 2^32 (the pairs are exact in
        // 32-bit two's complement)
        constexpr uint32_t kBias = 0x4B400000u * 257u;
        auto pair = [&](int g, int j) {
          return (int)((uint32_t)gb[g][j] * 256u + (uint32_t)gb[g + 1][j] - kBias);
        };
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          long long del[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int j = 2 * i + h;
            const int h01 = pair(0, j), h23 = pair(2, j), l45 = pair(4, j), l67 = pair(6, j);
            const long long hi = (long long)h01 * 65536 + h23, lo = (long long)l45 * 65536 + l67;
            del[h] = shift_round(hi, 32 + sh) + shift_round(lo, sh);
          }
          longlong2& qq = q[part * 4 + i];
          qq.x -= del[0];
          qq.y -= del[1];
        }
      }
    }
    if (apply) {
#pragma unroll
      for (int i = 0; i < NH / 4; ++i) rowp[i] = q[i];
      if (half2) {
#pragma unroll
        for (int i = NH / 4; i < NH / 2; ++i) rowp[i] = q[i];
      }
    }
    tc_fence_before();
    __syncthreads();                                 // s_er and the B tiles are rewritten next
  }
  if (s_fail && t == 0) atomicOr(a.err, 1u);
  // after an expired wait, give the products in flight another bounded wait
  // before their tensor memory is freed
  if (s_fail && committed > 0) mbar_wait(&bar, (committed - 1) & 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_free(tmem, 256);
}

// ---------------------------------------------------------------------------
// Stage 2: bulge chasing, two matrices per warp (a half-warp each: every FP64
// instruction serves both, the reflector's formation included); each band and
// its bulges in shared memory, entry (r, c) at W[r * kWin + (c - r + 7)]
// (c - r in -7..15).  Per step a right reflector of length L <= b clears a row
// beyond its superdiagonal over rows row .. row+15 (lane = row), then a left
// reflector clears the bulge below the diagonal over columns c0 .. c0+15
// (lane = column).
__device__ __forceinline__ void chase_reflector(double x, int l16, int L, int hb, double& v, double& tau,
                                                double& beta) {
  double p = (l16 >= 1 && l16 < L) ? x * x : 0.0;
  p += __shfl_xor_sync(0xffffffffu, p, 1);
  p += __shfl_xor_sync(0xffffffffu, p, 2);
  p += __shfl_xor_sync(0xffffffffu, p, 4);
  const double sq = __shfl_sync(0xffffffffu, p, hb), alpha = __shfl_sync(0xffffffffu, x, hb);
  if (sq == 0.0) { v = l16 == 0 ? 1.0 : 0.0; tau = 0.0; beta = alpha; return; }
  // |beta| = sqrt(alpha^2 + sq); d = alpha - beta (no cancellation);
  // tau = (beta - alpha) / beta = |d| / |beta|, v = x / d
  const double rn = rsqrt(fma(alpha, alpha, sq));
  const double nrm = fma(alpha, alpha, sq) * rn;
  beta = -copysign(nrm, alpha);
  const double d = alpha - beta;
  tau = fabs(d) * rn;
  v = l16 == 0 ? 1.0 : (l16 < L ? x * (1.0 / d) : 0.0);
}

// Steps of sweep i of the chase on an n x n band (right reflectors it stores).
// (step t has c0 = i + 1 + 8t and runs while c0 < n - 1)
__host__ __device__ __forceinline__ int sweep_steps(int i, int n) {
  const int m = n - 2 - i;
  return m > 0 ? (m + B - 1) / B : 0;
}

// Sweeps run pipelined: warp w of kChaseWarps takes sweeps w, w + kChaseWarps,
// ...; step t of sweep i starts once sweep i-1 has finished step t+3 (or all
// of its steps), which keeps the regions of concurrent steps apart (a step of
// sweep i touches rows [c0-8, c0+8) and columns [c0, c0+16) with
// c0 = i + 1 + 8t).  Progress words in shared memory, a ring of kRing slots
// holding i * 64 + steps done; waits are bounded (error word on expiry).
constexpr int kChaseWarps = 8, kRing = 16, kLag = 3;

__global__ void __launch_bounds__(kChaseWarps * 32) k_band_chase(BandArgs a, int nref) {
  extern __shared__ double Bw[];
  __shared__ int prog[kRing];
  __shared__ int s_fail;
  const int n = a.n, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int l16 = lane & 15, half = lane >> 4, hb = lane & 16;
  const int s = 2 * blockIdx.x + half;
  const bool live = s < a.S;                          // an odd batch leaves the last half idle
  double* W = Bw + (size_t)half * n * kWin;
  for (int i = threadIdx.x; i < 2 * n * kWin; i += blockDim.x) Bw[i] = 0.0;
  if (threadIdx.x < kRing) prog[threadIdx.x] = -1;
  if (threadIdx.x == 0) s_fail = 0;
  __syncthreads();
  for (int hh = 0; hh < 2; ++hh) {
    const int sm = 2 * blockIdx.x + hh;
    if (sm >= a.S) break;
    const double* band = a.band + (size_t)sm * n * (B + 1);
    double* Wm = Bw + (size_t)hh * n * kWin;
    for (int i = threadIdx.x; i < n * (B + 1); i += blockDim.x) {
      const int r = i / (B + 1), o = i % (B + 1);
      if (r + o < n) Wm[r * kWin + o + 7] = band[i];
    }
  }
  __syncthreads();
#define AT(r, c) W[(r) * kWin + ((c) - (r) + 7)]
  double* refl = a.refl + (size_t)(live ? s : 0) * nref * B;
  volatile int* vprog = prog;
  // reflector index of this warp's first sweep
  int base = 0;
  for (int i = 0; i < warp && i + 1 < n; ++i) base += sweep_steps(i, n);
  bool fail = false;
  for (int i = warp; i + 1 < n && !fail; i += kChaseWarps) {
    const int T = sweep_steps(i, n), Tp = i > 0 ? sweep_steps(i - 1, n) : 0;
    if (lane == 0) vprog[i % kRing] = i * 64;
    int c0 = i + 1, c1 = min(i + B, n - 1), row = i;
    for (int t = 0; t < T; ++t) {
      if (i > 0) {                                    // wait for sweep i-1 to be kLag steps ahead
        const int need = min(t + kLag, Tp);
        if (lane == 0) {
          uint32_t it = 0;
          for (;; ++it) {
            const int v = vprog[(i - 1) % kRing];
            if ((v >> 6) > i - 1 || ((v >> 6) == i - 1 && (v & 63) >= need)) break;
            if (it > tcptx::kSpinLimit || *(volatile int*)&s_fail) { atomicOr(&s_fail, 1); break; }
            __nanosleep(20);
          }
          __threadfence_block();
        }
        __syncwarp();
        if (*(volatile int*)&s_fail) { fail = true; break; }
      }
      const int L = c1 - c0 + 1;
      const int idx = base + t;
      double v, tau, beta, vv[B];
      // right reflector: clear row `row` at columns c0+1 .. c1; rows row .. row+15
      chase_reflector(l16 < L ? AT(row, c0 + l16) : 0.0, l16, L, hb, v, tau, beta);
      if (live && l16 < B) refl[(size_t)idx * B + l16] = l16 == 0 ? tau : v;
#pragma unroll
      for (int q = 0; q < B; ++q) vv[q] = __shfl_sync(0xffffffffu, v, hb + q);
      {
        const int r = row + l16;
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < B; ++q) {
          const int cc = c0 + q;
          if (r < n && cc <= c1 && cc - r >= -7) acc = fma(AT(r, cc), vv[q], acc);
        }
        acc *= tau;
        __syncwarp();
#pragma unroll
        for (int q = 0; q < B; ++q) {
          const int cc = c0 + q;
          if (r < n && cc <= c1 && cc - r >= -7) AT(r, cc) = fma(-acc, vv[q], AT(r, cc));
        }
        __syncwarp();
        if (l16 < L) AT(row, c0 + l16) = l16 == 0 ? beta : 0.0;
        __syncwarp();
      }
      // left reflector: clear column c0 at rows c0+1 .. c1; columns c0 .. c0+15
      chase_reflector(l16 < L ? AT(c0 + l16, c0) : 0.0, l16, L, hb, v, tau, beta);
#pragma unroll
      for (int q = 0; q < B; ++q) vv[q] = __shfl_sync(0xffffffffu, v, hb + q);
      {
        const int cc = c0 + l16;
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < B; ++q)
          if (cc < n && q < L) acc = fma(AT(c0 + q, cc), vv[q], acc);
        acc *= tau;
        __syncwarp();
#pragma unroll
        for (int q = 0; q < B; ++q)
          if (cc < n && q < L) AT(c0 + q, cc) = fma(-acc, vv[q], AT(c0 + q, cc));
        __syncwarp();
        if (l16 < L) AT(c0 + l16, c0) = l16 == 0 ? beta : 0.0;
        __syncwarp();
      }
      if (lane == 0) {                                // publish: step t of sweep i done
        __threadfence_block();
        vprog[i % kRing] = i * 64 + t + 1;
      }
      row = c0;
      c0 += B;
      c1 = min(c1 + B, n - 1);
    }
    for (int q = i; q < i + kChaseWarps && q + 1 < n; ++q) base += sweep_steps(q, n);
  }
  __syncthreads();
  if (s_fail) {
    if (threadIdx.x == 0) atomicOr(a.err, 1u);
    return;
  }
  if (live && warp == 0) {
    double* bd = a.bd + (size_t)s * 3 * n;
    for (int r = l16; r < n; r += 16) {
      bd[r] = AT(r, r);
      bd[n + r] = r + 1 < n ? AT(r, r + 1) : 0.0;
      bd[2 * n + r] = 0.0;
    }
  }
#undef AT
}

// ---------------------------------------------------------------------------
// v = P1 P2 v_B for up to 16 kept vectors of one matrix, one CTA of 128
// threads; the vectors in shared memory (row stride n + 1: the 16 vectors in
// different banks).  P2: the chase's sweeps in reverse order; the right
// reflectors of one sweep act on disjoint column blocks c0 = i + 1 + 8q, so
// they commute and are applied at once, one (reflector, vector) pair per
// thread.  P1: the panels' compact reflectors in reverse order,
// v <- v - U^T T_U U v: U staged in shared memory, thread (a, j) forms
// (U v_a)_j, then (T_U U v_a)_j, then thread (a, part) updates every eighth
// entry of v_a.
constexpr int kBtThreads = 128;
__global__ void __launch_bounds__(kBtThreads) k_band_backtr(BandArgs a, BandVecArgs va, int nref) {
  extern __shared__ double Vs[];                     // [16][n+1], then U [8][n]
  __shared__ double tv[16][B + 1], tp[16][B + 1];
  const int s = blockIdx.x, n = a.n, t = threadIdx.x;
  const int ld = n + 1;
  double* Us = Vs + (size_t)16 * ld;
  const int nk = min(va.nk[s], 16);
  double* vrow = va.vrows + (size_t)s * va.kstride * n;
  for (int e = t; e < nk * n; e += kBtThreads) Vs[(e / n) * ld + e % n] = vrow[e];
  __syncthreads();
  const double* refl = a.refl + (size_t)s * nref * B;
  int base = nref;                                    // reflector index of sweep i's first step
  for (int i = n - 2; i >= 0 && nk > 0; --i) {
    const int T = sweep_steps(i, n);
    base -= T;
    for (int p = t; p < nk * T; p += kBtThreads) {
      const int q = p / nk, av = p - q * nk;
      const double* rv = refl + (size_t)(base + q) * B;
      const double tau = rv[0];
      if (tau == 0.0) continue;
      const int c0 = i + 1 + B * q, L = min(B, n - c0);
      double* x = Vs + (size_t)av * ld + c0;
      double vv[B];
      vv[0] = 1.0;
#pragma unroll
      for (int l = 1; l < B; ++l) vv[l] = l < L ? rv[l] : 0.0;
      double acc = x[0];
#pragma unroll
      for (int l = 1; l < B; ++l)
        if (l < L) acc = fma(vv[l], x[l], acc);
      acc *= tau;
#pragma unroll
      for (int l = 0; l < B; ++l)
        if (l < L) x[l] = fma(-acc, vv[l], x[l]);
    }
    __syncthreads();
  }
  const double* Ad = (const double*)(a.Wk + (size_t)s * n * n);
  const int av = t & 15, hj = t >> 4;                 // vector, and j (or the part of the columns)
  for (int k = n - 2 * B; k >= 0 && nk > 0; k -= B) {
    const int cb = k + B, mp = n - cb;
    for (int e = t; e < B * mp; e += kBtThreads) {
      const int j = e / mp, c = e - j * mp;
      Us[j * n + c] = Ad[(size_t)(k + j) * n + cb + c];
    }
    __syncthreads();
    if (av < nk) {                                    // (U v_a)_j
      const double* x = Vs + (size_t)av * ld + cb;
      const double* u = Us + (size_t)hj * n;
      double acc = 0.0;
      for (int c = 0; c < mp; ++c) acc = fma(u[c], x[c], acc);
      tv[av][hj] = acc;
    }
    __syncthreads();
    if (av < nk) {                                    // (T_U U v_a)_i, T_U upper triangular
      double acc = 0.0;
      for (int j = hj; j < B; ++j) acc = fma(Ad[(size_t)(k + hj) * n + k + j], tv[av][j], acc);
      tp[av][hj] = acc;
    }
    __syncthreads();
    if (av < nk) {
      double* x = Vs + (size_t)av * ld + cb;
      double tq[B];
#pragma unroll
      for (int j = 0; j < B; ++j) tq[j] = tp[av][j];
      for (int c = hj; c < mp; c += B) {
        double y = x[c];
#pragma unroll
        for (int j = 0; j < B; ++j) y = fma(-Us[j * n + c], tq[j], y);
        x[c] = y;
      }
    }
    __syncthreads();
  }
  const double* sg = va.sig + (size_t)s * va.n_pad;
  const int* kept = va.kept + (size_t)s * va.kstride;
  for (int e = t; e < nk * n; e += kBtThreads) {
    const double x = Vs[(e / n) * ld + e % n];
    vrow[e] = va.unit_rows ? x : sg[kept[e / n]] * x;
  }
}

// ---------------------------------------------------------------------------
namespace {
constexpr size_t kGemmSmem = kABytes + 4 * 16 * 128 + 1024;      // A tiles, B tiles (N = 16), alignment
constexpr size_t kUpdSmemNeed = 2 * kTileBytes + 2 * 32 * 128 + 1024;
// requested so that at most two update CTAs share an SM (2 x 256 columns of tensor memory)
constexpr size_t kUpdSmem = 80 * 1024;
}  // namespace

cudaError_t launch_band_reduce(const BandArgs& a, bool chase, cudaStream_t st) {
  if (a.S <= 0) return cudaSuccess;
  if (!band_supported(a.n)) return cudaErrorInvalidValue;
  static_assert(kUpdSmemNeed <= kUpdSmem, "update tiles exceed the requested shared memory");
  static std::atomic<uint64_t> at_w{0}, at_x{0}, at_u{0};
  cudaError_t e = raise_smem_limit(k_band_gemm_w, (int)kGemmSmem, at_w);
  if (e == cudaSuccess) e = raise_smem_limit(k_band_gemm_x, (int)kGemmSmem, at_x);
  if (e == cudaSuccess) e = raise_smem_limit(k_band_update, (int)kUpdSmem, at_u);
  if (e != cudaSuccess) return e;
  const int n = a.n, S = a.S;
  k_band_init<<<S, 256, 0, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int k = 0; k < n; k += B) {
    k_band_qr<<<S, 256, 0, st>>>(a, k);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (k + B >= n) break;
    const int mp = n - k - B;
    const int tiles = (mp + kTileM - 1) / kTileM;
    k_band_gemm_w<<<dim3(S, tiles), 256, kGemmSmem, st>>>(a, k);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_band_lq<<<S, 256, 0, st>>>(a, k);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_band_gemm_x<<<dim3(S, tiles), 256, kGemmSmem, st>>>(a, k);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_band_update<<<dim3(S, tiles), 256, kUpdSmem, st>>>(a, k);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return chase ? launch_band_chase(a, st) : cudaSuccess;
}

cudaError_t launch_band_chase(const BandArgs& a, cudaStream_t st) {
  if (a.S <= 0) return cudaSuccess;
  if (!band_supported(a.n)) return cudaErrorInvalidValue;
  static std::atomic<uint64_t> at{0};
  cudaError_t e = raise_smem_limit(k_band_chase, (int)(2 * 256 * kWin * sizeof(double)), at);
  if (e != cudaSuccess) return e;
  k_band_chase<<<(a.S + 1) / 2, kChaseWarps * 32, 2 * a.n * kWin * sizeof(double), st>>>(a, band_nref(a.n));
  return cudaGetLastError();
}

cudaError_t launch_band_backtr(const BandVecArgs& va, cudaStream_t st) {
  const BandArgs& a = *va.band;
  if (a.S <= 0) return cudaSuccess;
  static std::atomic<uint64_t> at{0};
  auto bytes = [](int n) { return (size_t)(24 * n + 16) * sizeof(double); };
  const size_t smem = bytes(a.n);
  cudaError_t e = raise_smem_limit(k_band_backtr, (int)bytes(256), at);
  if (e != cudaSuccess) return e;
  k_band_backtr<<<a.S, kBtThreads, smem, st>>>(a, va, band_nref(a.n));
  return cudaGetLastError();
}

}  // namespace mctrg
