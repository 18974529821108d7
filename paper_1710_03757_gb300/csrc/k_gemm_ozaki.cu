// K5 at FP64 accuracy on the tensor cores: the plaquette GEMM M = X Yt^T by
// error-free splitting (Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59,
// 2012), with BF16 slices multiplied exactly by tcgen05.mma.
//
// Split (k_ozaki_split, one warp per row of X or Yt): with e the exponent of
// the row's largest magnitude (every |x| < 2^e) and P = (b-1) + b(s-1) = 55,
// the integer F = round(x 2^{P-e}) (|F| <= 2^P, read from the significand and
// exponent bits with integer shifts) is recoded into signed digits from the
// bottom, a_i = ((F + 2^{b-1}) mod 2^b) - 2^{b-1}, F <- (F - a_i) / 2^b, the
// top digit taking the rest, so x = 2^e sum_i a_i 2^{-(b-1)-b i} + r with
// |r| <= 2^{e-P-1}, |a_i| <= 2^{b-1} (b <= 8 bits: exact in BF16).  Only
// integer and FP32 operations per element: FP64 issues at 1/64 of the FP32
// rate on this GPU.  The slice planes hold a_i 2^{-(b-1)-b i} (a power-of-two
// scaling, still exact).
//
// Product: x y = 2^{e_x + e_y} sum_{i,j} A_i B_j.  All products of one group
// g = i + j carry the same weight, and their sum over K is an integer
// multiple of it bounded by m K 2^{2b-2} for m pairs; with b = 8 for K <= 256
// and b = 7 for K <= 1024 the groups of up to four pairs stay at or below
// 2^24, so their FP32 accumulation is exact, and the larger later groups
// round below 2^-53 of the leading one.  Groups g <= s-1 are kept (s(s+1)/2
// slice products; s = 7 for b = 8, s = 8 for b = 7, i.e. 55 bits of each
// operand): the dropped groups and residuals are below 2^-43 K-relative of
// |row max| |column max|, the order of an FP64 dot product's own error.
//
// GEMM (k_gemm_ozaki): one CTA of 128 threads per (tensor, 128-row tile,
// 64-column tile).  Tensor memory holds one 128 x 64 FP32 accumulator per
// group (s x 64 <= 512 columns).  Warp 0 lane 0 streams, per step, one
// 128-byte K slice of an A slice plane (128 rows) and of a B slice plane
// (64 rows) with 4-D TMA loads (K, row, tensor, slice) into a ring of
// shared-memory stages (128-byte swizzle); warp 1 lane 0 issues four
// tcgen05.mma (K = 16 each) per step into the group's accumulator; the
// epilogue sums the groups from the smallest in FP64, scales by 2^{e_x + e_y}
// and writes M matricized for the next level like the FP64 GEMM.  Every
// mbarrier wait is bounded; on expiry the kernel records an error word,
// waits (bounded) for the copies it issued, skips the epilogue and still
// frees its tensor memory.
#include <cuda_bf16.h>

#include <cstdint>

#include "common.cuh"
#include "kernels_tc.h"
#include "tc_ptx.cuh"

namespace mctrg {

using namespace tcptx;

namespace {
constexpr int kOzTileM = 128;    // output rows per CTA (tensor-memory lanes)
constexpr int kOzTileN = 64;     // output columns per CTA and per accumulator
constexpr int kOzKBlk = 64;      // BF16 elements per 128-byte K slice
constexpr int kOzStages = 8;
constexpr uint32_t kOzABytes = kOzTileM * 128u, kOzBBytes = kOzTileN * 128u;
constexpr uint32_t kOzStageBytes = kOzABytes + kOzBBytes;
}  // namespace

void ozaki_params(int K, int* bits, int* slices) {
  *bits = K <= 256 ? 8 : 7;
  *slices = K <= 256 ? 7 : 8;
}

bool gemm_ozaki_supported(int n, int K) { return n >= 1 && K >= kOzKBlk && K % kOzKBlk == 0 && K <= 1024; }

// 2^p for -126 <= p <= 127, from its exponent bits.
__device__ __forceinline__ float pow2f(int p) { return __int_as_float((127 + p) << 23); }

// 2^p as a double for any p (exponent bits in the normal range; beyond it a
// product of two powers, so underflow and overflow round as a scaling would).
__device__ __forceinline__ double pow2d(int p) {
  if (p >= -1022 && p <= 1023) return __hiloint2double((1023 + p) << 20, 0);
  const int h = p / 2;
  return __hiloint2double((1023 + h) << 20, 0) * __hiloint2double((1023 + (p - h)) << 20, 0);
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_ozaki_split(const double* src, int64_t rows, int K, int slices, int bits,
                                                     __nv_bfloat16* dst, int* expo) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (row >= rows) return;
  const double* x = src + row * K;
  // largest magnitude: the bit patterns of non-negative doubles order like their values
  long long mb = 0;
  for (int k = lane; k < K; k += 32) mb = max(mb, __double_as_longlong(x[k]) & 0x7FFFFFFFFFFFFFFFll);
  for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  // e with max = f 2^e, f in [0.5, 1): every |x| < 2^e
  int e = (int)(mb >> 52) - 1022;
  if ((mb >> 52) == 0) {
    e = 0;
    if (mb != 0) frexp(__longlong_as_double(mb), &e);   // subnormal largest value
  }
  if (lane == 0) expo[row] = e;
  const size_t plane = (size_t)rows * K;
  const int P = (bits - 1) + bits * (slices - 1);   // fraction bits kept (55)
  for (int k = lane; k < K; k += 32) {
    // |x| 2^{P-e} as an integer, rounded to nearest: x = q 2^{E-52}, q the
    // 53-bit significand, so the value is q 2^{E-52+P-e} with E <= e-1
    const long long bitsx = __double_as_longlong(x[k]);
    const int be = (int)((bitsx >> 52) & 0x7ff);
    const long long q = (bitsx & 0xFFFFFFFFFFFFFll) | (be ? (1ll << 52) : 0ll);
    const int sh = (be ? be - 1075 : -1074) + P - e;
    long long F;
    if (sh >= 0) F = q << sh;                   // sh <= P - 53 (= 2)
    else if (sh > -62) F = (q + (1ll << (-sh - 1))) >> (-sh);
    else F = 0;
    if (bitsx < 0) F = -F;
    // signed digits from the bottom: d in [-2^{b-1}, 2^{b-1}), the top one the rest
    __nv_bfloat16* o = dst + (size_t)row * K + k;
    // (the digit depends only on the low bits of F: 32-bit arithmetic and a
    // 32-bit conversion, both off the FP64 pipe)
    const int half = 1 << (bits - 1), mask = (1 << bits) - 1;
    for (int i = slices - 1; i >= 1; --i) {
      const int d = (int)(((unsigned)(F & 0xffffffffll) + (unsigned)half) & (unsigned)mask) - half;
      F = (F - d) >> bits;
      o[(size_t)i * plane] = __float2bfloat16_rn(__int2float_rn(d) * pow2f(-(bits - 1) - bits * i));
    }
    o[0] = __float2bfloat16_rn(__int2float_rn((int)F) * pow2f(-(bits - 1)));
  }
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128, 1)
    k_gemm_ozaki(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB, GemmOzArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[kOzStages], empty_bar[kOzStages], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  const int n = a.n, S = a.slices;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int it = blockIdx.x, mt = blockIdx.y, nt = blockIdx.z;
  const int KB = a.K / kOzKBlk;
  constexpr uint32_t ncols = 512;

  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < kOzStages; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
    mbar_init(&done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(&tmem_slot)), "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer: steps in group order (g, then i, then the K slices)
    int step = 0, issued = 0;
    for (int g = 0; g < S && !s_fail; ++g)
      for (int i = 0; i <= g && !s_fail; ++i)
        for (int kb = 0; kb < KB; ++kb, ++step) {
          const int s = step % kOzStages, round = step / kOzStages;
          if (round > 0 && !mbar_wait(&empty_bar[s], (round - 1) & 1)) { atomicOr(&s_fail, 1); break; }
          uint8_t* st = smem + (size_t)s * kOzStageBytes;
          mbar_expect_tx(&full_bar[s], kOzStageBytes);
          tma_load_4d(st, &mA, kb * kOzKBlk, mt * kOzTileM, it, i, &full_bar[s]);
          tma_load_4d(st + kOzABytes, &mB, kb * kOzKBlk, nt * kOzTileN, it, g - i, &full_bar[s]);
          issued = step + 1;
        }
    if (s_fail) {
      // before leaving, let the copies already issued land (bounded)
      for (int q = issued - kOzStages < 0 ? 0 : issued - kOzStages; q < issued; ++q)
        mbar_wait(&full_bar[q % kOzStages], (q / kOzStages) & 1);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: accumulator g at tensor-memory columns 64 g
    const uint32_t idesc = umma_idesc(1, kOzTileM, kOzTileN);
    int step = 0;
    bool ok = true;
    for (int g = 0; g < S && ok; ++g)
      for (int i = 0; i <= g && ok; ++i)
        for (int kb = 0; kb < KB; ++kb, ++step) {
          const int s = step % kOzStages, round = step / kOzStages;
          if (!mbar_wait(&full_bar[s], round & 1)) { atomicOr(&s_fail, 1); ok = false; break; }
          tc_fence_after();
          const uint32_t base = smem_u32(smem + (size_t)s * kOzStageBytes);
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {      // 32 bytes of K per instruction
            const uint64_t ad = umma_desc(base + ks * 32), bd = umma_desc(base + kOzABytes + ks * 32);
            umma<1>(tmem + (uint32_t)(g * kOzTileN), ad, bd, idesc, (i | kb | ks) ? 1u : 0u);
          }
          umma_commit(&empty_bar[s]);
        }
    umma_commit(&done_bar);
  }
  __syncwarp();
  const bool done = mbar_wait(&done_bar, 0);
  if (!done) atomicOr(&s_fail, 1);
  tc_fence_after();
  __syncthreads();
  if (!s_fail) {
    // epilogue: warp w owns accumulator rows 32w .. 32w+31 (tensor-memory lanes)
    const int r = mt * kOzTileM + warp * 32 + lane;          // output row (al, be)
    const int D = a.D;
    const int64_t item = a.c0 + it;
    int par = a.fixed_parity;
    if (par < 0) par = tensor_parity(a.L, a.level_new, item % a.Nnew);
    double* Mo = a.M + (int64_t)it * n * n;
    const int* ey = a.expY + (int64_t)it * n;
    const int er = r < n ? a.expX[(int64_t)it * n + r] : 0;
    const int al = r / D, be = r - al * D;
    // group g holds an integer I_g times 2^{-2(b-1)-b g} (exact below 2^24; the
    // later, larger groups are integers too, at most 2^27): read back as
    // integers (an FP32 scaling by a power of two and a conversion), packed
    // into two 64-bit words (groups 0..3 and 4..s-1, each below 2^53), and
    // only those two are converted to FP64 and scaled by 2^{e_x + e_y}
    const int bits = a.bits;
    const int w0 = 2 * (bits - 1);                  // weight exponent of group 0
    const int split = S < 4 ? S : 4;                 // groups in the first word
    for (int c0 = 0; c0 < kOzTileN; c0 += 32) {
      long long hi[32], lo[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) { hi[j] = 0; lo[j] = 0; }
      for (int g = 0; g < S; ++g) {
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(g * kOzTileN + c0), v);
        const float up = pow2f(w0 + bits * g);
        if (g < split) {
#pragma unroll
          for (int j = 0; j < 32; ++j) hi[j] = (hi[j] << bits) + __float2int_rn(__uint_as_float(v[j]) * up);
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) lo[j] = (lo[j] << bits) + __float2int_rn(__uint_as_float(v[j]) * up);
        }
      }
      if (r < n) {
        // value = hi 2^{-w0 - b (split-1)} + lo 2^{-w0 - b (S-1)}, times 2^{er + ec}
        const int ph = -w0 - bits * (split - 1) + er, pl = -w0 - bits * (S - 1) + er;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int cc = nt * kOzTileN + c0 + j;
          if (cc < n) {
            const int de = cc / D, ga = cc - de * D;
            const int ec = ey[cc];
            const double val = fma((double)hi[j], pow2d(ph + ec), (double)lo[j] * pow2d(pl + ec));
            if (par == 0) Mo[(int64_t)r * n + cc] = val;
            else Mo[(int64_t)(be * D + de) * n + (ga * D + al)] = val;
          }
        }
      }
    }
  } else if (threadIdx.x == 0) {
    atomicOr(a.err, 1u);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// ---------------------------------------------------------------------------
// Slice planes [slices][items][n][K] (BF16) as a 4-D tensor (K, row, item,
// slice), box = one 128-byte K slice x box_rows rows.
static bool encode_slices(CUtensorMap* m, const void* base, uint64_t K, uint64_t n, uint64_t items, uint64_t slices,
                          uint32_t box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[4] = {K, n, items, slices};
  cuuint64_t strides[3] = {K * 2, n * K * 2, items * n * K * 2};
  cuuint32_t box[4] = {(cuuint32_t)kOzKBlk, box_rows, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

cudaError_t launch_ozaki_split(const double* src, int64_t rows, int K, void* dst, int* expo, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  int bits, slices;
  ozaki_params(K, &bits, &slices);
  const int64_t blocks = (rows + 7) / 8;
  k_ozaki_split<<<(unsigned)blocks, 256, 0, st>>>(src, rows, K, slices, bits, (__nv_bfloat16*)dst, expo);
  return cudaGetLastError();
}

cudaError_t launch_gemm_ozaki(const GemmOzArgs& a, const void* Xs, const void* Ys, cudaStream_t st) {
  if (a.n_items <= 0) return cudaSuccess;
  if (!gemm_ozaki_supported(a.n, a.K) || a.n_items > (1 << 30)) return cudaErrorInvalidValue;
  if (a.slices * kOzTileN > 512) return cudaErrorInvalidValue;
  int bits = 0, slices = 0;
  ozaki_params(a.K, &bits, &slices);
  if (a.bits != bits || a.slices != slices) return cudaErrorInvalidValue;
  CUtensorMap mA, mB;
  if (!encode_slices(&mA, Xs, a.K, a.n, a.n_items, a.slices, kOzTileM) ||
      !encode_slices(&mB, Ys, a.K, a.n, a.n_items, a.slices, kOzTileN))
    return cudaErrorInvalidValue;
  const size_t smem = (size_t)kOzStages * kOzStageBytes + 1024;
  static std::atomic<uint64_t> attr{0};
  cudaError_t e = raise_smem_limit(k_gemm_ozaki, (int)smem, attr);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)a.n_items, (unsigned)((a.n + kOzTileM - 1) / kOzTileM),
            (unsigned)((a.n + kOzTileN - 1) / kOzTileN));
  k_gemm_ozaki<<<grid, 128, smem, st>>>(mA, mB, a);
  return cudaGetLastError();
}

}  // namespace mctrg
