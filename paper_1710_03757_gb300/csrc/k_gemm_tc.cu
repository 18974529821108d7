// K5 on the tensor cores: the plaquette GEMM T' = X Yt^T in TF32 or BF16 with
// FP32 accumulation (the precision pattern of the contraction), sm_103a
// tcgen05 path.
//
// Per tensor, X and Yt (n x K, FP64 from k_form_xy) are scaled by their
// largest magnitude and rounded to TF32 (in an FP32 container) or BF16; with
// `passes` = 3 the rounding residual is kept as a second operand and the
// product is hi*hi + hi*lo + lo*hi (an error-compensated split), which brings
// the inputs' relative error from 2^-11 (TF32) / 2^-8 (BF16) to about its
// square.  The FP32 result times the two scales is written in FP64, already
// matricized for the next level, for the FP64 SVD.
//
// Kernel: one CTA of 128 threads per (tensor, 128-row tile, 256-column tile
// of the output); n a multiple of 256 up to 1024 (chi = 16 ... 32).
// The accumulator (128 rows x 256 FP32 columns) lives in tensor memory.
// Warp 0 lane 0 loads 128-byte-wide K slices of both operands with TMA
// (128-byte swizzle) into a ring of shared-memory stages; warp 1 lane 0
// issues tcgen05.mma (K = 32 bytes per instruction, four per slice) and
// releases each stage with tcgen05.commit; all four warps then read the
// accumulator rows they own from tensor memory (tcgen05.ld) for the epilogue.
// Every wait on an mbarrier is bounded; on expiry the kernel records an
// error word, waits (bounded) for the copies it issued, skips the epilogue
// and still frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <cstring>

#include "common.cuh"
#include "kernels_tc.h"
#include "tc_ptx.cuh"

namespace mctrg {

using namespace tcptx;

// ---------------------------------------------------------------------------
// Per-tensor scaling and rounding of X / Yt.
template <int KIND>
__global__ void k_convert_scaled(const double* src, int64_t per_item, void* hi_, void* lo_, double* scale) {
  __shared__ double red[32];
  const int64_t it = blockIdx.x;
  const double* s = src + it * per_item;
  double m = 0.0;
  for (int64_t e = threadIdx.x; e < per_item; e += blockDim.x) m = fmax(m, fabs(s[e]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmax(mm, red[w]);
    red[0] = mm > 0.0 ? mm : 1.0;
    scale[it] = red[0];
  }
  __syncthreads();
  const double inv = 1.0 / red[0];
  if constexpr (KIND == 0) {
    float* hi = (float*)hi_ + it * per_item;
    float* lo = lo_ ? (float*)lo_ + it * per_item : nullptr;
    for (int64_t e = threadIdx.x; e < per_item; e += blockDim.x) {
      const double v = s[e] * inv;
      uint32_t h;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"((float)v));
      const float hf = __uint_as_float(h);
      hi[e] = hf;
      if (lo) {
        uint32_t l;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"((float)(v - (double)hf)));
        lo[e] = __uint_as_float(l);
      }
    }
  } else {
    __nv_bfloat16* hi = (__nv_bfloat16*)hi_ + it * per_item;
    __nv_bfloat16* lo = lo_ ? (__nv_bfloat16*)lo_ + it * per_item : nullptr;
    for (int64_t e = threadIdx.x; e < per_item; e += blockDim.x) {
      const double v = s[e] * inv;
      const __nv_bfloat16 h = __double2bfloat16(v);
      hi[e] = h;
      if (lo) lo[e] = __double2bfloat16(v - (double)__bfloat162float(h));
    }
  }
}

template <int KIND>
__global__ void __launch_bounds__(128, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mBh,
              const __grid_constant__ CUtensorMap mAl, const __grid_constant__ CUtensorMap mBl, GemmTcArgs a,
              int stages) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[kTcMaxStages], empty_bar[kTcMaxStages], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  const int n = a.n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t it = blockIdx.x;
  const int mt = blockIdx.y;                            // 128-row tile of the output
  const int nt = blockIdx.z;                            // 256-column tile of the output
  constexpr int NT = 256;
  constexpr int kElems = KIND == 0 ? 32 : 64;           // elements per 128-byte row
  const int KB = a.K / kElems;
  const uint32_t a_bytes = 128u * 128u, b_bytes = (uint32_t)NT * 128u;
  const uint32_t part = a_bytes + b_bytes;
  const uint32_t stage_bytes = (a.passes == 3 ? 2u : 1u) * part;
  const uint32_t ncols = NT;

  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < stages; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
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
    // producer: one 128-byte K slice of A (this tile's 128 rows) and B (this tile's 256 rows) per stage
    const int ya = (int)(it * n + mt * 128), yb = (int)(it * n + nt * NT);
    int issued = 0;
    for (int kb = 0; kb < KB; ++kb) {
      const int s = kb % stages, round = kb / stages;
      if (round > 0 && !mbar_wait(&empty_bar[s], (round - 1) & 1)) { atomicOr(&s_fail, 1); break; }
      uint8_t* st = smem + (size_t)s * stage_bytes;
      mbar_expect_tx(&full_bar[s], stage_bytes);
      tma_load_2d(st, &mAh, kb * kElems, ya, &full_bar[s]);
      tma_load_2d(st + a_bytes, &mBh, kb * kElems, yb, &full_bar[s]);
      if (a.passes == 3) {
        tma_load_2d(st + part, &mAl, kb * kElems, ya, &full_bar[s]);
        tma_load_2d(st + part + a_bytes, &mBl, kb * kElems, yb, &full_bar[s]);
      }
      issued = kb + 1;
    }
    if (s_fail) {
      // before leaving, let the copies already issued land (bounded)
      for (int kb = issued - stages < 0 ? 0 : issued - stages; kb < issued; ++kb)
        mbar_wait(&full_bar[kb % stages], (kb / stages) & 1);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t idesc = umma_idesc(KIND, 128, NT);
    for (int kb = 0; kb < KB; ++kb) {
      const int s = kb % stages, round = kb / stages;
      if (!mbar_wait(&full_bar[s], round & 1)) { atomicOr(&s_fail, 1); break; }
      tc_fence_after();
      const uint32_t base = smem_u32(smem + (size_t)s * stage_bytes);
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {                    // 32 bytes of K per instruction
        const uint64_t ah = umma_desc(base + ks * 32), bh = umma_desc(base + a_bytes + ks * 32);
        umma<KIND>(tmem, ah, bh, idesc, (kb | ks) ? 1u : 0u);
        if (a.passes == 3) {
          const uint64_t al = umma_desc(base + part + ks * 32), bl = umma_desc(base + part + a_bytes + ks * 32);
          umma<KIND>(tmem, ah, bl, idesc, 1u);
          umma<KIND>(tmem, al, bh, idesc, 1u);
        }
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
    const int r = mt * 128 + warp * 32 + lane;                    // output row (al, be)
    const double sc = a.scaleX[it] * a.scaleY[it];
    const int D = a.D;
    const int64_t item = a.c0 + it;
    int par = a.fixed_parity;
    if (par < 0) par = tensor_parity(a.L, a.level_new, item % a.Nnew);
    double* Mo = a.M + it * (int64_t)n * n;
    const int al = r / D, be = r - al * D;
    for (int c0 = 0; c0 < NT; c0 += 32) {
      uint32_t v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (r < n) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int cc = nt * NT + c0 + j;
          const int de = cc / D, ga = cc - de * D;
          const double val = (double)__uint_as_float(v[j]) * sc;
          if (par == 0) Mo[(int64_t)r * n + cc] = val;
          else Mo[(int64_t)(be * D + de) * n + (ga * D + al)] = val;
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
// rows x K matrix (row-major, 16-byte aligned), box = 128-byte K slice x box_rows rows.
static bool encode_map(CUtensorMap* m, const void* base, int kind, uint64_t rows, uint64_t K, uint32_t box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
  if (!enc) return false;
  const uint32_t esize = kind == 0 ? 4 : 2;
  cuuint64_t dims[2] = {K, rows};
  cuuint64_t strides[1] = {K * esize};
  cuuint32_t box[2] = {128u / esize, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, kind == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                   const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool gemm_tc_supported(int n, int K, int kind) {
  return n % 256 == 0 && n <= 1024 && K % (kind == 0 ? 32 : 64) == 0 && K >= 64;
}

cudaError_t launch_convert_scaled(const double* src, int64_t per_item, int64_t n_items, int kind, void* hi, void* lo,
                                  double* scale, cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  if (kind == 0) k_convert_scaled<0><<<(unsigned)n_items, 256, 0, st>>>(src, per_item, hi, lo, scale);
  else k_convert_scaled<1><<<(unsigned)n_items, 256, 0, st>>>(src, per_item, hi, lo, scale);
  return cudaGetLastError();
}

cudaError_t launch_gemm_tc(const GemmTcArgs& a, int kind, const void* Xh, const void* Yh, const void* Xl,
                           const void* Yl, cudaStream_t st) {
  if (a.n_items <= 0) return cudaSuccess;
  if (!gemm_tc_supported(a.n, a.K, kind)) return cudaErrorInvalidValue;
  CUtensorMap mAh, mBh, mAl, mBl;
  const uint64_t rows = (uint64_t)a.n_items * a.n;
  if (!encode_map(&mAh, Xh, kind, rows, a.K, 128) || !encode_map(&mBh, Yh, kind, rows, a.K, 256))
    return cudaErrorInvalidValue;
  if (a.passes == 3) {
    if (!encode_map(&mAl, Xl, kind, rows, a.K, 128) || !encode_map(&mBl, Yl, kind, rows, a.K, 256))
      return cudaErrorInvalidValue;
  } else {
    mAl = mAh;
    mBl = mBh;
  }
  const uint32_t part = 128u * 128u + 256u * 128u;
  const uint32_t stage_bytes = (a.passes == 3 ? 2u : 1u) * part;
  int stages = (int)((200u * 1024u) / stage_bytes);
  if (stages > kTcMaxStages) stages = kTcMaxStages;
  if (stages < 1) return cudaErrorInvalidValue;
  const size_t smem = (size_t)stages * stage_bytes + 1024;
  dim3 grid((unsigned)a.n_items, (unsigned)(a.n / 128), (unsigned)(a.n / 256));
  if (kind == 0) {
    cudaFuncSetAttribute(k_gemm_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_gemm_tc<0><<<grid, 128, smem, st>>>(mAh, mBh, mAl, mBl, a, stages);
  } else {
    cudaFuncSetAttribute(k_gemm_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_gemm_tc<1><<<grid, 128, smem, st>>>(mAh, mBh, mAl, mBl, a, stages);
  }
  return cudaGetLastError();
}

}  // namespace mctrg
