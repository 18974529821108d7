// The batched SVD for callers that cannot allocate device memory.
//
// mctrg_svd_batched allocates its working rows with cudaMalloc and releases
// them with cudaFree, and cudaFree waits for the whole device.  Some callers
// cannot accept that: a program whose device memory is owned by another
// allocator (a framework's caching allocator that already holds nearly all
// of it), a latency-critical loop that must never stall the device, or code
// that is not allowed to call an allocator at all.  This variant runs the
// same kernels with its working memory in one fixed array compiled into the
// library, so it allocates nothing.
#include <cstdint>
#include <mutex>

#include "../../include/mctrg.h"
#include "common.cuh"
#include "kernels.h"

namespace mctrg {
cudaError_t svd_chunk(const double* M, int n, int64_t count, double* sigma, double* vt, int max_sweeps,
                      double* W, double* sig, int* perm, int* nnz, uint32_t* flags, cudaStream_t st);
}

namespace {

// Fixed working memory: 16 MiB on every device that loads the library, held
// until the process exits.  Word 0 collects the OR of the matrices' flags.
constexpr size_t kScratchBytes = size_t(16) << 20;
constexpr size_t kScratchDoubles = kScratchBytes / sizeof(double);
static __device__ __align__(256) double g_svd_scratch[kScratchDoubles];

constexpr int kMaxDevices = 256;
// One call at a time per process.  The array and this lock belong to one
// process (and one loaded copy of the library): calls from other processes
// have arrays of their own and are not serialized against these.
std::mutex g_lock;
double* g_scratch_addr[kMaxDevices] = {};  // device address of the array, per device

// The array's name is only a host-side stand-in; its device address is
// looked up once per device, with that device current.
int scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MCTRG_ECUDA;
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_svd_scratch) != cudaSuccess || !p) return MCTRG_ECUDA;
    g_scratch_addr[dev] = (double*)p;
  }
  *out = g_scratch_addr[dev];
  return MCTRG_OK;
}

__global__ void k_or_flags(const uint32_t* f, int64_t n) {
  uint32_t v = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v |= f[i];
  if (v) atomicOr((unsigned int*)&g_svd_scratch[0], v);
}

__global__ void k_clear_flag_word() { ((unsigned int*)&g_svd_scratch[0])[0] = 0u; }

// Wait for the work already queued on `st` before the caller releases the
// lock; returns `status` (the wait's own failure leaves nothing more to do).
int drain(cudaStream_t st, int status) {
  cudaStreamSynchronize(st);
  return status;
}

}  // namespace

extern "C" int mctrg_svd_batched_noalloc(const double* M, int n, int64_t batch, double* sigma, double* vt,
                                         int max_sweeps, void* stream) {
  if (!M || !sigma || n < 1 || batch < 1 || batch > (1 << 30)) return MCTRG_EINVAL;
  if (n > MCTRG_SVD_NOALLOC_MAX_N) return MCTRG_EINVAL;
  if (max_sweeps <= 0) max_sweeps = 40;
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(g_lock);
  double* base = nullptr;
  int s = scratch_for_current_device(&base);
  if (s != MCTRG_OK) return s;
  // per matrix: rows (n_pad x n), sorted values (n_pad), order (n_pad ints),
  // nonzero count (1 int) and flags (1 word), in double-sized slots
  const int np = n + (n & 1);
  const size_t per = (size_t)np * n + np + (np + 1) / 2 + 1;
  const size_t avail = kScratchDoubles - 1;
  const int64_t chunk = (int64_t)(avail / per);
  if (chunk < 1) return MCTRG_EINVAL;
  const int64_t C = chunk < batch ? chunk : batch;
  double* W = base + 1;
  double* sig = W + (size_t)C * np * n;
  int* perm = (int*)(sig + (size_t)C * np);
  int* nnz = perm + (size_t)C * np;
  uint32_t* flags = (uint32_t*)(nnz + C);
  k_clear_flag_word<<<1, 1, 0, st>>>();
  if (cudaGetLastError() != cudaSuccess) return drain(st, MCTRG_ECUDA);
  for (int64_t b0 = 0; b0 < batch; b0 += C) {
    const int64_t cnt = (C < batch - b0) ? C : batch - b0;
    // an error after work was queued returns only once that work has left
    // the shared array (drain), so the next call cannot race with it
    if (cudaMemsetAsync(flags, 0, sizeof(uint32_t) * cnt, st) != cudaSuccess) return drain(st, MCTRG_ECUDA);
    if (mctrg::svd_chunk(M + (size_t)b0 * n * n, n, cnt, sigma + (size_t)b0 * n,
                         vt ? vt + (size_t)b0 * n * n : nullptr, max_sweeps, W, sig, perm, nnz, flags,
                         st) != cudaSuccess)
      return drain(st, MCTRG_ECUDA);
    k_or_flags<<<1, 256, 0, st>>>(flags, cnt);
    if (cudaGetLastError() != cudaSuccess) return drain(st, MCTRG_ECUDA);
  }
  unsigned int word = 0;
  if (cudaMemcpyAsync(&word, base, sizeof(word), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return drain(st, MCTRG_ECUDA);
  if (cudaStreamSynchronize(st) != cudaSuccess) return MCTRG_ECUDA;
  return (word & mctrg::FLAG_NOCONV) ? MCTRG_ENOCONV : MCTRG_OK;
}
