// noalloc.cu -- y = A x and <d, y> for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the moment they need this product:
// numerical code called back from inside a custom device memory pool or
// allocator (a nested allocation would re-enter the allocator that is running),
// and real-time loops in which cudaMalloc may block on the driver or
// synchronize the device.  This entry point therefore allocates nothing: the caller passes the
// matrix, the input and the outputs as device pointers, and the only scratch
// memory (per-CTA partial sums of the dot product and the arrival counter of
// the final reduction) is the file-scope device array below, which exists on
// every GPU that loads the library until the process exits.
//
// Set-up: the first call on a device (with that device current) resolves the
// array's device address with cudaGetSymbolAddress; make that first call
// before any stream capture (a first call on a capturing stream is refused
// with KRYLOV_EINVAL).  All calls share the array and it keeps the
// contents of the last call: the counter is cleared at the start of every
// call, and two calls whose work overlaps on the GPU (different streams,
// different host threads) race on it -- serialize them.
#include <algorithm>
#include <climits>
#include <mutex>

#include "../../include/krylov.h"
#include "kernels.cuh"

namespace {

constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_MAX_CTAS = 2048;  // partials: 2048 doubles = 16 KiB

struct NoallocScratch {
  double part[NOALLOC_MAX_CTAS];
  unsigned counter;
};

// The scratch: 16 KiB + 4 bytes per device (modest, fixed maximum size).
static __device__ __align__(256) NoallocScratch krylov_noalloc_scratch;

__global__ void __launch_bounds__(NOALLOC_THREADS) spmv_dot_noalloc_kernel(
    int n, const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ val,
    const double* __restrict__ x, double* __restrict__ y, const double* __restrict__ d, double* dot_out,
    NoallocScratch* scr, int rows_per_cta) {
  __shared__ double red[32];
  __shared__ int s_last;
  // 64-bit row indices: r0 + rows_per_cta and i + blockDim.x may pass INT_MAX
  // for n near the limit; CTAs past the last row (the grid is capped, so
  // rows_per_cta is rounded up) have an empty range and add 0 to the dot.
  const long long r0 = (long long)blockIdx.x * rows_per_cta;
  const long long r1 = min((long long)n, r0 + rows_per_cta);
  double acc = 0.0;
  for (long long i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    double yi = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) yi = fma(val[e], x[ci[e]], yi);
    y[i] = yi;
    if (d) acc = fma(d[i], yi, acc);
  }
  if (!d) return;
  const double v = krylov::block_sum(acc, red);
  if (threadIdx.x == 0) scr->part[blockIdx.x] = v;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(&scr->counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const double t = (threadIdx.x < 32) ? krylov::warp_sum_partials(scr->part, (int)gridDim.x, 1, 0) : 0.0;
  if (threadIdx.x == 0) {
    *dot_out = t;
    scr->counter = 0u;
  }
}

std::mutex g_setup_mutex;
NoallocScratch* g_scratch_ptr[256] = {nullptr};

}  // namespace

extern "C" krylov_status krylov_spmv_dot_noalloc(int64_t n, int64_t nnz, const int32_t* row_ptr,
                                                 const int32_t* col_idx, const double* val, const double* x,
                                                 double* y, const double* dot_with, double* dot_out,
                                                 void* stream) {
  if (n < 1 || n > INT_MAX - 1 || nnz < 0 || nnz > INT_MAX) return KRYLOV_EINVAL;
  if (!row_ptr || !x || !y || (nnz > 0 && (!col_idx || !val))) return KRYLOV_EINVAL;
  if ((dot_with == nullptr) != (dot_out == nullptr)) return KRYLOV_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return KRYLOV_ECUDA;
  NoallocScratch* scr = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
      // the symbol lookup may load the module, which is not allowed while the
      // stream is being captured: refuse instead of invalidating the capture
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      if (cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cs) != cudaSuccess) return KRYLOV_ECUDA;
      if (cs != cudaStreamCaptureStatusNone) return KRYLOV_EINVAL;
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, krylov_noalloc_scratch) != cudaSuccess || p == nullptr) return KRYLOV_ECUDA;
      g_scratch_ptr[dev] = static_cast<NoallocScratch*>(p);
    }
    scr = g_scratch_ptr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int grid = (int)std::min<int64_t>(NOALLOC_MAX_CTAS, (n + NOALLOC_THREADS - 1) / NOALLOC_THREADS);
  const int rows_per_cta = (int)((n + grid - 1) / grid);
  if (dot_with && cudaMemsetAsync(&scr->counter, 0, sizeof(unsigned), st) != cudaSuccess) return KRYLOV_ECUDA;
  spmv_dot_noalloc_kernel<<<grid, NOALLOC_THREADS, 0, st>>>((int)n, row_ptr, col_idx, val, x, y, dot_with,
                                                            dot_out, scr, rows_per_cta);
  if (cudaGetLastError() != cudaSuccess) return KRYLOV_ECUDA;
  return KRYLOV_OK;
}
