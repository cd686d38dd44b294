// setup_kernels.cu -- one-time work at handle creation: CSR validation, the
// lossless float32 narrowing test of the matrix values, and the device-side
// transpose used by the adjoint (counting sort by column, then each row of
// A^T sorted by the original row index, so the result is deterministic).
#include <algorithm>

#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "internal.h"
#include "kernels.cuh"

namespace krylov {
namespace {

__global__ void validate_kernel(int n, int64_t nnz, const int* rp, const int* ci, int ncols, int* bad) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < n; i += stride) {
    const int a = rp[i], b = rp[i + 1];
    if (b < a || a < 0 || (int64_t)b > nnz) atomicOr(bad, 1);
  }
  if (tid == 0 && (rp[0] != 0 || (int64_t)rp[n] != nnz)) atomicOr(bad, 2);
  for (int64_t e = tid; e < nnz; e += stride) {
    const int c = ci[e];
    if (c < 0 || c >= ncols) atomicOr(bad, 4);
  }
}

__global__ void narrow_kernel(int64_t nnz, const double* v, float* v32, int* inexact) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += stride) {
    const float f = __double2float_rn(v[e]);
    v32[e] = f;
    if ((double)f != v[e]) atomicOr(inexact, 1);
  }
}

__global__ void split_kernel(int64_t nnz, const double* v, float2* vff) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += stride) {
    const float h = __double2float_rn(v[e]);
    vff[e] = make_float2(h, __double2float_rn(v[e] - (double)h));
  }
}

__global__ void count_cols_kernel(int64_t nnz, const int* ci, int* cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += stride) atomicAdd(&cnt[ci[e]], 1);
}

// Exclusive scan of n counts into rp (n+1) by one CTA: chunked serial sums.
__global__ void scan_kernel(int n, const int* cnt, int* rp) {
  __shared__ long long part[1024];
  const int T = blockDim.x, tid = threadIdx.x;
  const int chunk = (n + T - 1) / T;
  const int a = tid * chunk, b = min(n, a + chunk);
  long long s = 0;
  for (int i = a; i < b; ++i) s += cnt[i];
  part[tid] = s;
  __syncthreads();
  if (tid == 0) {
    long long acc = 0;
    for (int t = 0; t < T; ++t) {
      const long long v = part[t];
      part[t] = acc;
      acc += v;
    }
  }
  __syncthreads();
  long long acc = part[tid];
  for (int i = a; i < b; ++i) {
    rp[i] = (int)acc;
    acc += cnt[i];
  }
  if (tid == T - 1) rp[n] = (int)acc;
}

__global__ void scatter_kernel(int n, const int* rp, const int* ci, const double* v, const int* rpt, int* cursor,
                               int* cit, double* vt) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      const int c = ci[e];
      const int pos = rpt[c] + atomicAdd(&cursor[c], 1);
      cit[pos] = i;
      vt[pos] = v[e];
    }
  }
}

__global__ void sort_rows_kernel(int n, const int* rpt, int* cit, double* vt) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int a = rpt[i], b = rpt[i + 1];
    for (int e = a + 1; e < b; ++e) {
      const int kc = cit[e];
      const double kv = vt[e];
      int f = e - 1;
      while (f >= a && cit[f] > kc) {
        cit[f + 1] = cit[f];
        vt[f + 1] = vt[f];
        --f;
      }
      cit[f + 1] = kc;
      vt[f + 1] = kv;
    }
  }
}

// Largest 16-byte-aligned nonzero span of a 256-row tile (tiles start at
// multiples of 256): ((rp[end] + 3) & ~3) - (rp[start] & ~3).
// Largest nonzero span of a 256-row tile, both ends rounded out to multiples
// of 8 entries (the staged copies start on 16-byte boundaries for 2-byte
// column offsets as well as 4-byte columns).
__global__ void tile_span_kernel(int n, const int* rp, int* out) {
  const int stride = gridDim.x * blockDim.x;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; (int64_t)t * 256 < n; t += stride) {
    const int ts = t * 256;
    const int te = min(ts + 256, n);
    const int span = ((rp[te] + 7) & ~7) - (rp[ts] & ~7);
    atomicMax(out, span);
  }
}

// max over nonzeros of |col - row| (the bandwidth of the operator).
__global__ void band_kernel(int n, const int* rp, const int* ci, int* out) {
  const int stride = gridDim.x * blockDim.x;
  int b = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    for (int e = rp[i]; e < rp[i + 1]; ++e) b = max(b, abs(ci[e] - i));
  if (b > 0) atomicMax(out, b);
}

// dcol[e] = col[e] - row(e) (requires a bandwidth below 2^15).
__global__ void delta16_kernel(int n, const int* rp, const int* ci, int16_t* dcol) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    for (int e = rp[i]; e < rp[i + 1]; ++e) dcol[e] = (int16_t)(ci[e] - i);
}

// max_i sum_j |a_ij| (the infinity norm), as the bit pattern of a nonnegative
// double (which orders like the double itself).
__global__ void row_abs_sum_kernel(int n, const int* rp, const double* val, unsigned long long* out) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double acc = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) acc += fabs(val[e]);
    atomicMax(out, (unsigned long long)__double_as_longlong(acc));
  }
}

// Self-test of the bounded mbarrier wait that the staged kernels use.  Case 0
// waits on a phase that completes (one plain arrival), case 1 on a phase that
// never completes (16 transaction bytes announced, no copy issued: nothing
// will ever arrive).  out[c] = 1 if the wait of case c gave up, out[2 + c] =
// its duration in nanoseconds.  No copy is in flight at any time, so the CTA
// may leave with the phase of case 1 still open.
__global__ void wait_probe_kernel(unsigned long long limit_ns, unsigned long long* out) {
  __shared__ __align__(8) uint64_t bar[2];
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive(&bar[0]);
    mbar_arrive_expect_tx(&bar[1], 16);
    for (int c = 0; c < 2; ++c) {
      const uint64_t t0 = global_ns();
      const bool done = mbar_wait_bounded(&bar[c], 0u, limit_ns);
      out[c] = done ? 0ull : 1ull;
      out[2 + c] = global_ns() - t0;
    }
  }
}

}  // namespace

cudaError_t probe_bounded_wait(unsigned long long limit_ns, unsigned long long* d_out, cudaStream_t st) {
  wait_probe_kernel<<<1, 32, 0, st>>>(limit_ns, d_out);
  return cudaGetLastError();
}

// Raise (never lower) a kernel's dynamic shared-memory limit.  The limit is
// per function and context, so threads that launch the same kernel with
// different sizes (batched instances) must not undo each other's setting.
cudaError_t raise_smem_limit(const void* kern, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> cur;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& c = cur[{dev, kern}];
  if (bytes <= c) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) c = bytes;
  return e;
}

namespace {

int grid_for(int64_t work) {
  int64_t g = (work + 255) / 256;
  if (g < 1) g = 1;
  if (g > 8192) g = 8192;
  return (int)g;
}

}  // namespace

cudaError_t validate_csr(int n, int64_t nnz, const int* rp, const int* ci, int* d_flag, int* h_flag,
                         cudaStream_t st, int ncols) {
  cudaMemsetAsync(d_flag, 0, sizeof(int), st);
  validate_kernel<<<grid_for(std::max<int64_t>(n, nnz)), 256, 0, st>>>(n, nnz, rp, ci, ncols > 0 ? ncols : n,
                                                                        d_flag);
  cudaMemcpyAsync(h_flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  return cudaStreamSynchronize(st);
}

cudaError_t narrow_values(int64_t nnz, const double* v, float* v32, int* d_flag, int* h_flag, cudaStream_t st) {
  cudaMemsetAsync(d_flag, 0, sizeof(int), st);
  if (nnz > 0) narrow_kernel<<<grid_for(nnz), 256, 0, st>>>(nnz, v, v32, d_flag);
  cudaMemcpyAsync(h_flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  return cudaStreamSynchronize(st);
}

cudaError_t csr_bandwidth(int n, const int* rp, const int* ci, int* d_flag, int* h_flag, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(d_flag, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  band_kernel<<<grid_for(n), 256, 0, st>>>(n, rp, ci, d_flag);
  e = cudaMemcpyAsync(h_flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

cudaError_t csr_delta16(int n, const int* rp, const int* ci, int16_t* dcol, cudaStream_t st) {
  delta16_kernel<<<grid_for(n), 256, 0, st>>>(n, rp, ci, dcol);
  return cudaGetLastError();
}

cudaError_t tile_span_max(int n, const int* rp, int* d_flag, int* h_flag, cudaStream_t st) {
  cudaMemsetAsync(d_flag, 0, sizeof(int), st);
  tile_span_kernel<<<grid_for((n + 255) / 256), 256, 0, st>>>(n, rp, d_flag);
  cudaMemcpyAsync(h_flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  return cudaStreamSynchronize(st);
}

cudaError_t norm_inf(int n, const int* rp, const double* val, int* d_flag, int* h_flag, double* out,
                     cudaStream_t st) {
  unsigned long long* bits = reinterpret_cast<unsigned long long*>(d_flag);
  cudaMemsetAsync(bits, 0, sizeof(unsigned long long), st);
  row_abs_sum_kernel<<<grid_for(n), 256, 0, st>>>(n, rp, val, bits);
  cudaMemcpyAsync(h_flag, bits, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
  const cudaError_t e = cudaStreamSynchronize(st);
  std::memcpy(out, h_flag, sizeof(double));
  return e;
}

cudaError_t split_values(int64_t nnz, const double* v, float2* vff, cudaStream_t st) {
  if (nnz > 0) split_kernel<<<grid_for(nnz), 256, 0, st>>>(nnz, v, vff);
  return cudaGetLastError();
}

cudaError_t transpose_csr(int n, int64_t nnz, const int* rp, const int* ci, const double* v, int* rpt, int* cit,
                          double* vt, int* work, cudaStream_t st) {
  // work: 2n ints (counts, cursors)
  cudaMemsetAsync(work, 0, sizeof(int) * 2 * (size_t)n, st);
  if (nnz > 0) count_cols_kernel<<<grid_for(nnz), 256, 0, st>>>(nnz, ci, work);
  scan_kernel<<<1, 1024, 0, st>>>(n, work, rpt);
  scatter_kernel<<<grid_for(n), 256, 0, st>>>(n, rp, ci, v, rpt, work + n, cit, vt);
  sort_rows_kernel<<<grid_for(n), 256, 0, st>>>(n, rpt, cit, vt);
  return cudaGetLastError();
}

}  // namespace krylov
