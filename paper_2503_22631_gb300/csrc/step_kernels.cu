// step_kernels.cu -- the streaming kernels of one restart cycle.
//
// One launch of step_kernel handles basis column j of a cycle (Algorithm 1's
// loop body, with the truncated orthogonalization of Sec. 5 "incomplete" and
// the sketch of Sec. 2.1) in a single pass over the rows:
//
//   materialize   w_j = rho_j (p_{j-1} - sum_{q in win(j-1)} h_q w_q)
//                 (the orthogonalization of the previous product, rounded to
//                 the basis storage type and stored in slot j)
//   sketch        u_j += S e_i w_j[i] for the zeta entries of column i of S,
//                 generated in-kernel (Eq. 3), accumulated in shared memory
//   product       p_j = A w_j, where w_j at a neighbour column c is
//                 recomputed from p_{j-1}[c] and the window vectors at c with
//                 the same rounded arithmetic, so w_j is never re-read
//   dots          <w_q, p_j> for the window of the next column, ||p_j||^2,
//                 ||w_j||^2
//
// Basis vectors are stored unnormalized: rho_j only keeps ||w_j|| near 1
// (estimated from ||p||^2 - sum h_q^2 ||w_q||^2), the exact norm is reduced
// here and h_q = <w_q, p_j> / ||w_q||^2 are projection coefficients, so the
// Arnoldi-like relation A w_{j-1} = sum h_q w_q + w_j / rho_j (Eq. 5) holds
// for whatever rho_j was used.  Whitening absorbs the column scaling.
//
// Reductions are deterministic: per-CTA partials in a fixed slot, then the
// last CTA to arrive (atomic ticket) sums them in CTA order and writes the
// next column's coefficients.  The sketch partials stay per CTA and are
// summed once per cycle by sketch_reduce_kernel.
#include <cmath>

#include "internal.h"
#include "kernels.cuh"

namespace krylov {
namespace {

template <typename VT> struct Types {
  using A = float;   // arithmetic
  using P = float;   // raw product storage
  using Sk = float;  // sketch partials
};
template <> struct Types<double> {
  using A = double;
  using P = double;
  using Sk = double;
};

constexpr int NQ = 2 + MAX_WINDOW;  // scalar partials per CTA: ||w||^2, ||p||^2, dots

__device__ __forceinline__ void reducer_step(const StepLaunch& L, const CycleDev& cd,
                                             const double* tot, int mat, int spmv) {
  const int j = L.j;
  const double sig2 = tot[0];
  cd.sig2[j] = sig2;
  if (!isfinite(sig2)) cd.flags[2] |= ERR_NONFINITE;
  const int ldr = L.m + 1;  // R is (m+1) x m, column-major
  if (mat) {
    const double rho = cd.coef[(size_t)(j - 1) * (MAX_WINDOW + 1) + MAX_WINDOW];
    cd.R[(size_t)(j - 1) * ldr + j] = 1.0 / rho;
    const double rnorm = sqrt(sig2) / rho;
    const double pprev = cd.pi[j - 1];
    if (!(rnorm > L.thr * sqrt(pprev))) {
      if (cd.flags[1] == 0) {
        cd.flags[1] = 1;
        cd.flags[0] = j;
      }
    }
  }
  if (spmv && cd.flags[1] == 0) {
    const double pi = tot[1];
    cd.pi[j] = pi;
    if (!isfinite(pi)) cd.flags[2] |= ERR_NONFINITE;
    const int dlo = max(0, j - L.k + 1);
    double est = pi;
    double* c = cd.coef + (size_t)j * (MAX_WINDOW + 1);
    for (int q = 0; q < MAX_WINDOW; ++q) {
      const int slot = dlo + q;
      double h = 0.0;
      if (slot <= j) {
        const double s2 = cd.sig2[slot];
        h = (s2 > 0.0) ? tot[2 + q] / s2 : 0.0;
        est -= h * h * s2;
        cd.R[(size_t)j * ldr + slot] = h;
      }
      c[q] = h;
    }
    est = fmax(est, 1e-20 * pi);
    c[MAX_WINDOW] = (pi > 0.0) ? 1.0 / sqrt(est) : 1.0;
  }
}

template <typename VT, typename AT, bool MAT, bool SPMV, int ZM>
__global__ void __launch_bounds__(STEP_THREADS) step_kernel(const StepLaunch L, const CycleDev cd) {
  using A = typename Types<VT>::A;
  using P = typename Types<VT>::P;
  using Sk = typename Types<VT>::Sk;
  extern __shared__ __align__(16) unsigned char smem[];
  Sk* bins = reinterpret_cast<Sk*>(smem);
  __shared__ A red[32];
  __shared__ double tot[NQ];
  __shared__ int s_last;

  const int j = L.j;
  if (cd.flags[0] < j) return;  // an earlier column broke down

  const int nw = blockDim.x >> 5, wid = threadIdx.x >> 5;
  for (int e = threadIdx.x; e < nw * L.s; e += blockDim.x) bins[e] = Sk(0);
  __syncthreads();

  const VT* W = static_cast<const VT*>(L.W);
  VT* Wj = static_cast<VT*>(L.W) + (int64_t)j * L.ldw;
  const P* pprev = static_cast<const P*>(L.p_prev);
  const int lo = MAT ? max(0, j - L.k) : j;
  const int nl = j - lo;
  A h[MAX_WINDOW];
  A rho = A(1);
#pragma unroll
  for (int q = 0; q < MAX_WINDOW; ++q) h[q] = A(0);
  if (MAT) {
    const double* c = cd.coef + (size_t)(j - 1) * (MAX_WINDOW + 1);
#pragma unroll
    for (int q = 0; q < MAX_WINDOW; ++q) h[q] = (q < nl) ? A(c[q]) : A(0);
    rho = A(c[MAX_WINDOW]);
  }
  const int dlo = max(0, j - L.k + 1);
  const int nd = j - dlo + 1;
  const int off = dlo - lo;

  SketchSpec sp;
  sp.s = L.s;
  sp.zeta = L.zeta;
  sp.lim = 32768u - 32768u % (uint32_t)L.s;
  sp.k0 = (uint32_t)(L.seed & 0xFFFFFFFFull);
  sp.k1 = (uint32_t)(L.seed >> 32);
  sp.scale = 1.f;

  A acc_sig = A(0), acc_pi = A(0);
  A acc_dot[MAX_WINDOW];
#pragma unroll
  for (int q = 0; q < MAX_WINDOW; ++q) acc_dot[q] = A(0);
  int bad = 0;
  Sk* mybins = bins + wid * L.s;

  const int r0 = blockIdx.x * L.rows_per_cta;
  const int r1 = min(L.n, r0 + L.rows_per_cta);
  for (int i = r0 + (int)threadIdx.x; i < r1; i += blockDim.x) {
    A wl[MAX_WINDOW];
    A wj;
    if (MAT) {
      A acc = A(pprev[i]);
#pragma unroll
      for (int q = 0; q < MAX_WINDOW; ++q) {
        wl[q] = A(0);
        if (q < nl) {
          wl[q] = Store<VT>::load(W + (int64_t)(lo + q) * L.ldw + i);
          acc = fma_rn(-h[q], wl[q], acc);
        }
      }
      wj = stored<VT, A>(mul_rn(acc, rho));
      Store<VT>::put(Wj + i, wj);
    } else {
#pragma unroll
      for (int q = 0; q < MAX_WINDOW; ++q) wl[q] = A(0);
      wj = Store<VT>::load(Wj + i);
    }
    acc_sig = fma_rn(wj, wj, acc_sig);

    const Sk wv = Sk(wj);
    const int got = sketch_column<ZM>((uint32_t)i, sp, [&](int row, bool neg) {
      atomicAdd(&mybins[row], neg ? -wv : wv);
    });
    bad |= (got < L.zeta);

    if (SPMV) {
      const int e0 = L.row_ptr[i], e1 = L.row_ptr[i + 1];
      A accp = A(0);
      for (int e = e0; e < e1; ++e) {
        const int c = L.col[e];
        const A av = A(static_cast<const AT*>(L.val)[e]);
        A wc;
        if (MAT) {
          A t = A(pprev[c]);
#pragma unroll
          for (int q = 0; q < MAX_WINDOW; ++q)
            if (q < nl) t = fma_rn(-h[q], A(Store<VT>::load(W + (int64_t)(lo + q) * L.ldw + c)), t);
          wc = stored<VT, A>(mul_rn(t, rho));
        } else {
          wc = Store<VT>::load(Wj + c);
        }
        accp = fma_rn(av, wc, accp);
      }
      const P pst = P(accp);
      static_cast<P*>(L.p_out)[i] = pst;
      const A pv = A(pst);
      acc_pi = fma_rn(pv, pv, acc_pi);
#pragma unroll
      for (int q = 0; q < MAX_WINDOW; ++q) {
        if (q < nd) {
          A wq = wj;
          if (dlo + q != j) {
#pragma unroll
            for (int r = 0; r < MAX_WINDOW; ++r)
              if (r == q + off) wq = wl[r];
          }
          acc_dot[q] = fma_rn(wq, pv, acc_dot[q]);
        }
      }
    }
  }

  // ---- CTA partials ----
  double* part = L.part + (size_t)blockIdx.x * NQ;
  {
    A v = block_sum(acc_sig, red);
    if (threadIdx.x == 0) part[0] = double(v);
    v = block_sum(acc_pi, red);
    if (threadIdx.x == 0) part[1] = double(v);
#pragma unroll
    for (int q = 0; q < MAX_WINDOW; ++q) {
      v = block_sum(acc_dot[q], red);
      if (threadIdx.x == 0) part[2 + q] = double(v);
    }
  }
  __syncthreads();
  Sk* out = static_cast<Sk*>(L.sk_part) + (size_t)blockIdx.x * L.s;
  for (int b = threadIdx.x; b < L.s; b += blockDim.x) {
    Sk acc = Sk(0);
    for (int w = 0; w < nw; ++w) acc += bins[w * L.s + b];
    out[b] = acc;
  }
  if (bad) atomicOr(&cd.flags[2], ERR_SKETCH);

  // ---- last CTA reduces the scalars in CTA order ----
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(cd.counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x < NQ) {
    double acc = 0.0;
    for (int c = 0; c < (int)gridDim.x; ++c) acc += __ldcg(L.part + (size_t)c * NQ + threadIdx.x);
    tot[threadIdx.x] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    reducer_step(L, cd, tot, MAT ? 1 : 0, SPMV ? 1 : 0);
    *cd.counter = 0u;
  }
}

template <typename VT, typename AT, bool MAT, bool SPMV>
void launch_step_t(const StepLaunch& L, const CycleDev& cd, int m, cudaStream_t st) {
  using Sk = typename Types<VT>::Sk;
  const size_t smem = (size_t)(STEP_THREADS / 32) * L.s * sizeof(Sk);
  if (L.zeta <= 8) {
    auto k = step_kernel<VT, AT, MAT, SPMV, 8>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<L.grid, STEP_THREADS, smem, st>>>(L, cd);
  } else {
    auto k = step_kernel<VT, AT, MAT, SPMV, MAX_ZETA>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<L.grid, STEP_THREADS, smem, st>>>(L, cd);
  }
}

template <typename VT, typename AT>
void dispatch_mat(const StepLaunch& L, const CycleDev& cd, int m, cudaStream_t st) {
  if (L.mat && L.spmv) launch_step_t<VT, AT, true, true>(L, cd, m, st);
  else if (L.mat) launch_step_t<VT, AT, true, false>(L, cd, m, st);
  else if (L.spmv) launch_step_t<VT, AT, false, true>(L, cd, m, st);
  else launch_step_t<VT, AT, false, false>(L, cd, m, st);
}

// ---------------------------------------------------------------------------
__device__ __forceinline__ bool last_block(unsigned* counter, int* s_last) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) *s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (*s_last) __threadfence();
  return *s_last != 0;
}

__global__ void norm_b_kernel(const double* b, int n, double* part, CycleDev cd, int rows_per_cta) {
  __shared__ double red[32];
  __shared__ int s_last;
  double acc = 0.0;
  const int r0 = blockIdx.x * rows_per_cta, r1 = min(n, r0 + rows_per_cta);
  for (int i = r0 + (int)threadIdx.x; i < r1; i += blockDim.x) acc = fma(b[i], b[i], acc);
  const double v = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = v;
  if (!last_block(cd.counter, &s_last)) return;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int c = 0; c < (int)gridDim.x; ++c) t += __ldcg(part + c);
    cd.scal[4] = t;
    const double eta = sqrt(t);
    cd.scal[0] = eta;
    cd.scal[1] = (eta > 0.0) ? 1.0 / eta : 0.0;
    if (!isfinite(t)) cd.flags[2] |= ERR_NONFINITE;
    *cd.counter = 0u;
  }
}

template <typename VT>
__global__ void start_kernel(const double* b, VT* W0, int n, CycleDev cd) {
  const double inv = cd.scal[1];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double v = b[i] * inv;
    if constexpr (sizeof(VT) == 8) W0[i] = v;
    else Store<VT>::put(W0 + i, __double2float_rn(v));
  }
}

// Cycle end: x += W_m z and the next start vector v = (w_{m+1} - W_m g) / tau
// (written into slot 0), with ||y||^2 and ||x||^2 reduced for the stop test.
template <typename VT>
__global__ void __launch_bounds__(STEP_THREADS) update_kernel(VT* W, int64_t ldw, int n, int m_eff,
                                                              int has_next, const double* zg, int m,
                                                              double* x, double* part, CycleDev cd,
                                                              int rows_per_cta) {
  __shared__ double zs[256], gs[256];
  __shared__ double red[32];
  __shared__ int s_last;
  for (int q = threadIdx.x; q < m_eff; q += blockDim.x) {
    zs[q] = zg[q];
    gs[q] = zg[m + q];
  }
  const double tau_inv = zg[2 * m];
  __syncthreads();
  double ay = 0.0, ax = 0.0;
  const int r0 = blockIdx.x * rows_per_cta, r1 = min(n, r0 + rows_per_cta);
  for (int i = r0 + (int)threadIdx.x; i < r1; i += blockDim.x) {
    double y = 0.0;
    double v = has_next ? double(Store<VT>::load(W + (int64_t)m_eff * ldw + i)) : 0.0;
    for (int q = 0; q < m_eff; ++q) {
      const double w = double(Store<VT>::load(W + (int64_t)q * ldw + i));
      y = fma(w, zs[q], y);
      v = fma(-w, gs[q], v);
    }
    const double xn = x[i] + y;
    x[i] = xn;
    if (has_next) {
      const double vn = v * tau_inv;
      if constexpr (sizeof(VT) == 8) W[i] = vn;
      else Store<VT>::put(W + i, __double2float_rn(vn));
    }
    ay = fma(y, y, ay);
    ax = fma(xn, xn, ax);
  }
  double v = block_sum(ay, red);
  if (threadIdx.x == 0) part[2 * blockIdx.x] = v;
  v = block_sum(ax, red);
  if (threadIdx.x == 0) part[2 * blockIdx.x + 1] = v;
  if (!last_block(cd.counter, &s_last)) return;
  if (threadIdx.x < 2) {
    double t = 0.0;
    for (int c = 0; c < (int)gridDim.x; ++c) t += __ldcg(part + 2 * c + threadIdx.x);
    cd.scal[2 + threadIdx.x] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) *cd.counter = 0u;
}

template <typename Sk>
__global__ void sketch_reduce_kernel(const Sk* part, int ncols, int grid, int s, double scale,
                                     int64_t col_stride, double* U) {
  const int j = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ncols || r >= s) return;
  const Sk* p = part + (size_t)j * col_stride;
  double acc = 0.0;
  for (int c = 0; c < grid; ++c) acc += double(p[(size_t)c * s + r]);
  U[(size_t)j * s + r] = acc * scale;
}

__global__ void spmv_f64_kernel(int n, const int* rp, const int* ci, const double* val, const double* x,
                                double* y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) acc = fma(val[e], x[ci[e]], acc);
    y[i] = acc;
  }
}

__global__ void dot_f64_kernel(const double* a, const double* b, int n, double* part, double* out,
                               unsigned* counter, int rows_per_cta) {
  __shared__ double red[32];
  __shared__ int s_last;
  double acc = 0.0;
  const int r0 = blockIdx.x * rows_per_cta, r1 = min(n, r0 + rows_per_cta);
  for (int i = r0 + (int)threadIdx.x; i < r1; i += blockDim.x) acc = fma(a[i], b[i], acc);
  const double v = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = v;
  if (!last_block(counter, &s_last)) return;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int c = 0; c < (int)gridDim.x; ++c) t += __ldcg(part + c);
    *out = t;
    *counter = 0u;
  }
}

__global__ void sketch_columns_kernel(int64_t col0, int64_t count, SketchSpec sp, int* rows,
                                      signed char* signs, int* err) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  int e = 0;
  int* rr = rows + t * sp.zeta;
  signed char* ss = signs + t * sp.zeta;
  const int got = sketch_column<MAX_ZETA>((uint32_t)(col0 + t), sp, [&](int row, bool neg) {
    rr[e] = row;
    ss[e] = neg ? (signed char)-1 : (signed char)1;
    ++e;
  });
  if (got < sp.zeta) atomicOr(err, ERR_SKETCH);
}

}  // namespace

namespace {
template <typename VT, typename AT>
int occupancy_t(int zeta, int s) {
  using Sk = typename Types<VT>::Sk;
  const size_t smem = (size_t)(STEP_THREADS / 32) * s * sizeof(Sk);
  int blocks = 0;
  if (zeta <= 8) {
    auto k = step_kernel<VT, AT, true, true, 8>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, STEP_THREADS, smem);
  } else {
    auto k = step_kernel<VT, AT, true, true, MAX_ZETA>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, STEP_THREADS, smem);
  }
  return blocks < 1 ? 1 : blocks;
}
}  // namespace

// Resident CTAs per SM of the main step kernel (one persistent wave).
int step_ctas_per_sm(int basis, int zeta, int s, int vals_f32) {
  if (basis == 0) return vals_f32 ? occupancy_t<double, float>(zeta, s) : occupancy_t<double, double>(zeta, s);
  if (basis == 1) return occupancy_t<float, float>(zeta, s);
  return occupancy_t<__nv_bfloat16, float>(zeta, s);
}

void launch_step(int basis, const StepLaunch& L, const CycleDev& cd, int m, cudaStream_t st) {
  if (basis == 0) {
    if (L.val_f32) dispatch_mat<double, float>(L, cd, m, st);
    else dispatch_mat<double, double>(L, cd, m, st);
  } else if (basis == 1) {
    dispatch_mat<float, float>(L, cd, m, st);
  } else {
    dispatch_mat<__nv_bfloat16, float>(L, cd, m, st);
  }
}

void launch_norm_b(const double* b, int n, double* part, int grid, const CycleDev& cd, cudaStream_t st) {
  const int rpc = (n + grid - 1) / grid;
  norm_b_kernel<<<grid, STEP_THREADS, 0, st>>>(b, n, part, cd, rpc);
}

void launch_start(int basis, const double* b, void* W0, int n, const CycleDev& cd, int grid,
                  cudaStream_t st) {
  if (basis == 0) start_kernel<double><<<grid, STEP_THREADS, 0, st>>>(b, (double*)W0, n, cd);
  else if (basis == 1) start_kernel<float><<<grid, STEP_THREADS, 0, st>>>(b, (float*)W0, n, cd);
  else start_kernel<__nv_bfloat16><<<grid, STEP_THREADS, 0, st>>>(b, (__nv_bfloat16*)W0, n, cd);
}

void launch_update(int basis, void* W, int64_t ldw, int n, int m_eff, int has_next, const double* zg,
                   double* x, double* part, int grid, const CycleDev& cd, int m, cudaStream_t st) {
  const int rpc = (n + grid - 1) / grid;
  if (basis == 0)
    update_kernel<double><<<grid, STEP_THREADS, 0, st>>>((double*)W, ldw, n, m_eff, has_next, zg, m, x,
                                                          part, cd, rpc);
  else if (basis == 1)
    update_kernel<float><<<grid, STEP_THREADS, 0, st>>>((float*)W, ldw, n, m_eff, has_next, zg, m, x,
                                                         part, cd, rpc);
  else
    update_kernel<__nv_bfloat16><<<grid, STEP_THREADS, 0, st>>>((__nv_bfloat16*)W, ldw, n, m_eff,
                                                                 has_next, zg, m, x, part, cd, rpc);
}

void launch_sketch_reduce(int basis, const void* sk_part, int ncols, int grid, int s, int zeta,
                          int64_t col_stride, double* U, cudaStream_t st) {
  dim3 g((s + 127) / 128, ncols);
  const double scale = 1.0 / std::sqrt((double)zeta);
  if (basis == 0)
    sketch_reduce_kernel<double><<<g, 128, 0, st>>>((const double*)sk_part, ncols, grid, s, scale,
                                                    col_stride, U);
  else
    sketch_reduce_kernel<float><<<g, 128, 0, st>>>((const float*)sk_part, ncols, grid, s, scale,
                                                   col_stride, U);
}

void launch_spmv_f64(int n, const int* row_ptr, const int* col, const double* val, const double* x,
                     double* y, cudaStream_t st) {
  const int grid = std::max(1, std::min(4096, (n + 255) / 256));
  spmv_f64_kernel<<<grid, 256, 0, st>>>(n, row_ptr, col, val, x, y);
}

void launch_dot_f64(const double* a, const double* b, int n, double* part, int grid, double* out,
                    unsigned* counter, cudaStream_t st) {
  const int rpc = (n + grid - 1) / grid;
  dot_f64_kernel<<<grid, STEP_THREADS, 0, st>>>(a, b, n, part, out, counter, rpc);
}

void launch_sketch_columns(int64_t col0, int64_t count, int s, int zeta, uint64_t seed, int* rows,
                           signed char* signs, int* err, cudaStream_t st) {
  SketchSpec sp;
  sp.s = s;
  sp.zeta = zeta;
  sp.lim = 32768u - 32768u % (uint32_t)s;
  sp.k0 = (uint32_t)(seed & 0xFFFFFFFFull);
  sp.k1 = (uint32_t)(seed >> 32);
  sp.scale = 1.f;
  const int grid = (int)((count + 255) / 256);
  if (grid > 0) sketch_columns_kernel<<<grid, 256, 0, st>>>(col0, count, sp, rows, signs, err);
}

}  // namespace krylov

namespace krylov {
namespace {
__global__ void cycle_reset_kernel(CycleDev cd, int m) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    cd.flags[0] = m;
    cd.flags[1] = 0;
  }
}
}  // namespace
void launch_cycle_reset(const CycleDev& cd, int m, cudaStream_t st) { cycle_reset_kernel<<<1, 32, 0, st>>>(cd, m); }
}  // namespace krylov
