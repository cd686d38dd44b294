// cycle_kernels.cu -- the streaming kernels around the Arnoldi steps of a
// restart cycle, and the sparse-sign table.
//
//   norm_b_kernel         ||b|| (cycle 1 start, Algorithm 2 line 2 with the
//                         truncated mode's w_1 = b / ||b||)
//   start_kernel          w_1 = b / ||b|| in the basis storage type
//   update_kernel         cycle end (Algorithm 2, solution update):
//                         x += W_m z and the next start vector
//                         v = (w_{m+1} - W_m g) / tau of the whitened restart
//   sketch_reduce_kernel  U[:, j] = (1/sqrt(zeta)) * sum over CTAs of the
//                         per-CTA sketch partials, in CTA order
//   sketch_table_kernel   the sparse sign embedding S of Sec. 2.1, Eq. (3),
//                         generated once per handle with the counter-based
//                         generator (S is likewise generated once per run and
//                         stored in App. A)
#include <algorithm>
#include <climits>
#include <cmath>

#include "internal.h"
#include "kernels.cuh"

namespace krylov {
namespace {

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
  const double t = (threadIdx.x < 32) ? warp_sum_partials(part, (int)gridDim.x, 1, 0) : 0.0;
  if (threadIdx.x == 0) {
    cd.scal[4] = t;
    const double eta = sqrt(t);
    cd.scal[0] = eta;
    cd.scal[1] = (eta > 0.0) ? 1.0 / eta : 0.0;
    cd.scal[5] = 1.0;  // w_1 = b / ||b||
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

__global__ void ff_start_kernel(const double* b, float2* W0, int n, CycleDev cd) {
  const double inv = cd.scal[1];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const ff v = ff_from_double(b[i] * inv);
    W0[i] = make_float2(v.hi, v.lo);
  }
}

// Compensated accumulation of products (float-float): S + E tracks sum a * w.
struct ffsum {
  float S = 0.f, E = 0.f;
  __device__ __forceinline__ void add_prod(ff a, ff w) {
    const float p = __fmul_rn(a.hi, w.hi);
    float e = __fmaf_rn(a.hi, w.hi, -p);
    e = __fmaf_rn(a.hi, w.lo, e);
    e = __fmaf_rn(a.lo, w.hi, e);
    const ff t = two_sum(S, p);
    S = t.hi;
    E = __fadd_rn(E, __fadd_rn(t.lo, e));
  }
  __device__ __forceinline__ ff result() const { return fast_two_sum(S, E); }
};

// Cycle end for the float64 / float32 / bfloat16 bases: x += W_m z and the
// next start vector v = (w_{m+1} - W_m g) tau^{-1}, one pass over the basis.
// Basis slices are loaded UPD_BATCH at a time (all in flight before use).
// float64: float64 arithmetic.  float32 / bfloat16: products of the stored
// value with z (and g) held as float-float pairs, summed with error-free
// transformations on the FP32 pipes (the result is float64-accurate for the
// stored basis; float64 FMAs here would make the pass FP64-bound on GB300).
constexpr int UPD_BATCH = 8;

template <typename VT>
__global__ void __launch_bounds__(STEP_THREADS) update_kernel(VT* W, int64_t ldw, int n, int m_eff,
                                                              int has_next, const double* zg, int m,
                                                              double* x, double* part, CycleDev cd,
                                                              int rows_per_cta) {
  constexpr bool WIDE = sizeof(VT) == 8;
  __shared__ double zs[256], gs[256];
  __shared__ ff zf[256], gf[256];
  __shared__ double red[32];
  __shared__ int s_last, s_ez;
  // z enters the float pairs scaled by 2^-ez (max |z| in [1, 2)): a tiny
  // update (z ~ 1e-50 for a very stiff first cycle) must not underflow in
  // float; the sum is scaled back in float64
  if (threadIdx.x == 0) s_ez = INT_MIN;
  __syncthreads();
  for (int q = threadIdx.x; q < m_eff; q += blockDim.x)
    if (zg[q] != 0.0 && isfinite(zg[q])) atomicMax(&s_ez, ilogb(zg[q]));
  __syncthreads();
  const int ez = (s_ez == INT_MIN) ? 0 : s_ez;
  for (int q = threadIdx.x; q < m_eff; q += blockDim.x) {
    zs[q] = zg[q];
    gs[q] = zg[m + q];
    zf[q] = ff_from_double(ldexp(zg[q], -ez));
    gf[q] = ff_neg(ff_from_double(zg[m + q]));
  }
  const double tau_inv = zg[2 * m];
  __syncthreads();
  double ay = 0.0, ax = 0.0, av = 0.0;
  const int r0 = blockIdx.x * rows_per_cta, r1 = min(n, r0 + rows_per_cta);
  for (int i = r0 + (int)threadIdx.x; i < r1; i += blockDim.x) {
    double y, v;
    if constexpr (WIDE) {
      y = 0.0;
      v = has_next ? double(Store<VT>::load(W + (int64_t)m_eff * ldw + i)) : 0.0;
      for (int q0 = 0; q0 < m_eff; q0 += UPD_BATCH) {
        double wv[UPD_BATCH];
#pragma unroll
        for (int u = 0; u < UPD_BATCH; ++u)
          if (q0 + u < m_eff) wv[u] = double(Store<VT>::load(W + (int64_t)(q0 + u) * ldw + i));
#pragma unroll
        for (int u = 0; u < UPD_BATCH; ++u)
          if (q0 + u < m_eff) {
            y = fma(wv[u], zs[q0 + u], y);
            v = fma(-wv[u], gs[q0 + u], v);
          }
      }
    } else {
      ffsum fy, fv;
      if (has_next) fv.S = Store<VT>::load(W + (int64_t)m_eff * ldw + i);
      for (int q0 = 0; q0 < m_eff; q0 += UPD_BATCH) {
        float wv[UPD_BATCH];
#pragma unroll
        for (int u = 0; u < UPD_BATCH; ++u)
          if (q0 + u < m_eff) wv[u] = Store<VT>::load(W + (int64_t)(q0 + u) * ldw + i);
#pragma unroll
        for (int u = 0; u < UPD_BATCH; ++u)
          if (q0 + u < m_eff) {
            const ff w{wv[u], 0.f};
            fy.add_prod(zf[q0 + u], w);
            if (has_next) fv.add_prod(gf[q0 + u], w);
          }
      }
      const ff ry = fy.result(), rv = fv.result();
      y = ldexp((double)ry.hi + (double)ry.lo, ez);
      v = (double)rv.hi + (double)rv.lo;
    }
    const double xn = x[i] + y;
    x[i] = xn;
    if (has_next) {
      const double vn = v * tau_inv;
      double vs;
      if constexpr (WIDE) {
        W[i] = vn;
        vs = vn;
      } else {
        const float f = __double2float_rn(vn);
        Store<VT>::put(W + i, f);
        vs = (double)stored<VT, float>(f);
      }
      av = fma(vs, vs, av);
    }
    ay = fma(y, y, ay);
    ax = fma(xn, xn, ax);
  }
  double v = block_sum(ay, red);
  if (threadIdx.x == 0) part[3 * blockIdx.x] = v;
  v = block_sum(ax, red);
  if (threadIdx.x == 0) part[3 * blockIdx.x + 1] = v;
  v = block_sum(av, red);
  if (threadIdx.x == 0) part[3 * blockIdx.x + 2] = v;
  if (!last_block(cd.counter, &s_last)) return;
  if (threadIdx.x < 96) {  // warp q sums column q
    const int q = (int)(threadIdx.x >> 5);
    const double t = warp_sum_partials(part, (int)gridDim.x, 3, q);
    if ((threadIdx.x & 31) == 0) cd.scal[q < 2 ? 2 + q : 5] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) *cd.counter = 0u;
}

// Cycle end for the float-float basis (x stays float64).
__global__ void __launch_bounds__(STEP_THREADS) ff_update_kernel(float2* W, int64_t ldw, int n, int m_eff,
                                                                 int has_next, const double* zg, int m, double* x,
                                                                 double* part, CycleDev cd, int rows_per_cta) {
  __shared__ ff zs[256], gs[256];
  __shared__ double red[32];
  __shared__ int s_last, s_ez;
  // z scaled by 2^-ez in the float pairs (see update_kernel), scaled back in float64
  if (threadIdx.x == 0) s_ez = INT_MIN;
  __syncthreads();
  for (int q = threadIdx.x; q < m_eff; q += blockDim.x)
    if (zg[q] != 0.0 && isfinite(zg[q])) atomicMax(&s_ez, ilogb(zg[q]));
  __syncthreads();
  const int ez = (s_ez == INT_MIN) ? 0 : s_ez;
  for (int q = threadIdx.x; q < m_eff; q += blockDim.x) {
    zs[q] = ff_from_double(ldexp(zg[q], -ez));
    gs[q] = ff_neg(ff_from_double(zg[m + q]));
  }
  const ff tau_inv = ff_from_double(zg[2 * m]);
  __syncthreads();
  // squared norms in float64: a float square of a tiny update would underflow
  // to zero and read as a converged cycle
  double ay = 0.0, ax = 0.0, av = 0.0;
  const int r0 = blockIdx.x * rows_per_cta, r1 = min(n, r0 + rows_per_cta);
  for (int i = r0 + (int)threadIdx.x; i < r1; i += blockDim.x) {
    ffsum y, v;
    if (has_next) {
      const float2 wm = W[(int64_t)m_eff * ldw + i];
      v.S = wm.x;
      v.E = wm.y;
    }
    for (int q0 = 0; q0 < m_eff; q0 += UPD_BATCH) {
      float2 wv[UPD_BATCH];
#pragma unroll
      for (int u = 0; u < UPD_BATCH; ++u)
        if (q0 + u < m_eff) wv[u] = W[(int64_t)(q0 + u) * ldw + i];
#pragma unroll
      for (int u = 0; u < UPD_BATCH; ++u)
        if (q0 + u < m_eff) {
          const ff w{wv[u].x, wv[u].y};
          y.add_prod(zs[q0 + u], w);
          if (has_next) v.add_prod(gs[q0 + u], w);
        }
    }
    const ff yy = y.result();
    const double yd = ldexp((double)yy.hi + (double)yy.lo, ez);
    const double xn = x[i] + yd;
    x[i] = xn;
    if (has_next) {
      const ff vn = ff_mul(v.result(), tau_inv);
      W[i] = make_float2(vn.hi, vn.lo);
      av = fma((double)vn.hi, (double)vn.hi, av);
    }
    ay = fma(yd, yd, ay);
    ax = fma(xn, xn, ax);
  }
  double v = block_sum(ay, red);
  if (threadIdx.x == 0) part[3 * blockIdx.x] = v;
  v = block_sum(ax, red);
  if (threadIdx.x == 0) part[3 * blockIdx.x + 1] = v;
  v = block_sum(av, red);
  if (threadIdx.x == 0) part[3 * blockIdx.x + 2] = v;
  if (!last_block(cd.counter, &s_last)) return;
  if (threadIdx.x < 96) {  // warp q sums column q
    const int q = (int)(threadIdx.x >> 5);
    const double t = warp_sum_partials(part, (int)gridDim.x, 3, q);
    if ((threadIdx.x & 31) == 0) cd.scal[q < 2 ? 2 + q : 5] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) *cd.counter = 0u;
}

// U[:, j] = scale * sum over CTAs of the per-CTA sketch partials of column j.
// Block (32 x SR_GROUPS): thread (x, y) sums CTAs y, y + SR_GROUPS, ... of
// sketch row 32 blockIdx.x + x; the SR_GROUPS partial sums are then added in
// group order (deterministic).
constexpr int SR_GROUPS = 8;
template <typename Sk>
__global__ void sketch_reduce_kernel(const Sk* part, int ncols, int grid, int s, double scale,
                                     int64_t col_stride, double* U) {
  __shared__ double acc_g[SR_GROUPS][32];
  const int j = blockIdx.y;
  const int r = blockIdx.x * 32 + (int)threadIdx.x;
  double acc = 0.0;
  if (j < ncols && r < s) {
    const Sk* p = part + (size_t)j * col_stride;
#pragma unroll 4
    for (int c = (int)threadIdx.y; c < grid; c += SR_GROUPS) acc += double(p[(size_t)c * s + r]);
  }
  acc_g[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && j < ncols && r < s) {
    double t = 0.0;
    for (int g = 0; g < SR_GROUPS; ++g) t += acc_g[g][threadIdx.x];
    U[(size_t)j * s + r] = t * scale;
  }
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
  const double t = (threadIdx.x < 32) ? warp_sum_partials(part, (int)gridDim.x, 1, 0) : 0.0;
  if (threadIdx.x == 0) {
    *out = t;
    *counter = 0u;
  }
}

// Columns of S generated by the same routine the step kernels use when they
// regenerate S (packed path for s <= 255, zeta <= 8; generic otherwise).
__global__ void sketch_columns_kernel(int64_t col0, int64_t count, SketchSpec sp, int* rows,
                                      signed char* signs, int* err) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  int* rr = rows + t * sp.zeta;
  signed char* ss = signs + t * sp.zeta;
  int got;
  if (sp.s <= 255 && sp.zeta <= 8) {
    uint32_t p0, p1, ng;
    got = sketch_column_packed((uint32_t)(col0 + t), sp, sketch_inv_s(sp.s), &p0, &p1, &ng);
    for (int e = 0; e < got; ++e) {
      rr[e] = (int)(((e < 4 ? p0 : p1) >> (8 * (e & 3))) & 0xFFu);
      ss[e] = ((ng >> e) & 1u) ? (signed char)-1 : (signed char)1;
    }
  } else {
    int e = 0;
    got = sketch_column<MAX_ZETA>((uint32_t)(col0 + t), sp, [&](int row, bool neg) {
      rr[e] = row;
      ss[e] = neg ? (signed char)-1 : (signed char)1;
      ++e;
    });
  }
  if (got < sp.zeta) atomicOr(err, ERR_SKETCH);
}

// The table of S: packed (s <= 255, zeta <= 8): 8 row bytes per column in a
// uint2 (0xFF in unused bytes) and a sign byte; generic: zeta uint16 rows and
// a 32-bit sign mask per column.
__global__ void sketch_table_kernel(int n, SketchSpec sp, SketchTable tab, int* err, int64_t col0) {
  const int stride = gridDim.x * blockDim.x;
  const uint32_t inv_s = sketch_inv_s(sp.s);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    int got;
    if (tab.packed) {
      uint32_t p0, p1, ng;
      got = sketch_column_packed((uint32_t)(col0 + i), sp, inv_s, &p0, &p1, &ng);
      tab.rows8[i] = make_uint2(p0, p1);
      tab.neg8[i] = (uint8_t)ng;
    } else {
      int e = 0;
      uint32_t ng = 0u;
      uint16_t* rr = tab.rows16 + (size_t)i * sp.zeta;
      got = sketch_column<MAX_ZETA>((uint32_t)(col0 + i), sp, [&](int row, bool neg) {
        rr[e] = (uint16_t)row;
        ng |= (neg ? 1u : 0u) << e;
        ++e;
      });
      tab.neg32[i] = ng;
    }
    if (got < sp.zeta) atomicOr(err, ERR_SKETCH);
  }
}

__global__ void cycle_reset_kernel(CycleDev cd, int m, unsigned long long* acc0, int n_acc0) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    cd.flags[0] = m;
    cd.flags[1] = 0;
  }
  for (int e = threadIdx.x; e < n_acc0; e += blockDim.x) acc0[e] = 0ull;
}

// U[:, j] from the exact sketch of column j (float-float materialize
// kernels): int64 word sums T_w over all CTAs and the exponent E of the
// column's fixed-point scale, U = (T_0 2^(E-WB) + T_1 2^(E-2WB) + T_2
// 2^(E-3WB)) / sqrt(zeta).  The sums are exact (|T_w| < 2^53 converts
// exactly), so U does not depend on the order in which CTAs added them.
__global__ void sketch_finish_kernel(const long long* acc, int ncols, int s, int64_t col_stride, int wb, double scale,
                                     double* U) {
  const int j = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ncols || r >= s) return;
  const long long* a = acc + (size_t)j * col_stride;
  const int E = (int)a[3 * s];
  const double v = fma((double)a[r], ldexp(1.0, E - wb),
                       fma((double)a[s + r], ldexp(1.0, E - 2 * wb), (double)a[2 * s + r] * ldexp(1.0, E - 3 * wb)));
  U[(size_t)j * s + r] = v * scale;
}

}  // namespace

SketchSpec make_sketch_spec(int s, int zeta, uint64_t seed) {
  SketchSpec sp;
  sp.s = s;
  sp.zeta = zeta;
  sp.lim = 32768u - 32768u % (uint32_t)s;
  sp.k0 = (uint32_t)(seed & 0xFFFFFFFFull);
  sp.k1 = (uint32_t)(seed >> 32);
  sp.scale = 1.f;
  return sp;
}

void launch_cycle_reset(const CycleDev& cd, int m, cudaStream_t st, void* acc0, int n_acc0) {
  cycle_reset_kernel<<<1, 128, 0, st>>>(cd, m, static_cast<unsigned long long*>(acc0), n_acc0);
}

void launch_sketch_finish(const void* acc, int ncols, int s, int64_t col_stride, int wb, int zeta, double* U,
                          cudaStream_t st) {
  dim3 g((s + 127) / 128, ncols);
  sketch_finish_kernel<<<g, 128, 0, st>>>(static_cast<const long long*>(acc), ncols, s, col_stride, wb,
                                          1.0 / std::sqrt((double)zeta), U);
}

void launch_norm_b(const double* b, int n, double* part, int grid, const CycleDev& cd, cudaStream_t st) {
  const int rpc = (n + grid - 1) / grid;
  norm_b_kernel<<<grid, STEP_THREADS, 0, st>>>(b, n, part, cd, rpc);
}

void launch_start(int basis, const double* b, void* W0, int n, const CycleDev& cd, int grid, cudaStream_t st) {
  if (basis == 3) ff_start_kernel<<<grid, STEP_THREADS, 0, st>>>(b, (float2*)W0, n, cd);
  else if (basis == 0) start_kernel<double><<<grid, STEP_THREADS, 0, st>>>(b, (double*)W0, n, cd);
  else if (basis == 1) start_kernel<float><<<grid, STEP_THREADS, 0, st>>>(b, (float*)W0, n, cd);
  else start_kernel<__nv_bfloat16><<<grid, STEP_THREADS, 0, st>>>(b, (__nv_bfloat16*)W0, n, cd);
}

void launch_update(int basis, void* W, int64_t ldw, int n, int m_eff, int has_next, const double* zg, double* x,
                   double* part, int grid, const CycleDev& cd, int m, cudaStream_t st) {
  const int rpc = (n + grid - 1) / grid;
  if (basis == 3)
    ff_update_kernel<<<grid, STEP_THREADS, 0, st>>>((float2*)W, ldw, n, m_eff, has_next, zg, m, x, part, cd, rpc);
  else if (basis == 0)
    update_kernel<double><<<grid, STEP_THREADS, 0, st>>>((double*)W, ldw, n, m_eff, has_next, zg, m, x, part, cd,
                                                          rpc);
  else if (basis == 1)
    update_kernel<float><<<grid, STEP_THREADS, 0, st>>>((float*)W, ldw, n, m_eff, has_next, zg, m, x, part, cd, rpc);
  else
    update_kernel<__nv_bfloat16><<<grid, STEP_THREADS, 0, st>>>((__nv_bfloat16*)W, ldw, n, m_eff, has_next, zg, m,
                                                                 x, part, cd, rpc);
}

void launch_sketch_reduce(const void* sk_part, int ncols, int grid, int s, int zeta, int64_t col_stride, double* U,
                          cudaStream_t st) {
  dim3 g((s + 31) / 32, ncols);
  const double scale = 1.0 / std::sqrt((double)zeta);
  sketch_reduce_kernel<double><<<g, dim3(32, SR_GROUPS), 0, st>>>((const double*)sk_part, ncols, grid, s, scale,
                                                                  col_stride, U);
}

void launch_spmv_f64(int n, const int* row_ptr, const int* col, const double* val, const double* x, double* y,
                     cudaStream_t st) {
  const int grid = std::max(1, std::min(4096, (n + 255) / 256));
  spmv_f64_kernel<<<grid, 256, 0, st>>>(n, row_ptr, col, val, x, y);
}

void launch_dot_f64(const double* a, const double* b, int n, double* part, int grid, double* out, unsigned* counter,
                    cudaStream_t st) {
  const int rpc = (n + grid - 1) / grid;
  dot_f64_kernel<<<grid, STEP_THREADS, 0, st>>>(a, b, n, part, out, counter, rpc);
}

void launch_sketch_columns(int64_t col0, int64_t count, int s, int zeta, uint64_t seed, int* rows,
                           signed char* signs, int* err, cudaStream_t st) {
  const SketchSpec sp = make_sketch_spec(s, zeta, seed);
  const int grid = (int)((count + 255) / 256);
  if (grid > 0) sketch_columns_kernel<<<grid, 256, 0, st>>>(col0, count, sp, rows, signs, err);
}

void launch_sketch_table(int n, int s, int zeta, uint64_t seed, const SketchTable& tab, int* err, cudaStream_t st,
                         int64_t col0) {
  const SketchSpec sp = make_sketch_spec(s, zeta, seed);
  const int grid = std::max(1, std::min(8192, (n + 255) / 256));
  sketch_table_kernel<<<grid, 256, 0, st>>>(n, sp, tab, err, col0);
}

// Column r of a row-major n x ncols block <-> a contiguous vector.
namespace {
__global__ void gather_column_kernel(const double* __restrict__ B, int64_t n, int ncols, int r, double* __restrict__ b) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) b[i] = B[i * ncols + r];
}
__global__ void scatter_column_kernel(const double* __restrict__ x, int64_t n, int ncols, int r, double* __restrict__ X) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) X[i * ncols + r] = x[i];
}
int column_grid(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 4096); }
}  // namespace

namespace {
__global__ void zero_columns_kernel(double* X, int64_t n, int64_t ld, int ncols) {
  const int64_t total = n * ncols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    X[(e / ncols) * ld + e % ncols] = 0.0;
}
}  // namespace

void launch_zero_columns(double* X, int64_t n, int64_t ld, int ncols, cudaStream_t st) {
  const int64_t total = n * ncols;
  zero_columns_kernel<<<(int)std::min<int64_t>(4096, (total + 255) / 256), 256, 0, st>>>(X, n, ld, ncols);
}

void launch_gather_column(const double* B, int64_t n, int ncols, int r, double* b, cudaStream_t st) {
  gather_column_kernel<<<column_grid(n), 256, 0, st>>>(B, n, ncols, r, b);
}
void launch_scatter_column(const double* x, int64_t n, int ncols, int r, double* X, cudaStream_t st) {
  scatter_column_kernel<<<column_grid(n), 256, 0, st>>>(x, n, ncols, r, X);
}

}  // namespace krylov
