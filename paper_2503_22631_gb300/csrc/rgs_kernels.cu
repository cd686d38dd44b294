// rgs_kernels.cu -- the randomized Gram-Schmidt cycle (Algorithm 1) on the GPU.
//
// One step j of Algorithm 1 (window of the last k sketches; all of them when
// k >= m, the paper's method):
//
//   product     p = A w_j                     (the float-float product kernel
//                                              with L.rgs, or rgs_spmv_f64 for
//                                              the float64 basis) and ||p||^2
//   orthogonalize  u = S p (exact fixed-point sketch, summed over CTAs with
//                  int64 atomics), then in sketch space r_ij = <u_i, u>,
//                  u -= r_ij u_i over the window; r_{j+1,j} = ||u||,
//                  u_{j+1} = u / r_{j+1,j}                      (rgs_orth)
//   materialize w_{j+1} = (p - sum r_ij w_i) / r_{j+1,j}       (rgs_mat)
//
// The sketch-space orthogonalization is classical Gram-Schmidt applied twice
// ("twice is enough"), equal to the modified Gram-Schmidt loop of Algorithm 1
// in exact arithmetic and as stable; two passes of window-parallel dots
// replace the window-long chain of dependent dots.
//
// A cycle starts by sketching the stored start vector w (b / ||b|| in cycle 1,
// the previous cycle's w_{m+1} afterwards): alpha = ||S w||, u_0 = S w / alpha,
// w_0 = w / alpha; cycle 1 takes beta = ||b|| alpha, later cycles discard
// alpha as Algorithm 2 does.  The small problem uses R itself (no whitening):
// X = R_m, coupling r_{m+1,m}, next start vector w_{m+1}.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "internal.h"
#include "kernels.cuh"
#include "step_common.cuh"

namespace krylov {
namespace {

constexpr int NW = 3;  // fixed-point words per value (float64-class accuracy)
constexpr int RGS_MAX_S = 1024;
constexpr int RGS_MAX_WIN = 257;
constexpr int MAT_BATCH = 8;

__host__ __device__ __forceinline__ size_t rgs_bins_bytes(int s, int copies) {
  return (size_t)NW * s * copies * sizeof(int);
}

// value of entry i as a float pair (hi, lo) with hi + lo = the stored value
// to float-float accuracy
__device__ __forceinline__ ff src_value(const double* v, int64_t i) { return ff_from_double(v[i]); }
__device__ __forceinline__ ff src_value(const float2* v, int64_t i) {
  const float2 t = v[i];
  return ff{t.x, t.y};
}

// Last-CTA epilogues of the sketch kernel (one CTA, blockDim.x threads):
// u (s doubles in shared memory) is the exact sketch S v.
enum : int { RGS_START = 0, RGS_STEP = 1 };

__device__ void rgs_epilogue_start(const RgsArgs& a, const CycleDev& cd, int cycle, double* u, double* red) {
  const int s = a.s;
  double acc = 0.0;
  for (int r = threadIdx.x; r < s; r += blockDim.x) acc = fma(u[r], u[r], acc);
  const double nrm2 = block_sum(acc, red);
  __shared__ double s_alpha;
  if (threadIdx.x == 0) {
    const double alpha = sqrt(nrm2);
    s_alpha = alpha;
    cd.scal[7] = (alpha > 0.0) ? 1.0 / alpha : 0.0;  // w_0 = w / alpha
    if (cycle == 1) a.misc[0] = cd.scal[0] * alpha;   // beta = ||S b|| = ||b|| alpha
    if (!(alpha > 0.0) || !isfinite(alpha)) cd.flags[2] |= ERR_NONFINITE;
  }
  __syncthreads();
  const double inv = (s_alpha > 0.0) ? 1.0 / s_alpha : 0.0;
  for (int r = threadIdx.x; r < s; r += blockDim.x) a.U[r] = u[r] * inv;
}

__device__ void rgs_epilogue_step(const RgsArgs& a, const CycleDev& cd, int j, double* u, double* red, double* rw) {
  const int s = a.s, ldr = a.m + 1;
  const int lo = max(0, j - a.k + 1);
  const int nwin = j - lo + 1;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  double acc = 0.0;
  for (int r = threadIdx.x; r < s; r += blockDim.x) acc = fma(u[r], u[r], acc);
  const double un2 = block_sum(acc, red);  // ||S p|| before orthogonalization (thread 0)
  for (int q = threadIdx.x; q < nwin; q += blockDim.x) rw[q] = 0.0;
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
    // window-parallel dots c_q = <u_{lo+q}, u>
    __shared__ double c[RGS_MAX_WIN];
    for (int q = wid; q < nwin; q += nwarp) {
      const double* Uq = a.U + (size_t)(lo + q) * s;
      double d = 0.0;
      for (int r = lane; r < s; r += 32) d = fma(Uq[r], u[r], d);
      d = warp_sum(d);
      if (lane == 0) c[q] = d;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < s; r += blockDim.x) {
      double v = u[r];
      for (int q = 0; q < nwin; ++q) v = fma(-c[q], a.U[(size_t)(lo + q) * s + r], v);
      u[r] = v;
    }
    for (int q = threadIdx.x; q < nwin; q += blockDim.x) rw[q] += c[q];
    __syncthreads();
  }
  acc = 0.0;
  for (int r = threadIdx.x; r < s; r += blockDim.x) acc = fma(u[r], u[r], acc);
  const double rr2 = block_sum(acc, red);
  __shared__ double s_r;
  if (threadIdx.x == 0) {
    const double rn = sqrt(rr2);
    s_r = rn;
    for (int q = 0; q < nwin; ++q) cd.R[(size_t)j * ldr + lo + q] = rw[q];
    if (!isfinite(rn) || !isfinite(un2)) cd.flags[2] |= ERR_NONFINITE;
    if (!(rn > a.thr * sqrt(un2))) {  // happy breakdown: the cycle ends with j + 1 columns
      if (cd.flags[1] == 0) {
        cd.flags[1] = 1;
        cd.flags[0] = j + 1;
      }
    } else if (j + 1 <= a.m) {
      cd.R[(size_t)j * ldr + j + 1] = rn;
    }
  }
  __syncthreads();
  if (cd.flags[1] == 0) {
    const double inv = 1.0 / s_r;
    for (int r = threadIdx.x; r < s; r += blockDim.x) a.U[(size_t)(j + 1) * s + r] = u[r] * inv;
  }
}

// Exact sketch of a vector v (rows of this CTA into fixed-point bins, bin sums
// added to a.acc with int64 atomics), then the epilogue of `mode` in the last
// CTA.  The fixed-point scale comes from a bound B >= max |v_i|.
template <typename SRC, int SKM>
__global__ void __launch_bounds__(STEP_THREADS) rgs_sketch_kernel(const RgsArgs a, const CycleDev cd, const SRC* v,
                                                                   int mode, int j, int cycle) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  __shared__ int s_last;
  __shared__ FxScale s_fx;
  __shared__ double u[RGS_MAX_S];
  __shared__ double rw[RGS_MAX_WIN];
  if (cd.flags[1] != 0) return;  // breakdown earlier in this cycle
  const int C = a.copies;
  int* bins = reinterpret_cast<int*>(smem);  // [NW][s][C]
  const int nb = NW * a.s * C;
  for (int e = threadIdx.x; e < nb; e += blockDim.x) bins[e] = 0;
  if (threadIdx.x == 0) {
    // bound: ||v|| from the reducer that produced v
    const double B = ((mode == RGS_START) ? sqrt(cd.scal[5]) : sqrt(cd.pi[j])) * 1.0001 + 1e-300;
    FxScale f;
    f.E = ilogb(B) + 2;
    f.to_fixed = ldexpf(1.0f, a.fx_wb - f.E);
    f.word = ldexpf(1.0f, a.fx_wb);
    s_fx = f;
  }
  __syncthreads();
  const FxScale fxs = s_fx;
  const int cp = (threadIdx.x & 31) & (C - 1);
  const int sC = a.s * C;
  StepLaunch L{};  // only the sketch fields are read by the column loaders
  L.s = a.s;
  L.zeta = a.zeta;
  L.seed = a.seed;
  L.sk_tab = a.sk_tab;
  const SketchSpec sp = spec_of(L);
  const uint32_t inv_s = sketch_inv_s(a.s);
  int bad = 0;
  const int r0 = blockIdx.x * a.rows_per_cta;
  const int r1 = min(a.n, r0 + a.rows_per_cta);
  for (int i = r0 + (int)threadIdx.x; i < r1; i += blockDim.x) {
    const ff x = src_value(v, i);
    typename SkColOf<SKM>::type col;
    col.load(L, sp, inv_s, i);
    bad |= (col.got < a.zeta);
    const FxWords<NW> xw = fx_split<NW>(x.hi, x.lo, fxs);
    for (int e = 0; e < col.got; ++e) fx_emit<NW>(bins, sC, col.row(e), cp, xw, col.neg(e), C);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NW * a.s; e += blockDim.x) {
    const int w = e / a.s, b = e % a.s;
    long long t = 0;
    const int* cl = bins + (w * a.s + b) * C;
    for (int c = 0; c < C; ++c) t += cl[(c + b) & (C - 1)];
    if (t != 0) atomicAdd(reinterpret_cast<unsigned long long*>(a.acc + e), (unsigned long long)t);
  }
  if (bad) atomicOr(&cd.flags[2], ERR_SKETCH);
  if (!last_block_flag(cd.counter, &s_last)) return;
  for (int b = threadIdx.x; b < a.s; b += blockDim.x) {
    double val = 0.0;
    for (int w = 0; w < NW; ++w) {
      long long* slot = a.acc + w * a.s + b;
      const long long t = __ldcg(slot);
      *slot = 0;  // ready for the next sketch
      val += ldexp((double)t, fxs.E - (w + 1) * a.fx_wb);
    }
    u[b] = val / sqrt((double)a.zeta);
  }
  __syncthreads();
  if (mode == RGS_START) rgs_epilogue_start(a, cd, cycle, u, red);
  else rgs_epilogue_step(a, cd, j, u, red, rw);
  __syncthreads();
  if (threadIdx.x == 0) *cd.counter = 0u;
}

// w_0 <- w_0 / alpha (the start vector after its sketch norm is known)
template <typename VT>
__global__ void rgs_scale0_kernel(VT* W0, int n, const CycleDev cd) {
  const double inv = cd.scal[7];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if constexpr (sizeof(VT) == 8 && !std::is_same<VT, float2>::value) {
      W0[i] = W0[i] * inv;
    } else {
      const float2 t = W0[i];
      const ff r = ff_mul(ff{t.x, t.y}, ff_from_double(inv));
      W0[i] = make_float2(r.hi, r.lo);
    }
  }
}

// w_{j+1} = (p - sum_{q in window} r_{qj} w_q) / r_{j+1,j}, window slices
// loaded MAT_BATCH at a time.
__global__ void __launch_bounds__(STEP_THREADS) rgs_mat_f64_kernel(const RgsArgs a, const CycleDev cd,
                                                                    const double* p, int j) {
  __shared__ double rc[RGS_MAX_WIN];
  __shared__ double s_inv;
  if (cd.flags[1] != 0) return;
  const int ldr = a.m + 1;
  const int lo = max(0, j - a.k + 1), nwin = j - lo + 1;
  for (int q = threadIdx.x; q < nwin; q += blockDim.x) rc[q] = cd.R[(size_t)j * ldr + lo + q];
  if (threadIdx.x == 0) s_inv = 1.0 / cd.R[(size_t)j * ldr + j + 1];
  __syncthreads();
  const double inv = s_inv;
  const double* W = static_cast<const double*>(a.W);
  double* Wn = static_cast<double*>(a.W) + (int64_t)(j + 1) * a.ldw;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
    double acc = p[i];
    for (int q0 = 0; q0 < nwin; q0 += MAT_BATCH) {
      double wv[MAT_BATCH];
#pragma unroll
      for (int u = 0; u < MAT_BATCH; ++u)
        if (q0 + u < nwin) wv[u] = W[(int64_t)(lo + q0 + u) * a.ldw + i];
#pragma unroll
      for (int u = 0; u < MAT_BATCH; ++u)
        if (q0 + u < nwin) acc = fma(-rc[q0 + u], wv[u], acc);
    }
    Wn[i] = acc * inv;
  }
}

__global__ void __launch_bounds__(STEP_THREADS) rgs_mat_ff_kernel(const RgsArgs a, const CycleDev cd,
                                                                   const float2* p, int j) {
  __shared__ ff rc[RGS_MAX_WIN];
  __shared__ ff s_inv;
  if (cd.flags[1] != 0) return;
  const int ldr = a.m + 1;
  const int lo = max(0, j - a.k + 1), nwin = j - lo + 1;
  for (int q = threadIdx.x; q < nwin; q += blockDim.x) rc[q] = ff_neg(ff_from_double(cd.R[(size_t)j * ldr + lo + q]));
  if (threadIdx.x == 0) s_inv = ff_from_double(1.0 / cd.R[(size_t)j * ldr + j + 1]);
  __syncthreads();
  const ff inv = s_inv;
  const float2* W = static_cast<const float2*>(a.W);
  float2* Wn = static_cast<float2*>(a.W) + (int64_t)(j + 1) * a.ldw;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
    const float2 p2 = p[i];
    ff acc{p2.x, p2.y};
    for (int q0 = 0; q0 < nwin; q0 += MAT_BATCH) {
      float2 wv[MAT_BATCH];
#pragma unroll
      for (int u = 0; u < MAT_BATCH; ++u)
        if (q0 + u < nwin) wv[u] = W[(int64_t)(lo + q0 + u) * a.ldw + i];
#pragma unroll
      for (int u = 0; u < MAT_BATCH; ++u)
        if (q0 + u < nwin) acc = ff_add(acc, ff_mul(rc[q0 + u], ff{wv[u].x, wv[u].y}));
    }
    const ff w = ff_mul(acc, inv);
    Wn[i] = make_float2(w.hi, w.lo);
  }
}

// p = A w_j (float64 basis) with ||p||^2 reduced by the last CTA into cd.pi[j];
// matrix values stored as AT (float when the narrowing is lossless).
template <typename AT>
__global__ void __launch_bounds__(STEP_THREADS) rgs_spmv_f64_kernel(const StepLaunch L, const CycleDev cd) {
  __shared__ double red[32];
  __shared__ int s_last;
  if (cd.flags[1] != 0) return;
  const double* W = static_cast<const double*>(L.W);
  const double* wj = W + (int64_t)L.j * L.ldw;
  const AT* val = static_cast<const AT*>(L.val);
  double* p = static_cast<double*>(L.p_out);
  const int r0 = blockIdx.x * L.rows_per_cta, r1 = min(L.n, r0 + L.rows_per_cta);
  double acc = 0.0;
  for (int i = r0 + (int)threadIdx.x; i < r1; i += blockDim.x) {
    double y = 0.0;
    for (int e = L.row_ptr[i]; e < L.row_ptr[i + 1]; ++e) y = fma((double)val[e], wj[L.col[e]], y);
    p[i] = y;
    acc = fma(y, y, acc);
  }
  const double v = block_sum(acc, red);
  if (threadIdx.x == 0) L.part[blockIdx.x] = v;
  if (!last_block_flag(cd.counter, &s_last)) return;
  if (threadIdx.x < 32) {
    const double t = warp_sum_partials(L.part, (int)gridDim.x, 1, 0);
    if (threadIdx.x == 0) {
      cd.pi[L.j] = t;
      if (!isfinite(t)) cd.flags[2] |= ERR_NONFINITE;
      *cd.counter = 0u;
    }
  }
}

// Small problem of a randomized Gram-Schmidt cycle: X = R_m (me x me, zero
// padded), coupling of the previous cycle, basis map T^{-1} = I, next start
// vector w_{m+1} (g = 0, tau = 1), and the norms the exp scaling needs.
__global__ void rgs_small_kernel(SmallDev sd, CycleDev cd, int M, int me, int has_next, int cycle, double t) {
  const int ldr = M + 1;
  double* X = sd.Xblk + (size_t)(cycle - 1) * M * M;
  for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
    const int r = e % M, c = e / M;
    X[e] = (r < me && c < me) ? cd.R[(size_t)c * ldr + r] : 0.0;
    sd.Tinv[e] = (r == c && r < me) ? 1.0 : 0.0;
  }
  for (int q = threadIdx.x; q < M; q += blockDim.x) sd.zg[M + q] = 0.0;
  __syncthreads();
  if (threadIdx.x == 0) {
    double cmax = 0.0;
    for (int c = 0; c < me; ++c) {
      double cs = 0.0;
      for (int r = 0; r < me; ++r) cs += fabs(X[(size_t)c * M + r]);
      cmax = fmax(cmax, cs);
    }
    if (cycle >= 2) {
      sd.gam[cycle - 2] = sd.misc[1];  // r_{m+1,m} of the previous cycle (alpha discarded)
      sd.misc[3] = fabs(t * sd.misc[1]);
    } else {
      sd.misc[3] = 0.0;
    }
    sd.misc[1] = has_next ? cd.R[(size_t)(me - 1) * ldr + me] : 0.0;
    sd.zg[2 * M] = has_next ? 1.0 : 0.0;
    sd.misc[2] = fabs(t) * cmax;
    sd.misc[4] = 1.0;
    if (!isfinite(cmax) || !isfinite(sd.misc[1])) cd.flags[2] |= ERR_NONFINITE;
  }
}

size_t rgs_sketch_smem(const RgsArgs& a) { return rgs_bins_bytes(a.s, a.copies); }

template <typename SRC>
void launch_sketch(const RgsArgs& a, const CycleDev& cd, const SRC* v, int mode, int j, int cycle, cudaStream_t st) {
  const size_t smem = rgs_sketch_smem(a);
  switch (a.sk_mode) {
    case SK_TAB8: {
      auto k = rgs_sketch_kernel<SRC, SK_TAB8>;
      raise_smem_limit((const void*)k, smem);
      k<<<a.grid, STEP_THREADS, smem, st>>>(a, cd, v, mode, j, cycle);
      break;
    }
    case SK_TAB16: {
      auto k = rgs_sketch_kernel<SRC, SK_TAB16>;
      raise_smem_limit((const void*)k, smem);
      k<<<a.grid, STEP_THREADS, smem, st>>>(a, cd, v, mode, j, cycle);
      break;
    }
    case SK_GEN8: {
      auto k = rgs_sketch_kernel<SRC, SK_GEN8>;
      raise_smem_limit((const void*)k, smem);
      k<<<a.grid, STEP_THREADS, smem, st>>>(a, cd, v, mode, j, cycle);
      break;
    }
    default: {
      auto k = rgs_sketch_kernel<SRC, SK_GEN>;
      raise_smem_limit((const void*)k, smem);
      k<<<a.grid, STEP_THREADS, smem, st>>>(a, cd, v, mode, j, cycle);
      break;
    }
  }
}

int stream_grid(int n) { return std::max(1, std::min(4096, (n + STEP_THREADS - 1) / STEP_THREADS)); }

}  // namespace

void launch_rgs_start(const RgsArgs& a, const CycleDev& cd, int cycle, cudaStream_t st) {
  if (a.basis == 3) {
    float2* W0 = static_cast<float2*>(a.W);
    launch_sketch(a, cd, (const float2*)W0, RGS_START, 0, cycle, st);
    rgs_scale0_kernel<float2><<<stream_grid(a.n), STEP_THREADS, 0, st>>>(W0, a.n, cd);
  } else {
    double* W0 = static_cast<double*>(a.W);
    launch_sketch(a, cd, (const double*)W0, RGS_START, 0, cycle, st);
    rgs_scale0_kernel<double><<<stream_grid(a.n), STEP_THREADS, 0, st>>>(W0, a.n, cd);
  }
}

void launch_rgs_product_f64(const StepLaunch& L, const CycleDev& cd, cudaStream_t st) {
  if (L.val_f32) rgs_spmv_f64_kernel<float><<<L.grid, STEP_THREADS, 0, st>>>(L, cd);
  else rgs_spmv_f64_kernel<double><<<L.grid, STEP_THREADS, 0, st>>>(L, cd);
}

void launch_rgs_orth(const RgsArgs& a, const CycleDev& cd, const void* p, int j, cudaStream_t st) {
  if (a.basis == 3) launch_sketch(a, cd, static_cast<const float2*>(p), RGS_STEP, j, 0, st);
  else launch_sketch(a, cd, static_cast<const double*>(p), RGS_STEP, j, 0, st);
}

void launch_rgs_mat(const RgsArgs& a, const CycleDev& cd, const void* p, int j, cudaStream_t st) {
  if (a.basis == 3)
    rgs_mat_ff_kernel<<<stream_grid(a.n), STEP_THREADS, 0, st>>>(a, cd, static_cast<const float2*>(p), j);
  else
    rgs_mat_f64_kernel<<<stream_grid(a.n), STEP_THREADS, 0, st>>>(a, cd, static_cast<const double*>(p), j);
}

void launch_rgs_small(const SmallDev& sd, const CycleDev& cd, int m, int me, int has_next, int cycle, double t,
                      cudaStream_t st) {
  rgs_small_kernel<<<1, 256, 0, st>>>(sd, cd, m, me, has_next, cycle, t);
}

}  // namespace krylov
