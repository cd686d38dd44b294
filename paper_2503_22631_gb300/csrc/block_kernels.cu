// block_kernels.cu -- the block form of the truncated cycle: nb independent
// right-hand sides of one matrix advanced together (float-float basis).
//
// The basis and the products are stored as float-float pairs or, for the
// float32 basis, as floats (basis32); the arithmetic is float-float in both,
// and every value used after a store (norms, sketches, dots, the next kernel)
// is the stored one.
//
// Every vector of the cycle is stored row-major n x nb (the nb values of a row
// contiguous), so one pass over A serves all right-hand sides: a warp takes a
// row, its lanes take right-hand sides lane and lane + 32, the column index
// and value of a nonzero are read once (broadcast) and the gather of w_j at
// that column reads nb contiguous float-float entries.  The sketch table is
// read once per row for all right-hand sides; the bins of right-hand side r
// are the column r of a [3 words][s][nb] shared array (distinct banks across
// the lanes), summed over CTAs with int64 atomics into an exact [3][s][nb]
// accumulator per basis column.  Per-right-hand-side scalars (norms, window
// coefficients, R, flags) live in the single-vector layout repeated nb times
// (BatchStride), so the small-problem kernels run unchanged per problem.
#include <algorithm>
#include <climits>
#include <cmath>

#include "internal.h"
#include "kernels.cuh"
#include "step_common.cuh"

namespace krylov {
namespace {

constexpr int NWB = 3;       // fixed-point words per value
constexpr int BK_MAXNB = 64; // right-hand sides per block
constexpr int BK_WARPS = STEP_THREADS / 32;

__device__ __forceinline__ ff ldf(const float2* p) {
  const float2 v = *p;
  return ff{v.x, v.y};
}
__device__ __forceinline__ ff ldv(const float2* p) { return ldf(p); }
__device__ __forceinline__ ff ldv(const float* p) { return ff{*p, 0.f}; }
// store v in the storage type; returns the stored value
__device__ __forceinline__ ff stv(float2* p, ff v) {
  *p = make_float2(v.hi, v.lo);
  return v;
}
__device__ __forceinline__ ff stv(float* p, ff v) {
  const float f = __fadd_rn(v.hi, v.lo);
  *p = f;
  return ff{f, 0.f};
}

// ---- norms of the right-hand sides and the start vectors ------------------
__global__ void __launch_bounds__(STEP_THREADS) bk_norm_kernel(const BlockLaunch B, const double* b, int64_t ldb) {
  __shared__ double red[BK_WARPS][BK_MAXNB];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double a0 = 0.0, a1 = 0.0;
  const int r0 = blockIdx.x * B.rows_per_cta, r1 = min(B.n, r0 + B.rows_per_cta);
  for (int i = r0 + wid; i < r1; i += BK_WARPS) {
    const double* bi = b + (int64_t)i * ldb;
    if (lane < B.nb) a0 = fma(bi[lane], bi[lane], a0);
    if (lane + 32 < B.nb) a1 = fma(bi[lane + 32], bi[lane + 32], a1);
  }
  red[wid][lane] = a0;
  red[wid][lane + 32] = a1;
  __syncthreads();
  for (int r = threadIdx.x; r < B.nb; r += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < BK_WARPS; ++w) t += red[w][r];
    B.part[(size_t)blockIdx.x * BK_MAXNB + r] = t;
  }
  if (!last_block_flag(B.counter, &s_last)) return;
  for (int r = wid; r < B.nb; r += BK_WARPS) {
    const double t = warp_sum_partials(B.part, (int)gridDim.x, BK_MAXNB, r);
    if (lane == 0) {
      const CycleDev c = offset_cd(B.cd, B.bs, r);
      const double eta = sqrt(t);
      c.scal[4] = t;
      c.scal[0] = eta;
      c.scal[1] = (eta > 0.0) ? 1.0 / eta : 0.0;
      c.scal[5] = 1.0;  // bound on ||w_1||^2
      if (!isfinite(t)) c.flags[2] |= ERR_NONFINITE;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *B.counter = 0u;
}

template <typename VT>
__global__ void bk_start_kernel(const BlockLaunch B, const double* b, int64_t ldb) {
  const int64_t total = (int64_t)B.n * B.nb;
  VT* W = static_cast<VT*>(B.W);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / B.nb), r = (int)(e % B.nb);
    const double inv = offset_cd(B.cd, B.bs, r).scal[1];
    (void)stv(W + e, ff_from_double(b[(int64_t)i * ldb + r] * inv));
  }
}

// ---- materialize + sketch of column j for every right-hand side ------------
template <typename VT, bool MAT, int KW>
__global__ void __launch_bounds__(STEP_THREADS) bk_mat_kernel(const BlockLaunch B) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float s_tofix[BK_MAXNB];
  __shared__ int s_E[BK_MAXNB];
  __shared__ ff s_h[KW][BK_MAXNB];
  __shared__ ff s_rho[BK_MAXNB];
  __shared__ double red[BK_WARPS][BK_MAXNB];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nb = B.nb, s = B.s, j = B.j;
  int* bins = reinterpret_cast<int*>(smem);  // [NWB][s][nb]
  for (int e = threadIdx.x; e < NWB * s * nb; e += blockDim.x) bins[e] = 0;
  const int lo = MAT ? max(0, j - B.k) : j;
  const int nl = j - lo;
  for (int r = threadIdx.x; r < nb; r += blockDim.x) {
    const CycleDev c = offset_cd(B.cd, B.bs, r);
    const double bound = (MAT ? c.scal[6] : sqrt(c.scal[5])) * 1.0001 + 1e-300;
    const int E = ilogb(bound) + 2;
    s_E[r] = E;
    s_tofix[r] = ldexpf(1.0f, B.fx_wb - E);
    if (blockIdx.x == 0) B.E[(size_t)j * BK_MAXNB + r] = E;
    const double* co = c.coef + (size_t)(j > 0 ? j - 1 : 0) * (MAX_WINDOW + 1);
    for (int q = 0; q < KW; ++q) s_h[q][r] = (MAT && q < nl) ? ff_neg(ff_from_double(co[q])) : ff{0.f, 0.f};
    s_rho[r] = MAT ? ff_from_double(co[MAX_WINDOW]) : ff{1.f, 0.f};
  }
  __syncthreads();
  const float word = ldexpf(1.0f, B.fx_wb);
  VT* const W = static_cast<VT*>(B.W);
  const VT* Wq[KW];
#pragma unroll
  for (int q = 0; q < KW; ++q) Wq[q] = W + (int64_t)(lo + (q < nl ? q : 0)) * B.slot;
  VT* Wj = W + (int64_t)j * B.slot;
  const VT* Pp = static_cast<const VT*>(B.p_prev);
  ffacc sig[2];
  const int r0 = blockIdx.x * B.rows_per_cta, r1 = min(B.n, r0 + B.rows_per_cta);
  for (int i = r0 + wid; i < r1; i += BK_WARPS) {
    const uint2 rows = __ldg(B.tab.rows8 + i);
    const uint32_t ng = __ldg(B.tab.neg8 + i);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = lane + 32 * h;
      if (r >= nb) continue;
      const int64_t e = (int64_t)i * nb + r;
      ff w;
      if (MAT) {
        ff acc = ldv(Pp + e);
#pragma unroll
        for (int q = 0; q < KW; ++q)
          if (q < nl) acc = ff_add(acc, ff_mul(s_h[q][r], ldv(Wq[q] + e)));
        w = stv(Wj + e, ff_mul(acc, s_rho[r]));
      } else {
        w = ldv(Wj + e);
      }
      sig[h].add_prod(w, w);
      FxScale f;
      f.E = s_E[r];
      f.to_fixed = s_tofix[r];
      f.word = word;
      const FxWords<NWB> xw = fx_split<NWB>(w.hi, w.lo, f);
#pragma unroll
      for (int z = 0; z < 8; ++z)
        if (z < B.zeta) {
          const int bin = (int)(((z < 4 ? rows.x : rows.y) >> (8 * (z & 3))) & 0xFFu);
          int* bp = bins + bin * nb + r;
          const bool neg = (ng >> z) & 1u;
#pragma unroll
          for (int wd = 0; wd < NWB; ++wd) atomicAdd(bp + wd * s * nb, neg ? -xw.q[wd] : xw.q[wd]);
        }
    }
  }
  {
    const ff a = sig[0].result(), b2 = sig[1].result();
    red[wid][lane] = ff_to_double(a);
    red[wid][lane + 32] = ff_to_double(b2);
  }
  __syncthreads();
  for (int r = threadIdx.x; r < nb; r += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < BK_WARPS; ++w) t += red[w][r];
    B.part[(size_t)blockIdx.x * BK_MAXNB + r] = t;
  }
  long long* acc = B.acc + (size_t)j * NWB * s * BK_MAXNB;
  for (int e = threadIdx.x; e < NWB * s * nb; e += blockDim.x) {
    const int t = bins[e];
    if (t != 0) {
      const int wd = e / (s * nb), rem = e % (s * nb);
      atomicAdd(reinterpret_cast<unsigned long long*>(acc + (size_t)wd * s * BK_MAXNB + rem), (unsigned long long)(long long)t);
    }
  }
  if (!last_block_flag(B.counter, &s_last)) return;
  for (int r = wid; r < nb; r += BK_WARPS) {
    const double sig2 = warp_sum_partials(B.part, (int)gridDim.x, BK_MAXNB, r);
    if (lane == 0) {
      const CycleDev c = offset_cd(B.cd, B.bs, r);
      const int ldr = B.m + 1;
      c.sig2[j] = sig2;
      if (!isfinite(sig2)) c.flags[2] |= ERR_NONFINITE;
      if (MAT) {
        const double rho = c.coef[(size_t)(j - 1) * (MAX_WINDOW + 1) + MAX_WINDOW];
        c.R[(size_t)(j - 1) * ldr + j] = 1.0 / rho;
        if (!(sqrt(sig2) / rho > B.thr * sqrt(c.pi[j - 1])) && c.flags[1] == 0) {
          c.flags[1] = 1;
          c.flags[0] = j;
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *B.counter = 0u;
}

// ---- product + window dots for every right-hand side -----------------------
template <typename VT, typename AT, int KW>
__global__ void __launch_bounds__(STEP_THREADS) bk_spmv_kernel(const BlockLaunch B) {
  __shared__ double red[BK_WARPS][BK_MAXNB];
  __shared__ double tot[NQ][BK_MAXNB];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nb = B.nb, j = B.j;
  const int dlo = max(0, j - B.k + 1);
  const int nd = j - dlo + 1;
  const VT* const W = static_cast<const VT*>(B.W);
  const VT* Wj = W + (int64_t)j * B.slot;
  const VT* Wd[KW];
#pragma unroll
  for (int q = 0; q < KW; ++q) Wd[q] = W + (int64_t)(dlo + (q < nd ? q : 0)) * B.slot;
  VT* Po = static_cast<VT*>(B.p_out);
  const AT* val = static_cast<const AT*>(B.val);
  ffacc pi[2], dots[KW][2];
  const int r0 = blockIdx.x * B.rows_p, r1 = min(B.n, r0 + B.rows_p);
  for (int i = r0 + wid; i < r1; i += BK_WARPS) {
    const int eb = __ldg(B.rp + i), ee = __ldg(B.rp + i + 1);
    ffacc acc[2];
    // nonzeros in batches of 4: indices and values first, then the gathers,
    // then the sums (storage order)
    for (int e0 = eb; e0 < ee; e0 += 4) {
      int cc[4];
      AT av[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (e0 + u < ee) {
          cc[u] = __ldg(B.ci + e0 + u);
          av[u] = __ldg(val + e0 + u);
        }
      ff wv[4][2];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (e0 + u < ee) {
          const VT* wc = Wj + (int64_t)cc[u] * nb;
          if (lane < nb) wv[u][0] = ldv(wc + lane);
          if (lane + 32 < nb) wv[u][1] = ldv(wc + lane + 32);
        }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (e0 + u < ee) {
#pragma unroll
          for (int h = 0; h < 2; ++h)
            if (lane + 32 * h < nb) {
              const float2 pe = prod_pe(av[u], wv[u][h]);
              acc[h].add_pe(pe.x, pe.y);
            }
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = lane + 32 * h;
      if (r >= nb) continue;
      const int64_t e = (int64_t)i * nb + r;
      const ff p = stv(Po + e, acc[h].result());
      pi[h].add_prod(p, p);
#pragma unroll
      for (int q = 0; q < KW; ++q)
        if (q < nd) dots[q][h].add_prod(ldv(Wd[q] + e), p);
    }
  }
  // per-CTA partials [NQ][nb] (slot 1: ||p||^2, 2 + q: <w_q, p>)
  for (int q = 1; q < 2 + nd; ++q) {
    ff a, b2;
    if (q == 1) {
      a = pi[0].result();
      b2 = pi[1].result();
    } else {
      a = ff{0.f, 0.f};
      b2 = ff{0.f, 0.f};
#pragma unroll
      for (int qq = 0; qq < KW; ++qq)
        if (qq == q - 2) {
          a = dots[qq][0].result();
          b2 = dots[qq][1].result();
        }
    }
    __syncthreads();
    red[wid][lane] = ff_to_double(a);
    red[wid][lane + 32] = ff_to_double(b2);
    __syncthreads();
    for (int r = threadIdx.x; r < nb; r += blockDim.x) {
      double t = 0.0;
      for (int w = 0; w < BK_WARPS; ++w) t += red[w][r];
      B.part[((size_t)blockIdx.x * NQ + q) * BK_MAXNB + r] = t;
    }
  }
  if (!last_block_flag(B.counter, &s_last)) return;
  for (int e = wid; e < (1 + nd) * nb; e += BK_WARPS) {
    const int q = 1 + e / nb, r = e % nb;
    const double t = warp_sum_partials(B.part + (size_t)q * BK_MAXNB + r, (int)gridDim.x, NQ * BK_MAXNB, 0);
    if (lane == 0) tot[q][r] = t;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < nb; r += blockDim.x) {
    const CycleDev c = offset_cd(B.cd, B.bs, r);
    if (c.flags[1] != 0) continue;
    const int ldr = B.m + 1;
    const double pv = tot[1][r];
    c.pi[j] = pv;
    if (!isfinite(pv)) c.flags[2] |= ERR_NONFINITE;
    double est = pv;
    double* co = c.coef + (size_t)j * (MAX_WINDOW + 1);
    for (int q = 0; q < MAX_WINDOW; ++q) {
      const int slot = dlo + q;
      double h = 0.0;
      if (slot <= j) {
        const double s2 = c.sig2[slot];
        h = (s2 > 0.0) ? tot[2 + q][r] / s2 : 0.0;
        est -= h * h * s2;
        c.R[(size_t)j * ldr + slot] = h;
      }
      co[q] = h;
    }
    est = fmax(est, 1e-20 * pv);
    co[MAX_WINDOW] = (pv > 0.0) ? 1.0 / sqrt(est) : 1.0;
    double bnd = sqrt(pv);
    for (int q = 0; q < MAX_WINDOW; ++q)
      if (dlo + q <= j) bnd += fabs(co[q]) * sqrt(c.sig2[dlo + q]);
    c.scal[6] = bnd * fabs(co[MAX_WINDOW]);
  }
  __syncthreads();
  if (threadIdx.x == 0) *B.counter = 0u;
}

// U_r[:, col] = S w_col for every right-hand side r (exact sums, one
// conversion), the accumulators zeroed for the next cycle.
__global__ void bk_sketch_fin_kernel(const BlockLaunch B, SmallDev sd, int ncols) {
  const int col = blockIdx.y;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = B.s, nb = B.nb;
  if (col >= ncols || e >= s * nb) return;
  const int bin = e / nb, r = e % nb;
  long long* acc = B.acc + (size_t)col * NWB * s * BK_MAXNB;
  const int E = B.E[(size_t)col * BK_MAXNB + r];
  double v = 0.0;
  for (int wd = 0; wd < NWB; ++wd) {
    long long* slot = acc + (size_t)wd * s * BK_MAXNB + bin * nb + r;
    v += ldexp((double)*slot, E - (wd + 1) * B.fx_wb);
    *slot = 0;
  }
  SmallDev d = offset_sd(sd, B.bs, r);
  d.U[(size_t)col * s + bin] = v / sqrt((double)B.zeta);
}

// x_r += W z_r (right-hand sides still active), next start vector
// v_r = (w_{m+1} - W g_r) / tau_r into slot 0, and per right-hand side
// ||y||^2, ||x||^2, ||v||^2.
template <typename VT>
__global__ void __launch_bounds__(STEP_THREADS) bk_update_kernel(const BlockLaunch B, SmallDev sd, int m_eff,
                                                                  int has_next, double* x, int64_t ldx,
                                                                  const int* active) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[3][BK_WARPS][BK_MAXNB];
  __shared__ ff s_tinv[BK_MAXNB];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nb = B.nb, M = B.m;
  ff* zf = reinterpret_cast<ff*>(smem);  // [m_eff][nb]: z_r scaled by 2^-ez_r
  ff* gf = zf + (size_t)m_eff * nb;     // [m_eff][nb]: -g_r
  __shared__ int s_ez[BK_MAXNB];
  // each z_r enters the float pairs scaled so that max |z_r| is in [1, 2) (a
  // tiny update must not underflow in float); sums are scaled back in float64
  for (int r = threadIdx.x; r < nb; r += blockDim.x) s_ez[r] = INT_MIN;
  __syncthreads();
  for (int e = threadIdx.x; e < m_eff * nb; e += blockDim.x) {
    const int q = e / nb, r = e % nb;
    const double z = offset_sd(sd, B.bs, r).zg[q];
    if (z != 0.0 && isfinite(z)) atomicMax(&s_ez[r], ilogb(z));
  }
  __syncthreads();
  for (int r = threadIdx.x; r < nb; r += blockDim.x)
    if (s_ez[r] == INT_MIN) s_ez[r] = 0;
  __syncthreads();
  for (int e = threadIdx.x; e < m_eff * nb; e += blockDim.x) {
    const int q = e / nb, r = e % nb;
    const SmallDev d = offset_sd(sd, B.bs, r);
    zf[e] = ff_from_double(ldexp(d.zg[q], -s_ez[r]));
    gf[e] = ff_neg(ff_from_double(d.zg[M + q]));
  }
  for (int r = threadIdx.x; r < nb; r += blockDim.x) s_tinv[r] = ff_from_double(offset_sd(sd, B.bs, r).zg[2 * M]);
  __syncthreads();
  VT* const W = static_cast<VT*>(B.W);
  double ay[2] = {0.0, 0.0}, ax[2] = {0.0, 0.0}, av[2] = {0.0, 0.0};
  const int r0 = blockIdx.x * B.rows_p, r1 = min(B.n, r0 + B.rows_p);
  for (int i = r0 + wid; i < r1; i += BK_WARPS) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = lane + 32 * h;
      if (r >= nb) continue;
      const int64_t e = (int64_t)i * nb + r;
      ffacc y, v;
      if (has_next) {
        const ff wm = ldv(W + (int64_t)m_eff * B.slot + e);
        v.S = wm.hi;
        v.E = wm.lo;
      }
      for (int q0 = 0; q0 < m_eff; q0 += 4) {
        ff wv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (q0 + u < m_eff) wv[u] = ldv(W + (int64_t)(q0 + u) * B.slot + e);
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (q0 + u < m_eff) {
            y.add_prod(zf[(q0 + u) * nb + r], wv[u]);
            if (has_next) v.add_prod(gf[(q0 + u) * nb + r], wv[u]);
          }
      }
      const ff yy = y.result();
      const double yd = ldexp((double)yy.hi + (double)yy.lo, s_ez[r]);
      double* xp = x + (int64_t)i * ldx + r;
      const double xn = active[r] ? *xp + yd : *xp;
      *xp = xn;
      if (has_next) {
        const ff vn = stv(W + e, ff_mul(v.result(), s_tinv[r]));
        av[h] = fma((double)vn.hi, (double)vn.hi, av[h]);
      }
      ay[h] = fma(yd, yd, ay[h]);
      ax[h] = fma(xn, xn, ax[h]);
    }
  }
  for (int h = 0; h < 2; ++h) {
    red[0][wid][lane + 32 * h] = ay[h];
    red[1][wid][lane + 32 * h] = ax[h];
    red[2][wid][lane + 32 * h] = av[h];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 3 * nb; e += blockDim.x) {
    const int q = e / nb, r = e % nb;
    double t = 0.0;
    for (int w = 0; w < BK_WARPS; ++w) t += red[q][w][r];
    B.part[((size_t)blockIdx.x * 3 + q) * BK_MAXNB + r] = t;
  }
  if (!last_block_flag(B.counter, &s_last)) return;
  for (int e = wid; e < 3 * nb; e += BK_WARPS) {
    const int q = e / nb, r = e % nb;
    const double t = warp_sum_partials(B.part + (size_t)q * BK_MAXNB + r, (int)gridDim.x, 3 * BK_MAXNB, 0);
    if (lane == 0) offset_cd(B.cd, B.bs, r).scal[q < 2 ? 2 + q : 5] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) *B.counter = 0u;
}

}  // namespace

size_t bk_mat_smem(int s, int nb) { return (size_t)NWB * s * nb * sizeof(int); }

int bk_ctas_per_sm(int kernel, size_t smem) {
  const void* k = (kernel == 0) ? (const void*)bk_mat_kernel<float2, true, 2>
                  : (kernel == 1) ? (const void*)bk_spmv_kernel<float2, float2, 2>
                                  : (const void*)bk_update_kernel<float2>;
  raise_smem_limit(k, smem);
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, STEP_THREADS, smem);
  return std::max(1, b);
}

namespace {

template <typename VT>
void bk_norm_start_t(const BlockLaunch& B, const double* b, int64_t ldb, cudaStream_t st) {
  bk_norm_kernel<<<B.grid, STEP_THREADS, 0, st>>>(B, b, ldb);
  const int64_t total = (int64_t)B.n * B.nb;
  const int g = (int)std::min<int64_t>(4096, (total + 255) / 256);
  bk_start_kernel<VT><<<g, 256, 0, st>>>(B, b, ldb);
}

template <typename VT>
void bk_step_t(const BlockLaunch& B, int mat, int spmv, cudaStream_t st) {
  const size_t smem = bk_mat_smem(B.s, B.nb);
  if (mat) {
    auto k = (B.k <= 2) ? bk_mat_kernel<VT, true, 2> : bk_mat_kernel<VT, true, MAX_WINDOW>;
    raise_smem_limit((const void*)k, smem);
    k<<<B.grid, STEP_THREADS, smem, st>>>(B);
  } else {
    auto k = (B.k <= 2) ? bk_mat_kernel<VT, false, 2> : bk_mat_kernel<VT, false, MAX_WINDOW>;
    raise_smem_limit((const void*)k, smem);
    k<<<B.grid, STEP_THREADS, smem, st>>>(B);
  }
  if (spmv) {
    if (B.val_f32) {
      if (B.k <= 2) bk_spmv_kernel<VT, float, 2><<<B.grid_p, STEP_THREADS, 0, st>>>(B);
      else bk_spmv_kernel<VT, float, MAX_WINDOW><<<B.grid_p, STEP_THREADS, 0, st>>>(B);
    } else {
      if (B.k <= 2) bk_spmv_kernel<VT, float2, 2><<<B.grid_p, STEP_THREADS, 0, st>>>(B);
      else bk_spmv_kernel<VT, float2, MAX_WINDOW><<<B.grid_p, STEP_THREADS, 0, st>>>(B);
    }
  }
}

template <typename VT>
void bk_update_t(const BlockLaunch& B, const SmallDev& sd, int m_eff, int has_next, double* x, int64_t ldx,
                 const int* active, cudaStream_t st) {
  const size_t smem = 2 * (size_t)m_eff * B.nb * sizeof(ff);
  raise_smem_limit((const void*)bk_update_kernel<VT>, smem);
  bk_update_kernel<VT><<<B.grid_p, STEP_THREADS, smem, st>>>(B, sd, m_eff, has_next, x, ldx, active);
}

}  // namespace

void launch_bk_norm_start(const BlockLaunch& B, const double* b, int64_t ldb, cudaStream_t st) {
  if (B.basis32) bk_norm_start_t<float>(B, b, ldb, st);
  else bk_norm_start_t<float2>(B, b, ldb, st);
}

void launch_bk_step(const BlockLaunch& B, int mat, int spmv, cudaStream_t st) {
  if (B.basis32) bk_step_t<float>(B, mat, spmv, st);
  else bk_step_t<float2>(B, mat, spmv, st);
}

void launch_bk_sketch_fin(const BlockLaunch& B, const SmallDev& sd, int ncols, cudaStream_t st) {
  dim3 g((B.s * B.nb + 255) / 256, ncols);
  bk_sketch_fin_kernel<<<g, 256, 0, st>>>(B, sd, ncols);
}

void launch_bk_update(const BlockLaunch& B, const SmallDev& sd, int m_eff, int has_next, double* x, int64_t ldx,
                      const int* active, cudaStream_t st) {
  if (B.basis32) bk_update_t<float>(B, sd, m_eff, has_next, x, ldx, active, st);
  else bk_update_t<float2>(B, sd, m_eff, has_next, x, ldx, active, st);
}

}  // namespace krylov
