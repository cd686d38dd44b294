// step_common.cuh -- device helpers shared by the Arnoldi-step kernels of the
// truncated (step_kernels.cu) and randomized Gram-Schmidt (rgs_kernels.cu)
// cycles: the last-CTA ticket, columns of the sparse sign embedding S (stored
// table or regenerated), the exact fixed-point sketch bins, and float-float
// loads, accumulators and block sums.
#pragma once

#include "internal.h"
#include "kernels.cuh"

namespace krylov {
namespace {

constexpr int NQ = 2 + MAX_WINDOW;  // scalar partials per CTA: ||w||^2, ||p||^2, dots
constexpr int MAX_WARPS = 32;       // warps of the largest CTA (1024 threads)
constexpr unsigned FULL = 0xffffffffu;

// Arrival ticket of the deterministic "last CTA reduces" pattern: true in the
// CTA that arrives last (it then sums the per-CTA partials in a fixed order).
__device__ __forceinline__ bool last_block_flag(unsigned* counter, int* s_last) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) *s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (*s_last) __threadfence();
  return *s_last != 0;
}

// Column i of S held by one lane: the entries (row, negative) e = 0..zeta-1,
// from the stored table or regenerated with the counter-based generator.
template <int SKM> struct SkCol {
  uint32_t p0 = 0xFFFFFFFFu, p1 = 0xFFFFFFFFu, ng = 0u;
  int got = 0;
  const uint16_t* r16 = nullptr;
  __device__ __forceinline__ void load(const StepLaunch& L, const SketchSpec& sp, uint32_t inv_s, int i) {
    if constexpr (SKM == SK_TAB8) {
      const uint2 r = __ldg(L.sk_tab.rows8 + i);
      p0 = r.x;
      p1 = r.y;
      ng = __ldg(L.sk_tab.neg8 + i);
      got = sp.zeta;
    } else if constexpr (SKM == SK_TAB16) {
      r16 = L.sk_tab.rows16 + (size_t)i * sp.zeta;
      ng = __ldg(L.sk_tab.neg32 + i);
      got = sp.zeta;
    } else if constexpr (SKM == SK_GEN8) {
      got = sketch_column_packed((uint32_t)i, sp, inv_s, &p0, &p1, &ng);
    }
  }
  __device__ __forceinline__ int row(int e) const {
    if constexpr (SKM == SK_TAB16) return (int)__ldg(r16 + e);
    return (int)(((e < 4 ? p0 : p1) >> (8 * (e & 3))) & 0xFFu);
  }
  __device__ __forceinline__ bool neg(int e) const { return (ng >> e) & 1u; }
};

// Generic regeneration (any s <= 32768, zeta <= 32): entries kept in a local array.
struct SkColGen {
  int rows[MAX_ZETA];
  uint32_t ng = 0u;
  int got = 0;
  __device__ __forceinline__ void load(const StepLaunch& L, const SketchSpec& sp, uint32_t inv_s, int i) {
    (void)L;
    (void)inv_s;
    got = 0;
    ng = 0u;
    sketch_column<MAX_ZETA>((uint32_t)i, sp, [&](int r, bool n) {
      rows[got] = r;
      ng |= (n ? 1u : 0u) << got;
      ++got;
    });
  }
  __device__ __forceinline__ int row(int e) const { return rows[e]; }
  __device__ __forceinline__ bool neg(int e) const { return (ng >> e) & 1u; }
};

template <int SKM> struct SkColOf { using type = SkCol<SKM>; };
template <> struct SkColOf<SK_GEN> { using type = SkColGen; };

// ---- exact fixed-point sketch bins ---------------------------------------
// A contribution v with |v| <= B is scaled by the power of two 2^(WB - E),
// E >= ceil(log2 B) + 1, so |x| < 2^(WB-1), and split into NW integer words
// x = q_0 + 2^-WB q_1 + 2^-2WB q_2 + ... + remainder, rounding with the
// 1.5 * 2^23 addition trick on the FP32 pipes: |q_0| <= 2^(WB-1), and a later
// word holds a rounding remainder (at most 1/2) plus the low part carried
// along, |q_w| < 1.2 * 2^(WB-1); what the last word leaves out (its rounding
// remainder and the low part dropped there) is below 0.6 * 2^-(NW-1)WB.  Word w of bin b
// lives in a lane-private column (address (w s + b) C + copy), so the integer
// atomic adds of a warp hit distinct banks; integer sums are exact and
// independent of the order in which threads arrive.  WB is chosen on the host
// so that no column can overflow (entries per column <= rows per CTA / C).
struct FxScale {
  float to_fixed;  // 2^(WB - E)
  float word;      // 2^WB
  int E;
};

template <int NW> struct FxWords {
  int q[NW];
};

// Split the contribution (h + l) of one row into its fixed-point words (once
// per row: every entry of the row adds the same value up to its sign).
template <int NW>
__device__ __forceinline__ FxWords<NW> fx_split(float h, float l, const FxScale& f) {
  const float magic = 12582912.0f;  // 1.5 * 2^23
  FxWords<NW> out;
  h = __fmul_rn(h, f.to_fixed);
  l = __fmul_rn(l, f.to_fixed);
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const float r = __fadd_rn(h, magic);
    out.q[w] = __float_as_int(r) - 0x4B400000;
    if (w + 1 < NW) {
      const ff d = two_sum(__fsub_rn(h, __fsub_rn(r, magic)), l);
      h = __fmul_rn(d.hi, f.word);
      l = __fmul_rn(d.lo, f.word);
    }
  }
  return out;
}

// Add +-words to bin `row` in this lane's column.
template <int NW>
__device__ __forceinline__ void fx_emit(int* bins, int sC, int row, int cp, const FxWords<NW>& x, bool neg,
                                        int C) {
  int* b = bins + row * C + cp;
#pragma unroll
  for (int w = 0; w < NW; ++w) atomicAdd(b + w * sC, neg ? -x.q[w] : x.q[w]);
}

// 2^k as a double, built from its exponent field (no FP64 arithmetic) in the
// normal range; ldexp outside it.
__device__ __forceinline__ double pow2d(int k) {
  return (k >= -1022 && k <= 1023) ? __longlong_as_double((long long)(k + 1023) << 52) : ldexp(1.0, k);
}

// Value of bin b of this CTA: sum of its words over the copies, as a double.
// Thread b starts at copy b mod C, so the lanes of a warp read C different
// banks at every step instead of all hitting one (integer sums: any order).
// The last two word sums are merged exactly in 64-bit integers (a word sum is
// below 2^35 in magnitude and WB <= 21, so t 2^WB + t' stays below 2^57),
// which leaves two conversions and power-of-two scalings: the FP64 pipe,
// shared by the CTAs of an SM, is what this per-CTA epilogue waits on.
template <int NW>
__device__ __forceinline__ double fx_value(const int* bins, int s, int C, int b, const FxScale& f, int WB) {
  static_assert(NW == 2 || NW == 3, "two or three fixed-point words");
  long long t[NW];
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    long long u = 0;
    const int* col = bins + (w * s + b) * C;
    for (int c = 0; c < C; ++c) u += col[(c + b) & (C - 1)];
    t[w] = u;
  }
  const long long low = t[NW - 2] * (1ll << WB) + t[NW - 1];
  const double vlow = (double)low * pow2d(f.E - NW * WB);
  if (NW == 2) return vlow;
  return fma((double)t[0], pow2d(f.E - WB), vlow);
}

__device__ __forceinline__ FxScale fx_scale(const StepLaunch& L, const CycleDev& cd, int mat) {
  // materialized column: the bound the previous product's reducer stored;
  // first column of a cycle: the bound of the start vector
  double B = mat ? cd.scal[6] : sqrt(cd.scal[5]);
  B = B * 1.0001 + 1e-300;
  FxScale f;
  f.E = ilogb(B) + 2;  // 2^(E-1) > B
  f.to_fixed = ldexpf(1.0f, L.fx_wb - f.E);
  f.word = ldexpf(1.0f, L.fx_wb);
  return f;
}

__host__ __device__ __forceinline__ size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// fixed-point sketch bins of a CTA: words x s x copies ints
__host__ __device__ __forceinline__ int fx_words(int basis) { return (basis == 0 || basis == 3) ? 3 : 2; }
__host__ __device__ __forceinline__ size_t bins_bytes(int basis, int s, int copies) {
  return (size_t)fx_words(basis) * s * copies * sizeof(int);
}

__device__ __forceinline__ SketchSpec spec_of(const StepLaunch& L) {
  SketchSpec t;
  t.s = L.s;
  t.zeta = L.zeta;
  t.lim = 32768u - 32768u % (uint32_t)L.s;
  t.k0 = (uint32_t)(L.seed & 0xFFFFFFFFull);
  t.k1 = (uint32_t)(L.seed >> 32);
  t.scale = 1.f;
  return t;
}

// ---- reducers of the step kernels ------------------------------------------
// The reducers run in the last CTA of a kernel while the rest of the GPU
// waits for it, and every float64 instruction of a lone warp holds the FP64
// pipe of its SM sub-partition for many cycles: so all loads come before any
// store (the stores may alias them, which would serialize round trips to L2),
// the window slots are handled by parallel lanes, and no quotient or square
// root is formed that another one already gives.

// Reducer of a materialized column j (lane 0): record ||w_j||^2 and flag a
// happy breakdown when ||w_j|| / rho_j, the norm of the orthogonalized
// product, is below thr ||A w_{j-1}||.  1 / rho_j = R[j, j-1] was stored by
// the reducer of the product p_{j-1}; the test is taken on squares.  Returns
// whether the cycle has ended in breakdown.
__device__ __forceinline__ bool reduce_mat(const StepLaunch& L, const CycleDev& cd, double sig2, int mat) {
  const int j = L.j;
  const int ldr = L.m + 1;  // R is (m+1) x m, column-major
  const double rsub = mat ? __ldcg(cd.R + (size_t)(j - 1) * ldr + j) : 0.0;
  const double pprev = mat ? __ldcg(cd.pi + j - 1) : 0.0;
  int brk = __ldcg(cd.flags + 1);
  cd.sig2[j] = sig2;
  if (!isfinite(sig2)) cd.flags[2] |= ERR_NONFINITE;
  if (mat) {
    const double rn2 = sig2 * (rsub * rsub);
    if (!(rn2 > (L.thr * L.thr) * pprev) && brk == 0) {
      cd.flags[1] = 1;
      cd.flags[0] = j;
      brk = 1;
    }
  }
  return brk != 0;
}

// Reducer of a product p_j = A w_j (one warp; lane q takes window slot
// dlo + q): projection coefficients h_q = <w_q, p_j> / ||w_q||^2, R[q, j] =
// h_q, the scale rho_{j+1} = 1 / sqrt(||p_j||^2 - sum_q h_q^2 ||w_q||^2) of
// the next column (the window is orthogonal) with R[j+1, j] = 1 / rho_{j+1},
// and the bound rho_{j+1} (||p_j|| + sum_q |h_q| ||w_q||) on |w_{j+1}[i]|
// (triangle inequality) for the next materialization's fixed-point sketch.
// brk: the cycle has already ended in breakdown (no further coefficients).
// own_s2: ||w_j||^2 when this kernel formed w_j itself (its reducer has only
// just stored it), negative otherwise (read from memory).
__device__ __forceinline__ void reduce_spmv(const StepLaunch& L, const CycleDev& cd, const double* tot, bool brk,
                                            double own_s2 = -1.0) {
  const int lane = threadIdx.x & 31;
  const int j = L.j;
  const int ldr = L.m + 1;
  const int dlo = max(0, j - L.k + 1);
  const int slot = dlo + lane;
  const bool inwin = !L.rgs && lane < MAX_WINDOW && slot <= j;
  const double s2 = !inwin ? 0.0 : ((slot == j && own_s2 >= 0.0) ? own_s2 : __ldcg(cd.sig2 + slot));
  const double pi = tot[1];
  const double dq = inwin ? tot[2 + lane] : 0.0;
  if (brk) return;
  if (lane == 0) {
    cd.pi[j] = pi;
    if (!isfinite(pi)) cd.flags[2] |= ERR_NONFINITE;
  }
  if (L.rgs) return;  // the sketch-space orthogonalization takes it from here
  const double h = (inwin && s2 > 0.0) ? dq / s2 : 0.0;
  double e2 = h * h * s2;
  double bq = inwin ? fabs(h) * sqrt(s2) : 0.0;
  static_assert(MAX_WINDOW == 4, "window sums over groups of four lanes");
  e2 += __shfl_xor_sync(FULL, e2, 1);
  e2 += __shfl_xor_sync(FULL, e2, 2);
  bq += __shfl_xor_sync(FULL, bq, 1);
  bq += __shfl_xor_sync(FULL, bq, 2);
  double* c = cd.coef + (size_t)j * (MAX_WINDOW + 1);
  if (inwin) cd.R[(size_t)j * ldr + slot] = h;
  if (lane < MAX_WINDOW) c[lane] = h;
  if (lane == 0) {
    const double est = fmax(pi - e2, 1e-20 * pi);
    const double r = (pi > 0.0) ? sqrt(est) : 1.0;  // 1 / rho_{j+1}
    const double rho = 1.0 / r;
    c[MAX_WINDOW] = rho;
    cd.R[(size_t)j * ldr + j + 1] = r;
    cd.scal[6] = (sqrt(pi) + bq) * rho;
  }
}

// ---------------------------------------------------------------------------
// Float-float basis ("df64"): (hi, lo) float pairs, arithmetic on the FP32
// pipes.

__device__ __forceinline__ ff ld_ff(const float2* p) {
  const float2 v = __ldg(p);
  return {v.x, v.y};
}
__device__ __forceinline__ void st_ff(float2* p, ff v) { *p = make_float2(v.hi, v.lo); }

// Compensated accumulation: S + E tracks a sum of float-float products.
struct ffacc {
  float S = 0.f, E = 0.f;
  __device__ __forceinline__ void add_prod(ff a, ff w) {
    const float p = __fmul_rn(a.hi, w.hi);
    float e = __fmaf_rn(a.hi, w.hi, -p);
    e = __fmaf_rn(a.hi, w.lo, e);
    e = __fmaf_rn(a.lo, w.hi, e);
    add_pe(p, e);
  }
  __device__ __forceinline__ void add_pe(float p, float e) {
    const ff t = two_sum(S, p);
    S = t.hi;
    E = __fadd_rn(E, __fadd_rn(t.lo, e));
  }
  __device__ __forceinline__ ff result() const { return fast_two_sum(S, E); }
};

// product of a matrix value and a float-float entry as (p, e), p + e accurate
// to float-float precision
__device__ __forceinline__ float2 prod_pe(float a, ff w) {
  const float p = __fmul_rn(a, w.hi);
  float e = __fmaf_rn(a, w.hi, -p);
  e = __fmaf_rn(a, w.lo, e);
  return make_float2(p, e);
}
__device__ __forceinline__ float2 prod_pe(float2 a, ff w) {
  const float p = __fmul_rn(a.x, w.hi);
  float e = __fmaf_rn(a.x, w.hi, -p);
  e = __fmaf_rn(a.x, w.lo, e);
  e = __fmaf_rn(a.y, w.hi, e);
  return make_float2(p, e);
}

// Block-wide float-float sum, result (as double) in thread 0.
// Block-wide float-float sum in a fixed order (warp shuffle tree, then the
// warp sums in warp order), kept as a pair; valid in thread 0.
__device__ __forceinline__ ff block_sum_ff_pair(ff v, float* sh_hi, float* sh_lo) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const ff u{__shfl_xor_sync(FULL, v.hi, o), __shfl_xor_sync(FULL, v.lo, o)};
    v = ff_add(v, u);
  }
  __syncthreads();
  if (lane == 0) {
    sh_hi[wid] = v.hi;
    sh_lo[wid] = v.lo;
  }
  __syncthreads();
  ff a{0.f, 0.f};
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a = ff_add(a, ff{sh_hi[w], sh_lo[w]});
  return a;
}

__device__ __forceinline__ double block_sum_ff(ff v, float* sh_hi, float* sh_lo) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const ff u{__shfl_xor_sync(FULL, v.hi, o), __shfl_xor_sync(FULL, v.lo, o)};
    v = ff_add(v, u);
  }
  __syncthreads();
  if (lane == 0) {
    sh_hi[wid] = v.hi;
    sh_lo[wid] = v.lo;
  }
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    ff a{0.f, 0.f};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a = ff_add(a, ff{sh_hi[w], sh_lo[w]});
    r = ff_to_double(a);
  }
  return r;
}

// ---- float-float reductions of the step scalars ---------------------------
// The scalars of a step (||p||^2, the window dots, ||w||^2) are summed over
// CTAs and turned into the next column's coefficients by the CTA that arrives
// last while the rest of the GPU waits on it.  Float64 is slow there: a warp
// instruction holds an FP64 pipe for tens of cycles whatever its active lanes,
// and a division or square root is a chain of them.  So the float-float step
// kernels keep these partials as float-float pairs (in the float64 slots of
// the partials array), sum and divide them on the FP32 pipes, and form float64
// only for the values the host and the projected problem read.

// a / b in float-float: a float quotient and one exact correction (Dekker
// 1971, "div2"); b must be nonzero.
__device__ __forceinline__ ff ff_div(ff a, ff b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const ff r = ff_add(a, ff_neg(ff_mul_f(b, q1)));  // a - q1 b
  return fast_two_sum(q1, __fdiv_rn(r.hi, b.hi));
}

// sqrt(a) in float-float for a >= 0: the float root and one Newton
// correction with the exact residual a - s^2 (Dekker 1971, "sqrt2").
__device__ __forceinline__ ff ff_sqrt(ff a) {
  if (!(a.hi > 0.f)) return ff{0.f, 0.f};
  const float s = __fsqrt_rn(a.hi);
  const float p = __fmul_rn(s, s);
  const float pe = __fmaf_rn(s, s, -p);  // s^2 = p + pe exactly
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), pe), a.lo);
  return fast_two_sum(s, __fdiv_rn(r, __fmul_rn(2.f, s)));
}

__device__ __forceinline__ void st_part_ff(double* slot, ff v) {
  *reinterpret_cast<float2*>(slot) = make_float2(v.hi, v.lo);
}

// CTA partials of nv <= NV float-float values (warp shuffle trees, then the
// warps in order, the order of block_sum_ff): lane q of warp 0 stores value q
// at part[q0 + q].  One block barrier.
template <int NV>
__device__ __forceinline__ void block_partials_ff(ff (&v)[NV], int nv, double* part, int q0, float2 (*sh)[NV]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      v[q] = ff_add(v[q], ff{__shfl_xor_sync(FULL, v[q].hi, o), __shfl_xor_sync(FULL, v[q].lo, o)});
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[wid][q] = make_float2(v[q].hi, v[q].lo);
  __syncthreads();
  if (wid == 0 && lane < nv) {
    ff a{0.f, 0.f};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a = ff_add(a, ff{sh[w][lane].x, sh[w][lane].y});
    st_part_ff(part + q0 + lane, a);
  }
}

// Column sums q0 .. q0 + nv - 1 (nv <= NV) of a count x stride array of
// float-float CTA partials, by the whole block in a fixed order: thread t
// adds rows t, t + T, t + 2T, ... (four rows per column in flight), then a
// shuffle tree per warp, then the warps in order.  A second array (part2,
// count2; count2 = 0 for none) is summed the same way and added.  The sums
// land in out[0 .. nv) (shared memory) for every thread and depend only on
// the counts.
template <int NV>
__device__ __forceinline__ void block_sum_partials_ff(const double* part, int count, const double* part2, int count2,
                                                      int stride, int q0, int nv, float2 (*sh)[NV], ff* out) {
  constexpr int B = 4;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, T = (int)blockDim.x;
  ff acc[2][NV];
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const double* pa = a ? part2 : part;
    const int ca = a ? count2 : count;
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[a][q] = ff{0.f, 0.f};
    for (int c0 = (int)threadIdx.x; c0 < ca; c0 += B * T) {
      float2 x[B][NV];
#pragma unroll
      for (int u = 0; u < B; ++u)
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          const int c = c0 + u * T;
          x[u][q] = (c < ca && q < nv) ? __ldcg(reinterpret_cast<const float2*>(pa + (size_t)c * stride + q0 + q))
                                       : make_float2(0.f, 0.f);
        }
#pragma unroll
      for (int u = 0; u < B; ++u)
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[a][q] = ff_add(acc[a][q], ff{x[u][q].x, x[u][q].y});
    }
#pragma unroll
    for (int q = 0; q < NV; ++q)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
        acc[a][q] = ff_add(acc[a][q], ff{__shfl_xor_sync(FULL, acc[a][q].hi, o), __shfl_xor_sync(FULL, acc[a][q].lo, o)});
    if (count2 <= 0) break;
  }
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q)
      sh[wid][q] = make_float2(acc[0][q].hi, acc[0][q].lo);
  __syncthreads();
  if (threadIdx.x < nv) {
    const int q = (int)threadIdx.x;
    ff a{0.f, 0.f};
    for (int w = 0; w < T / 32; ++w) a = ff_add(a, ff{sh[w][q].x, sh[w][q].y});
    out[q] = a;
  }
  __syncthreads();
  if (count2 > 0) {  // the second array, in the same order, added last
    if (lane == 0)
#pragma unroll
      for (int q = 0; q < NV; ++q) sh[wid][q] = make_float2(acc[1][q].hi, acc[1][q].lo);
    __syncthreads();
    if (threadIdx.x < nv) {
      const int q = (int)threadIdx.x;
      ff a{0.f, 0.f};
      for (int w = 0; w < T / 32; ++w) a = ff_add(a, ff{sh[w][q].x, sh[w][q].y});
      out[q] = ff_add(out[q], a);
    }
    __syncthreads();
  }
}

// Coefficients of column j >= 1 for the float-float materialize kernels,
// formed by every CTA from the CTA partials of the kernels before it, so that
// no last-CTA reducer sits between two kernels: ||w_{j-1}||^2 from the
// previous materialize kernel (with the happy-breakdown test of column j-1),
// ||p_{j-1}||^2 and the window dots <w_q, p_{j-1}> from the product
// kernel(s).  Every CTA sums the same partials in the same order and so holds
// the same values.  h_q = <w_q, p> / ||w_q||^2, rho_j = 1 / sqrt(||p||^2 -
// sum_q h_q <w_q, p>) (the window is orthogonal), R[j, j-1] = 1 / rho_j, and
// rho_j (||p|| + sum_q |h_q| ||w_q||) bounds |w_j[i]| (triangle inequality):
// it sets the fixed-point scale of the sketch.  Everything here runs on the
// FP32 pipes; CTA 0 stores the float-float pairs the next kernel reads at
// once and the float64 values for the host and the projected problem after
// its rows (mat_coefficients_store).  Returns false when the cycle ended
// before column j, or column j-1 ends it (flags set by CTA 0): nothing to
// materialize.
struct MatCoef {
  ff h[MAX_WINDOW];  // -h_q, ready to add
  ff rho, r, sig2, pi;
  float bound;
  FxScale fx;
  int ok, nd;
};

template <int KW>
__device__ __forceinline__ bool mat_coefficients(const StepLaunch& L, const CycleDev& cd, MatCoef& out) {
  constexpr int NP = 1 + KW;  // product columns: ||p||^2, dots
  constexpr int B = 4;        // rows per thread in flight per array
  __shared__ float2 sh[MAX_WARPS][1 + NP];
  __shared__ ff tot[1 + NP];  // [0] ||w_{j-1}||^2, [1] ||p_{j-1}||^2, [2 + q] <w_{dlo+q}, p_{j-1}>
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, T = (int)blockDim.x;
  const int jp = L.j - 1;
  const int dlo = max(0, jp - L.k + 1);
  const int nd = jp - dlo + 1;
  // warp 0: the flags, the older window norms and the inputs of the
  // breakdown test, issued with the partial sums so that the round trips
  // overlap
  ff s2{0.f, 0.f}, rsub{0.f, 0.f}, pprev{0.f, 0.f};
  int m_eff = 0;
  if (wid == 0) {
    const int slot = dlo + lane;
    if (lane < nd && slot < jp) {
      const float2 v = __ldcg(cd.sig2ff + slot);
      s2 = ff{v.x, v.y};
    }
    if (lane == 0) {
      m_eff = __ldcg(cd.flags);
      if (jp >= 1) {
        const float2 r = __ldcg(cd.rff + jp - 1), p = __ldcg(cd.piff + jp - 1);
        rsub = ff{r.x, r.y};
        pprev = ff{p.x, p.y};
      }
    }
  }
  // the partials, in a fixed order per thread: rows t, t + T, ... of each array
  const double* pw = L.part_w + (size_t)(jp & 1) * L.part_w_stride;
  const int cw = (int)gridDim.x, cp = L.grid_spmv;  // the materialize kernels of a cycle share a grid
  ff aw{0.f, 0.f}, ap[NP], al[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) ap[q] = al[q] = ff{0.f, 0.f};
  for (int c0 = (int)threadIdx.x; c0 < max(cw, cp); c0 += B * T) {
    float2 xw[B], xp[B][NP];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int c = c0 + u * T;
      xw[u] = (c < cw) ? __ldcg(reinterpret_cast<const float2*>(pw + c)) : make_float2(0.f, 0.f);
#pragma unroll
      for (int q = 0; q < NP; ++q)
        xp[u][q] = (c < cp && q <= nd) ? __ldcg(reinterpret_cast<const float2*>(L.part + (size_t)c * NQ + 1 + q))
                                       : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
      aw = ff_add(aw, ff{xw[u].x, xw[u].y});
#pragma unroll
      for (int q = 0; q < NP; ++q) ap[q] = ff_add(ap[q], ff{xp[u][q].x, xp[u][q].y});
    }
  }
  if (L.n_long > 0)  // the long-row kernel's partials, summed apart and added last
    for (int c = (int)threadIdx.x; c < L.grid_long; c += T)
#pragma unroll
      for (int q = 0; q < NP; ++q)
        if (q <= nd) {
          const float2 x = __ldcg(reinterpret_cast<const float2*>(L.part_long + (size_t)c * NQ + 1 + q));
          al[q] = ff_add(al[q], ff{x.x, x.y});
        }
  auto tree = [&](ff& v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = ff_add(v, ff{__shfl_xor_sync(FULL, v.hi, o), __shfl_xor_sync(FULL, v.lo, o)});
  };
  tree(aw);
#pragma unroll
  for (int q = 0; q < NP; ++q) tree(ap[q]);
  if (lane == 0) {
    sh[wid][0] = make_float2(aw.hi, aw.lo);
#pragma unroll
    for (int q = 0; q < NP; ++q) sh[wid][1 + q] = make_float2(ap[q].hi, ap[q].lo);
  }
  __syncthreads();
  if (threadIdx.x < 1 + NP) {
    ff a{0.f, 0.f};
    for (int w = 0; w < T / 32; ++w) a = ff_add(a, ff{sh[w][threadIdx.x].x, sh[w][threadIdx.x].y});
    tot[threadIdx.x] = a;
  }
  if (L.n_long > 0) {
#pragma unroll
    for (int q = 0; q < NP; ++q) tree(al[q]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
      for (int q = 0; q < NP; ++q) sh[wid][1 + q] = make_float2(al[q].hi, al[q].lo);
    __syncthreads();
    if (threadIdx.x >= 1 && threadIdx.x < 1 + NP) {
      ff a{0.f, 0.f};
      for (int w = 0; w < T / 32; ++w) a = ff_add(a, ff{sh[w][threadIdx.x].x, sh[w][threadIdx.x].y});
      tot[threadIdx.x] = ff_add(tot[threadIdx.x], a);
    }
  }
  __syncthreads();
  if (wid == 0) {
    const bool cta0 = (blockIdx.x == 0);
    const ff sig2 = tot[0], pi = tot[1];
    // the cycle ended before column j (an earlier breakdown): nothing to do;
    // else the happy breakdown of column j-1: ||w_{j-1}|| R[j-1, j-2] <
    // thr ||A w_{j-2}|| (as reduce_mat, on roots)
    int stop = 0;
    if (lane == 0) {
      if (m_eff < L.j) {
        stop = 2;
      } else if (jp >= 1 &&
                 !(__fsqrt_rn(sig2.hi) * rsub.hi > (float)L.thr * __fsqrt_rn(pprev.hi))) {
        stop = 1;
      }
    }
    stop = __shfl_sync(FULL, stop, 0);
    if (stop) {
      if (lane == 0) {
        out.ok = 0;
        if (cta0 && stop == 1) {
          cd.sig2[jp] = ff_to_double(sig2);
          cd.sig2ff[jp] = make_float2(sig2.hi, sig2.lo);
          cd.flags[1] = 1;
          cd.flags[0] = jp;
        }
      }
    } else {
      const int slot = dlo + lane;
      const bool inwin = lane < nd;
      const ff s2q = (slot == jp) ? sig2 : s2;
      const ff dq = inwin ? tot[2 + lane] : ff{0.f, 0.f};
      const ff h = (inwin && s2q.hi > 0.f) ? ff_div(dq, s2q) : ff{0.f, 0.f};
      ff e2 = ff_mul(h, dq);  // h_q^2 ||w_q||^2 = h_q <w_q, p>
      float bq = inwin ? fabsf(h.hi) * __fsqrt_rn(s2q.hi) : 0.f;
      static_assert(MAX_WINDOW == 4, "window sums over groups of four lanes");
#pragma unroll
      for (int o = 1; o <= 2; o <<= 1) {
        e2 = ff_add(e2, ff{__shfl_xor_sync(FULL, e2.hi, o), __shfl_xor_sync(FULL, e2.lo, o)});
        bq += __shfl_xor_sync(FULL, bq, o);
      }
      if (lane < MAX_WINDOW) out.h[lane] = ff_neg(h);
      if (lane == 0) {
        ff r{1.f, 0.f}, rho{1.f, 0.f};
        if (pi.hi > 0.f) {
          const ff est = ff_add(pi, ff_neg(e2));
          const float fl = 1e-20f * pi.hi;
          if (est.hi > fl && fl > 0.f) {
            r = ff_sqrt(est);
            rho = ff_div(ff{1.f, 0.f}, r);
          } else {  // (nearly) in the window's span, or a tiny product: floor in float64
            const double pd = ff_to_double(pi);
            const double rd = sqrt(fmax(pd - ff_to_double(e2), 1e-20 * pd));
            r = ff_from_double(rd);
            rho = ff_from_double(1.0 / rd);
          }
        }
        // float bound; the margin 1.0001 covers its roundings (as fx_scale)
        const float bound = (__fsqrt_rn(pi.hi) + bq) * rho.hi;
        FxScale f;
        const float bm = bound * 1.0001f;
        f.E = (bm >= 1.17549435e-38f && bm < 3.0e38f) ? ilogbf(bm) + 2 : ilogb((double)bound * 1.0001 + 1e-300) + 2;
        f.to_fixed = ldexpf(1.0f, L.fx_wb - f.E);
        f.word = ldexpf(1.0f, L.fx_wb);
        out.rho = rho;
        out.r = r;
        out.sig2 = sig2;
        out.pi = pi;
        out.bound = bound;
        out.nd = nd;
        out.fx = f;
        out.ok = 1;
        if (cta0) {  // the pairs the next materialize kernel reads
          cd.sig2ff[jp] = make_float2(sig2.hi, sig2.lo);
          cd.piff[jp] = make_float2(pi.hi, pi.lo);
          cd.rff[jp] = make_float2(r.hi, r.lo);
        }
      }
    }
  }
  __syncthreads();
  return out.ok != 0;
}

// CTA 0 of a materialize kernel, after its rows: the float64 values of column
// j-1 for the host and the projected problem (||w_{j-1}||^2, ||p_{j-1}||^2,
// R[:, j-1], the coefficients, the sketch bound), from mat_coefficients.
__device__ __forceinline__ void mat_coefficients_store(const StepLaunch& L, const CycleDev& cd, const MatCoef& c) {
  const int jp = L.j - 1, ldr = L.m + 1, dlo = max(0, jp - L.k + 1);
  const int t = (int)threadIdx.x;
  double* co = cd.coef + (size_t)jp * (MAX_WINDOW + 1);
  if (t < MAX_WINDOW) {
    const double hq = -ff_to_double(c.h[t]);
    co[t] = hq;
    if (t < c.nd) cd.R[(size_t)jp * ldr + dlo + t] = hq;
  } else if (t == MAX_WINDOW) {
    co[MAX_WINDOW] = ff_to_double(c.rho);
    cd.R[(size_t)jp * ldr + jp + 1] = ff_to_double(c.r);
  } else if (t == MAX_WINDOW + 1) {
    const double s2 = ff_to_double(c.sig2);
    cd.sig2[jp] = s2;
    if (!isfinite(s2)) atomicOr(&cd.flags[2], ERR_NONFINITE);
  } else if (t == MAX_WINDOW + 2) {
    const double pd = ff_to_double(c.pi);
    cd.pi[jp] = pd;
    if (!isfinite(pd)) atomicOr(&cd.flags[2], ERR_NONFINITE);
  } else if (t == MAX_WINDOW + 3) {
    cd.scal[6] = (double)c.bound;
  }
}

// Exact sketch of a column over all CTAs: each CTA adds its bins' word sums
// (over the lane copies, in int64) to the column's accumulator [3][s] with
// integer atomics, so the total is exact and independent of the order in
// which CTAs arrive; the projected problem's U is formed from it once per
// cycle.  word(b, c, w): word w < NW of copy c of bin b in shared memory;
// thread p sums pair (b, w) = (p / NW, p % NW) starting at copy b (bank
// spread).  With NW = 2 (float32 values) the third word of the accumulator
// stays zero.
template <int NW = 3, typename Word>
__device__ __forceinline__ void fx_accumulate(Word word, int s, int C, unsigned long long* acc) {
  for (int p = (int)threadIdx.x; p < NW * s; p += (int)blockDim.x) {
    const int b = p / NW, w = p - NW * b;
    long long u = 0;
#pragma unroll 8
    for (int c = 0; c < C; ++c) u += word(b, (c + b) & (C - 1), w);
    if (u != 0) atomicAdd(acc + (size_t)w * s + b, (unsigned long long)u);
  }
}

// The accumulator of column j of the float-float materialize kernels:
// [3][s] int64 word sums, then the exponent E of its fixed-point scale.
__device__ __forceinline__ unsigned long long* fx_acc_of(const StepLaunch& L, int j) {
  return reinterpret_cast<unsigned long long*>(L.sk_acc) + (size_t)j * L.sk_acc_stride;
}

// Reducer of ||p_j||^2 for the randomized Gram-Schmidt cycle (lane 0): the
// sketch-space orthogonalization takes it from there.
__device__ __forceinline__ void reduce_pi_ff(const StepLaunch& L, const CycleDev& cd, ff pi, bool brk) {
  if (brk) return;
  cd.pi[L.j] = ff_to_double(pi);
  if (!isfinite(pi.hi)) cd.flags[2] |= ERR_NONFINITE;
}

// Partial of ||w_j||^2 of a float-float materialize kernel's CTA, in the half
// j & 1 of part_w (the next materialize kernel reads the other half while
// this one writes).
__device__ __forceinline__ double* part_w_of(const StepLaunch& L, int j) {
  return L.part_w + (size_t)(j & 1) * L.part_w_stride;
}

// Last column of a cycle (no materialize kernel follows): the CTA that
// arrives last sums the ||w_m||^2 partials and records it with the breakdown
// test of column m (as reduce_mat), for the host and the projected problem.
__device__ __forceinline__ void ff_mat_finish(const StepLaunch& L, const CycleDev& cd, int mat) {
  __shared__ float2 sh[MAX_WARPS][1];
  __shared__ ff s_tot[1];
  __shared__ int s_last;
  if (!last_block_flag(cd.counter, &s_last)) return;
  const int j = L.j;
  float2 rsub{0.f, 0.f}, pprev{0.f, 0.f};
  int brk = 0;
  if (threadIdx.x == 0) {  // issued before the partial sums
    if (mat) {
      rsub = __ldcg(cd.rff + j - 1);
      pprev = __ldcg(cd.piff + j - 1);
    }
    brk = __ldcg(cd.flags + 1);
  }
  block_sum_partials_ff<1>(part_w_of(L, j), (int)gridDim.x, nullptr, 0, 1, 0, 1, sh, s_tot);
  if (threadIdx.x == 0) {
    const ff sig2 = s_tot[0];
    const double s2 = ff_to_double(sig2);
    cd.sig2[j] = s2;
    cd.sig2ff[j] = make_float2(sig2.hi, sig2.lo);
    if (!isfinite(s2)) cd.flags[2] |= ERR_NONFINITE;
    // the breakdown test of mat_coefficients
    if (mat && !(__fsqrt_rn(sig2.hi) * rsub.x > (float)L.thr * __fsqrt_rn(pprev.x)) && brk == 0) {
      cd.flags[1] = 1;
      cd.flags[0] = j;
    }
    *cd.counter = 0u;
  }
}

// Epilogue of a float-float product kernel: the CTA's ||p_j||^2 and window
// dots as float-float partials (columns 1, 2, ... of the partials), which the
// next materialize kernel's CTAs sum.  In a randomized Gram-Schmidt cycle
// (reduce set) the CTA that arrives last sums ||p_j||^2 (with the long-row
// kernel's partials, part2 / count2) and records it.
template <int KW>
__device__ __forceinline__ void ff_spmv_finish(const StepLaunch& L, const CycleDev& cd, const ffacc& acc_pi,
                                               const ffacc (&acc_dot)[KW], int nd, double* part_cta, bool reduce,
                                               const double* part, int count, const double* part2, int count2) {
  __shared__ float2 sh[MAX_WARPS][1 + KW];
  __shared__ ff s_tot[1 + KW];
  __shared__ int s_last;
  ff v[1 + KW];
  v[0] = acc_pi.result();
#pragma unroll
  for (int q = 0; q < KW; ++q) v[1 + q] = acc_dot[q].result();
  block_partials_ff<1 + KW>(v, 1 + nd, part_cta, 1, sh);
  if (!reduce) return;
  if (!last_block_flag(cd.counter, &s_last)) return;
  const int brk = __ldcg(cd.flags + 1);
  block_sum_partials_ff<1 + KW>(part, count, part2, count2, NQ, 1, 1, sh, s_tot);
  if (threadIdx.x == 0) {
    reduce_pi_ff(L, cd, s_tot[0], brk != 0);
    *cd.counter = 0u;
  }
}

// Launch with programmatic stream serialization and a block of `threads`.
template <typename... KArgs, typename... Args>
void launch_pdl_threads(void (*kern)(KArgs...), int grid, int threads, size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, args...);
}

// Launch with programmatic stream serialization (the kernel calls pdl_wait()
// before touching anything an earlier kernel produced).
template <typename... KArgs, typename... Args>
void launch_pdl(void (*kern)(KArgs...), int grid, size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(STEP_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, args...);
}

}  // namespace
}  // namespace krylov
