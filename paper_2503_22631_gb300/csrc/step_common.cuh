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
// E = ceil(log2 B) + 1, so |x| <= 2^(WB-1), and split into NW integer words
// x = q_0 + 2^-WB q_1 + 2^-2WB q_2 + ... (each |q_w| <= 2^(WB-1)), rounding
// with the 1.5 * 2^23 addition trick on the FP32 pipes.  Word w of bin b
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
