// step32_kernels.cu -- the Arnoldi-step kernels of the float32 and bfloat16
// bases with their row streams staged in shared memory by bulk asynchronous
// copies (the layout of the float-float pair in step_kernels.cu, with float32
// arithmetic):
//
//   s32_mat_tma_kernel    w_j = rho_j (p_{j-1} - sum_q h_q w_q) rounded to the
//                         storage type and stored in slot j; its sketch
//                         S w_j (exact fixed-point words of the STORED value)
//                         and ||w_j||^2
//   s32_spmv_tma_kernel   p_j = A w_j (float32 products summed in storage
//                         order, CSR tiles staged), ||p_j||^2 and the window
//                         dots <w_q, p_j>
//   s32_spmv_sell_kernel  the same product on the sliced layout (tiles padded
//                         to their longest row, slot-major), when the
//                         operator has one
//
// Per-thread sums are float32, CTA partials float-float pairs; as in the
// float-float pair, the materialize kernel's CTAs form the coefficients from
// the product kernel's partials (mat_coefficients) and the sketch of a column
// is one exact int64 sum per bin word.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "internal.h"
#include "kernels.cuh"
#include "step_common.cuh"

namespace krylov {
namespace {

constexpr int R32 = STEP_THREADS;         // rows per staged tile
constexpr int MT32_STAGES = 3;            // tiles in flight in the materialize kernel
constexpr int SP32_STAGES = 2;            // CSR tiles in flight in the product kernel
constexpr int RP32 = R32 + 4;             // staged row_ptr entries (16-byte multiple)
constexpr int FAST32 = 8;                 // rows up to this length issue all gathers together
constexpr uint64_t WAIT32_NS = 1000000000ull;  // 1 s bound on one staged-tile wait

template <typename VT> __device__ __forceinline__ float to_f(VT v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// Stage of the materialize kernel: the previous product (float, or the stored
// start vector when there is nothing to materialize), KW window columns, the
// packed sketch table (8 row bytes and a sign byte per column).
template <typename VT>
__host__ __device__ constexpr size_t mt32_stage_bytes(int kw) {
  return (size_t)R32 * (4 + kw * sizeof(VT) + 8 + 1);
}

template <typename VT, bool MAT, int KW, int C, int Z>
__global__ void __launch_bounds__(STEP_THREADS, 3) s32_mat_tma_kernel(const StepLaunch L, const CycleDev cd) {
  constexpr int NW = 2;  // fixed-point words per contribution (float32 significands)
  static_assert(C == 16 || C == 32, "lane copies of the bins");
  constexpr size_t SB = mt32_stage_bytes<VT>(KW);
  constexpr size_t OFF_W = (size_t)R32 * 4;
  constexpr size_t OFF_R = OFF_W + (size_t)R32 * KW * sizeof(VT);
  constexpr size_t OFF_N = OFF_R + (size_t)R32 * 8;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[MT32_STAGES];
  __shared__ float red[64];
  __shared__ MatCoef s_c;
  const int lane = threadIdx.x & 31;
  int* bins = reinterpret_cast<int*>(smem);  // [s][C][NW]
  unsigned char* stages = smem + align16((size_t)NW * L.s * C * sizeof(int));
  const int j = L.j;
  const int lo = MAT ? max(0, j - L.k) : j;
  const int nl = j - lo;
  const int r0 = blockIdx.x * L.rows_per_cta;
  const int r1 = min(L.n, r0 + L.rows_per_cta);
  const int ntiles = (r1 > r0) ? (r1 - r0 + R32 - 1) / R32 : 0;
  const VT* W = static_cast<const VT*>(L.W);
  VT* Wj = static_cast<VT*>(L.W) + (int64_t)j * L.ldw;
  const VT* Wq[KW];
#pragma unroll
  for (int q = 0; q < KW; ++q) Wq[q] = W + (int64_t)(lo + (q < nl ? q : 0)) * L.ldw;
  // the first part of a tile's copies (window, table) does not depend on the
  // kernel just before and is issued before the dependent-launch wait; the
  // product's copy arrives with the last byte count
  auto rows_of = [&](int t) { return (uint32_t)((min(R32, r1 - (r0 + t * R32)) + 15) & ~15); };
  auto issue_static = [&](int t) {
    const int st = t % MT32_STAGES;
    const int ts = r0 + t * R32;
    const uint32_t rc = rows_of(t);
    unsigned char* base = stages + st * SB;
    mbar_expect_tx(&bars[st], rc * (uint32_t)sizeof(VT) * (MAT ? (uint32_t)nl : 0u) + rc * 9u);
    if (MAT) {
#pragma unroll
      for (int q = 0; q < KW; ++q)
        if (q < nl)
          bulk_g2s(base + OFF_W + (size_t)q * R32 * sizeof(VT), Wq[q] + ts, rc * (uint32_t)sizeof(VT), &bars[st]);
    }
    bulk_g2s_stream(base + OFF_R, L.sk_tab.rows8 + ts, rc * 8u, &bars[st]);
    bulk_g2s_stream(base + OFF_N, L.sk_tab.neg8 + ts, rc, &bars[st]);
  };
  auto issue_p = [&](int t) {
    const int st = t % MT32_STAGES;
    const uint32_t rc = rows_of(t);
    const int ts = r0 + t * R32;
    if (MAT) {
      mbar_arrive_expect_tx(&bars[st], rc * 4u);
      bulk_g2s(stages + st * SB, static_cast<const float*>(L.p_prev) + ts, rc * 4u, &bars[st]);
    } else {
      mbar_arrive_expect_tx(&bars[st], rc * (uint32_t)sizeof(VT));
      bulk_g2s(stages + st * SB, Wj + ts, rc * (uint32_t)sizeof(VT), &bars[st]);
    }
  };
  if (threadIdx.x == 0) {
    for (int q = 0; q < MT32_STAGES; ++q) mbar_init(&bars[q], 1);
    fence_mbar_init();
  }
  {
    const int nb = NW * L.s * C;
    int4* b4 = reinterpret_cast<int4*>(bins);
    for (int e = threadIdx.x; e < nb / 4; e += blockDim.x) b4[e] = make_int4(0, 0, 0, 0);
    for (int e = (nb / 4) * 4 + threadIdx.x; e < nb; e += blockDim.x) bins[e] = 0;
  }
  const int npre = min(ntiles, MT32_STAGES);
  if (threadIdx.x == 0)
    for (int t = 0; t < npre; ++t) issue_static(t);
  pdl_wait();
  if (!MAT && cd.flags[0] < j) {  // the cycle ended before column j (breakdown)
    if (threadIdx.x == 0)
      for (int t = 0; t < npre; ++t) {
        mbar_arrive(&bars[t]);
        (void)mbar_wait_bounded(&bars[t], 0u, WAIT32_NS);
      }
    return;
  }
  // p_{j-1} is read even if the cycle has ended (mat_coefficients tells)
  if (threadIdx.x == 0)
    for (int t = 0; t < npre; ++t) issue_p(t);
  if (MAT) {  // the coefficients, from the partials of the kernels before (every CTA)
    if (!mat_coefficients<KW>(L, cd, s_c)) {  // the cycle ended before column j
      if (threadIdx.x == 0)  // let the issued copies land before leaving
        for (int t = 0; t < npre; ++t) (void)mbar_wait_bounded(&bars[t], 0u, WAIT32_NS);
      return;
    }
  } else if (threadIdx.x == 0) {  // the start vector, stored as it is
    s_c.fx = fx_scale(L, cd, 0);
    for (int q = 0; q < MAX_WINDOW; ++q) s_c.h[q] = ff{0.f, 0.f};
    s_c.rho = ff{1.f, 0.f};
  }
  __syncthreads();
  if (blockIdx.x == gridDim.x - 1 && j < L.m) {  // the next column's exact sketch starts from zero
    unsigned long long* nx = fx_acc_of(L, j + 1);
    for (int e = threadIdx.x; e < 3 * L.s; e += blockDim.x) nx[e] = 0ull;
  }
  const FxScale fxs = s_c.fx;
  int* const mybins = bins + (lane & (C - 1)) * NW;
  const int zeta = (Z > 0) ? Z : L.zeta;
  float h[KW];  // -h_q in float32
#pragma unroll
  for (int q = 0; q < KW; ++q) h[q] = s_c.h[q].hi;
  const float rho = s_c.rho.hi;
  float acc_sig = 0.f;
  bool timed_out = false;
  int last_issued = npre - 1;
  for (int t = 0; t < ntiles; ++t) {
    const int st = t % MT32_STAGES;
    const uint32_t par = (uint32_t)(t / MT32_STAGES) & 1u;
    if (!timed_out && !mbar_wait_bounded(&bars[st], par, WAIT32_NS)) timed_out = true;
    const unsigned char* base = stages + st * SB;
    const int k = (int)threadIdx.x;
    const int i = r0 + t * R32 + k;
    if (i < r1 && !timed_out) {
      float wj;
      if (MAT) {
        float a = reinterpret_cast<const float*>(base)[k];
#pragma unroll
        for (int q = 0; q < KW; ++q)
          if (q < nl) a = __fmaf_rn(h[q], to_f(reinterpret_cast<const VT*>(base + OFF_W + (size_t)q * R32 * sizeof(VT))[k]), a);
        const float v = a * rho;
        Store<VT>::put(Wj + i, v);
        wj = stored<VT, float>(v);  // the sketch and the norm see the stored value
      } else {
        wj = to_f(reinterpret_cast<const VT*>(base)[k]);
      }
      acc_sig = __fmaf_rn(wj, wj, acc_sig);
      const uint2 rr = reinterpret_cast<const uint2*>(base + OFF_R)[k];
      const uint32_t ng = (base + OFF_N)[k];
      const FxWords<NW> xw = fx_split<NW>(wj, 0.f, fxs);
      const int q0 = xw.q[0], q1 = xw.q[1];
      const int n0 = -q0, n1 = -q1;
#pragma unroll
      for (int e = 0; e < 8; ++e)
        if (Z == 8 || e < zeta) {
          const int row = (int)__byte_perm(e < 4 ? rr.x : rr.y, 0u, 0x4440u | (uint32_t)(e & 3));
          int* b = mybins + row * (C * NW);
          const bool neg = (ng >> e) & 1u;
          atomicAdd(b, neg ? n0 : q0);
          atomicAdd(b + 1, neg ? n1 : q1);
        }
    }
    __syncthreads();  // every thread is done with stage st
    if (threadIdx.x == 0 && t + MT32_STAGES < ntiles && !timed_out) {
      fence_proxy_async();
      issue_static(t + MT32_STAGES);
      issue_p(t + MT32_STAGES);
      last_issued = t + MT32_STAGES;
    }
  }
  pdl_trigger();
  if (timed_out) atomicOr(&cd.flags[2], ERR_TIMEOUT);
  if (threadIdx.x == 0 && timed_out) {
    for (int t = max(0, last_issued - MT32_STAGES + 1); t <= last_issued; ++t)
      (void)mbar_wait_bounded(&bars[t % MT32_STAGES], (uint32_t)(t / MT32_STAGES) & 1u, WAIT32_NS);
  }
  const ff v = block_sum_ff_pair(ff{acc_sig, 0.f}, red, red + 32);
  if (threadIdx.x == 0) st_part_ff(part_w_of(L, j) + blockIdx.x, v);
  __syncthreads();
  unsigned long long* acc = fx_acc_of(L, j);
  fx_accumulate<NW>([&](int b, int c, int w) { return (long long)bins[(b * C + c) * NW + w]; }, L.s, C, acc);
  if (blockIdx.x == 0) {
    if (threadIdx.x == 0) reinterpret_cast<long long*>(acc)[3 * L.s] = fxs.E;
    if (MAT) mat_coefficients_store(L, cd, s_c);
  }
  if (j == L.m) ff_mat_finish(L, cd, MAT ? 1 : 0);  // else the next materialize kernel sums the partials
}

// CTA partials of a float32 product kernel: ||p_j||^2 and the window dots as
// float-float pairs (columns 1, 2, ... of the partials), which the next
// materialize kernel's CTAs sum.
template <int KW>
__device__ __forceinline__ void s32_spmv_partials(float acc_pi, const float (&acc_dot)[KW], int nd, double* part_cta) {
  __shared__ float2 sh[MAX_WARPS][1 + KW];
  ff v[1 + KW];
  v[0] = ff{acc_pi, 0.f};
#pragma unroll
  for (int q = 0; q < KW; ++q) v[1 + q] = ff{acc_dot[q], 0.f};
  block_partials_ff<1 + KW>(v, 1 + nd, part_cta, 1, sh);
}

// Stage of the product kernel: row_ptr slice, column entries (4-byte indices,
// or 2-byte offsets col - row when DI), float values.  cap: a multiple of 8.
template <bool DI>
__host__ __device__ constexpr size_t sp32_stage_bytes(int cap) {
  return (size_t)RP32 * 4 + (size_t)cap * (DI ? 2 : 4) + (size_t)cap * 4;
}

template <typename VT, int KW, bool DI>
__global__ void __launch_bounds__(STEP_THREADS, 3) s32_spmv_tma_kernel(const StepLaunch L, const CycleDev cd) {
  using CT = typename std::conditional<DI, int16_t, int>::type;
  constexpr int EA = DI ? 8 : 4;  // staged nonzero ranges start on 16-byte boundaries
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[SP32_STAGES];
  const int j = L.j;
  const int cap = L.tma_cap;
  const size_t sb = sp32_stage_bytes<DI>(cap);
  auto rp_st = [&](int st) { return reinterpret_cast<int*>(smem + (size_t)st * sb); };
  auto col_st = [&](int st) { return reinterpret_cast<CT*>(rp_st(st) + RP32); };
  auto val_st = [&](int st) { return reinterpret_cast<float*>(col_st(st) + cap); };
  const CT* colsrc = DI ? reinterpret_cast<const CT*>(L.dcol) : reinterpret_cast<const CT*>(L.col);
  const VT* W = static_cast<const VT*>(L.W);
  const VT* Wj = W + (int64_t)j * L.ldw;
  const float* val = static_cast<const float*>(L.val);
  const int dlo = max(0, j - L.k + 1);
  const int nd = j - dlo + 1;
  const VT* Wd[KW];
#pragma unroll
  for (int q = 0; q < KW; ++q) Wd[q] = W + (int64_t)(dlo + (q < nd ? q : 0)) * L.ldw;
  const int r0 = blockIdx.x * L.rows_spmv;
  const int r1 = min(L.n, r0 + L.rows_spmv);
  const int ntiles = (r1 > r0) ? (r1 - r0 + R32 - 1) / R32 : 0;
  if (threadIdx.x == 0) {
    for (int q = 0; q < SP32_STAGES; ++q) mbar_init(&bars[q], 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto issue = [&](int t, int e0, int e1) {  // thread 0: stage tile t given its nonzero range
    const int st = t % SP32_STAGES;
    const int ts = r0 + t * R32;
    const int ea = e0 & ~(EA - 1), eb = (e1 + EA - 1) & ~(EA - 1);
    const uint32_t brp = RP32 * 4u, bcol = (uint32_t)(eb - ea) * (uint32_t)sizeof(CT),
                   bval = (uint32_t)(eb - ea) * 4u;
    mbar_arrive_expect_tx(&bars[st], brp + bcol + bval);
    bulk_g2s_stream(rp_st(st), L.row_ptr + ts, brp, &bars[st]);
    if (eb > ea) {
      bulk_g2s_stream(col_st(st), colsrc + ea, bcol, &bars[st]);
      bulk_g2s_stream(val_st(st), val + ea, bval, &bars[st]);
    }
  };
  auto tile_end = [&](int t) { return min(r0 + (t + 1) * R32, r1); };
  if (threadIdx.x == 0)
    for (int t = 0; t < min(ntiles, SP32_STAGES); ++t)
      issue(t, __ldg(L.row_ptr + r0 + t * R32), __ldg(L.row_ptr + tile_end(t)));
  pdl_wait();  // w_j comes from the kernel just before
  if (cd.flags[1] != 0) {  // breakdown in this cycle: no further products
    if (threadIdx.x == 0)
      for (int t = 0; t < min(ntiles, SP32_STAGES); ++t) (void)mbar_wait_bounded(&bars[t], 0u, WAIT32_NS);
    return;
  }
  float acc_pi = 0.f, acc_dot[KW];
#pragma unroll
  for (int q = 0; q < KW; ++q) acc_dot[q] = 0.f;
  bool timed_out = false;
  int last_issued = min(ntiles, SP32_STAGES) - 1;
  for (int t = 0; t < ntiles; ++t) {
    const int st = t % SP32_STAGES;
    const uint32_t par = (uint32_t)(t / SP32_STAGES) & 1u;
    const int ts = r0 + t * R32;
    const int i = ts + (int)threadIdx.x;
    const bool valid = i < tile_end(t);
    int nb0 = 0, nb1 = 0;
    if (threadIdx.x == 0 && t + SP32_STAGES < ntiles) {
      nb0 = __ldg(L.row_ptr + ts + SP32_STAGES * R32);
      nb1 = __ldg(L.row_ptr + tile_end(t + SP32_STAGES));
    }
    float wq[KW];
    if (valid) {
#pragma unroll
      for (int q = 0; q < KW; ++q)
        if (q < nd) wq[q] = to_f(Wd[q][i]);
    }
    if (!timed_out && !mbar_wait_bounded(&bars[st], par, WAIT32_NS)) timed_out = true;
    if (valid && !timed_out) {
      const int* rps = rp_st(st);
      const CT* cs = col_st(st);
      const float* vs = val_st(st);
      const int ea = rps[0] & ~(EA - 1);
      const int rb = rps[threadIdx.x] - ea, re = rps[threadIdx.x + 1] - ea;
      const int cbase = DI ? i : 0;
      float acc = 0.f;
      if (re - rb <= FAST32) {
        float wv[FAST32];
#pragma unroll
        for (int q = 0; q < FAST32; ++q)
          if (rb + q < re) wv[q] = to_f(Wj[cbase + (int)cs[rb + q]]);
#pragma unroll
        for (int q = 0; q < FAST32; ++q)
          if (rb + q < re) acc = __fmaf_rn(vs[rb + q], wv[q], acc);
      } else {
#pragma unroll 4
        for (int e = rb; e < re; ++e) acc = __fmaf_rn(vs[e], to_f(Wj[cbase + (int)cs[e]]), acc);
      }
      static_cast<float*>(L.p_out)[i] = acc;
      acc_pi = __fmaf_rn(acc, acc, acc_pi);
#pragma unroll
      for (int q = 0; q < KW; ++q)
        if (q < nd) acc_dot[q] = __fmaf_rn(wq[q], acc, acc_dot[q]);
    }
    __syncthreads();  // every thread is done with stage st
    if (threadIdx.x == 0 && t + SP32_STAGES < ntiles && !timed_out) {
      fence_proxy_async();
      issue(t + SP32_STAGES, nb0, nb1);
      last_issued = t + SP32_STAGES;
    }
  }
  pdl_trigger();
  if (timed_out) atomicOr(&cd.flags[2], ERR_TIMEOUT);
  if (threadIdx.x == 0 && timed_out) {
    for (int t = max(0, last_issued - SP32_STAGES + 1); t <= last_issued; ++t)
      (void)mbar_wait_bounded(&bars[t % SP32_STAGES], (uint32_t)(t / SP32_STAGES) & 1u, WAIT32_NS);
  }
  s32_spmv_partials<KW>(acc_pi, acc_dot, nd, L.part + (size_t)blockIdx.x * NQ);
}

// Product kernel on the sliced layout (see ff_spmv_sell_kernel): tiles padded
// to their longest row L, stored slot-major; the entry loop is unrolled for
// the tile's L.
constexpr size_t SELL32_STAGE = (size_t)SELL_MAXL * R32 * (2 + 4);

template <int NL, typename VT>
__device__ __forceinline__ float sell32_row(const int16_t* cs, const float* vs, const VT* Wj, int i, int k) {
  float wv[NL], av[NL];
#pragma unroll
  for (int q = 0; q < NL; ++q) {
    av[q] = vs[q * R32 + k];
    wv[q] = to_f(Wj[i + (int)cs[q * R32 + k]]);
  }
  float acc = 0.f;
#pragma unroll
  for (int q = 0; q < NL; ++q) acc = __fmaf_rn(av[q], wv[q], acc);
  return acc;
}

template <typename VT, int KW>
__global__ void __launch_bounds__(STEP_THREADS, 3) s32_spmv_sell_kernel(const StepLaunch L, const CycleDev cd) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[SP32_STAGES];
  auto col_st = [&](int st) { return reinterpret_cast<const int16_t*>(smem + (size_t)st * SELL32_STAGE); };
  auto val_st = [&](int st) {
    return reinterpret_cast<const float*>(smem + (size_t)st * SELL32_STAGE + (size_t)SELL_MAXL * R32 * 2);
  };
  const int j = L.j;
  const VT* W = static_cast<const VT*>(L.W);
  const VT* Wj = W + (int64_t)j * L.ldw;
  const float* sval = static_cast<const float*>(L.sell_val);
  const int dlo = max(0, j - L.k + 1);
  const int nd = j - dlo + 1;
  const VT* Wd[KW];
#pragma unroll
  for (int q = 0; q < KW; ++q) Wd[q] = W + (int64_t)(dlo + (q < nd ? q : 0)) * L.ldw;
  const int r0 = blockIdx.x * L.rows_spmv;
  const int r1 = min(L.n, r0 + L.rows_spmv);
  const int ntiles = (r1 > r0) ? (r1 - r0 + R32 - 1) / R32 : 0;
  const int g0 = r0 / R32;
  if (threadIdx.x == 0) {
    for (int q = 0; q < SP32_STAGES; ++q) mbar_init(&bars[q], 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto issue = [&](int t) {
    const int st = t % SP32_STAGES;
    const int e0 = __ldg(L.sell_off + g0 + t), e1 = __ldg(L.sell_off + g0 + t + 1);
    const uint32_t bc = (uint32_t)(e1 - e0) * 2u, bv = (uint32_t)(e1 - e0) * 4u;
    mbar_arrive_expect_tx(&bars[st], bc + bv);
    if (e1 > e0) {
      unsigned char* base = smem + (size_t)st * SELL32_STAGE;
      bulk_g2s_stream(base, L.sell_col + e0, bc, &bars[st]);
      bulk_g2s_stream(base + (size_t)SELL_MAXL * R32 * 2, sval + e0, bv, &bars[st]);
    }
  };
  if (threadIdx.x == 0)
    for (int t = 0; t < min(ntiles, SP32_STAGES); ++t) issue(t);
  pdl_wait();
  if (cd.flags[1] != 0) {
    if (threadIdx.x == 0)
      for (int t = 0; t < min(ntiles, SP32_STAGES); ++t) (void)mbar_wait_bounded(&bars[t], 0u, WAIT32_NS);
    return;
  }
  float acc_pi = 0.f, acc_dot[KW];
#pragma unroll
  for (int q = 0; q < KW; ++q) acc_dot[q] = 0.f;
  bool timed_out = false;
  int last_issued = min(ntiles, SP32_STAGES) - 1;
  for (int t = 0; t < ntiles; ++t) {
    const int st = t % SP32_STAGES;
    const uint32_t par = (uint32_t)(t / SP32_STAGES) & 1u;
    const int i = r0 + t * R32 + (int)threadIdx.x;
    const bool valid = i < r1;
    const int nl = (__ldg(L.sell_off + g0 + t + 1) - __ldg(L.sell_off + g0 + t)) / R32;
    float wq[KW];
    if (valid) {
#pragma unroll
      for (int q = 0; q < KW; ++q)
        if (q < nd) wq[q] = to_f(Wd[q][i]);
    }
    if (!timed_out && !mbar_wait_bounded(&bars[st], par, WAIT32_NS)) timed_out = true;
    if (valid && !timed_out) {
      const int16_t* cs = col_st(st);
      const float* vs = val_st(st);
      const int k = (int)threadIdx.x;
      float p;
      switch (nl) {  // the same for every thread of the CTA
        case 1: p = sell32_row<1>(cs, vs, Wj, i, k); break;
        case 2: p = sell32_row<2>(cs, vs, Wj, i, k); break;
        case 3: p = sell32_row<3>(cs, vs, Wj, i, k); break;
        case 4: p = sell32_row<4>(cs, vs, Wj, i, k); break;
        case 5: p = sell32_row<5>(cs, vs, Wj, i, k); break;
        case 6: p = sell32_row<6>(cs, vs, Wj, i, k); break;
        case 7: p = sell32_row<7>(cs, vs, Wj, i, k); break;
        case 8: p = sell32_row<8>(cs, vs, Wj, i, k); break;
        default: {
          float a = 0.f;
          for (int q = 0; q < nl; ++q) a = __fmaf_rn(vs[q * R32 + k], to_f(Wj[i + (int)cs[q * R32 + k]]), a);
          p = a;
        }
      }
      static_cast<float*>(L.p_out)[i] = p;
      acc_pi = __fmaf_rn(p, p, acc_pi);
#pragma unroll
      for (int q = 0; q < KW; ++q)
        if (q < nd) acc_dot[q] = __fmaf_rn(wq[q], p, acc_dot[q]);
    }
    __syncthreads();
    if (threadIdx.x == 0 && t + SP32_STAGES < ntiles && !timed_out) {
      fence_proxy_async();
      issue(t + SP32_STAGES);
      last_issued = t + SP32_STAGES;
    }
  }
  pdl_trigger();
  if (timed_out) atomicOr(&cd.flags[2], ERR_TIMEOUT);
  if (threadIdx.x == 0 && timed_out) {
    for (int t = max(0, last_issued - SP32_STAGES + 1); t <= last_issued; ++t)
      (void)mbar_wait_bounded(&bars[t % SP32_STAGES], (uint32_t)(t / SP32_STAGES) & 1u, WAIT32_NS);
  }
  s32_spmv_partials<KW>(acc_pi, acc_dot, nd, L.part + (size_t)blockIdx.x * NQ);
}

template <typename K> int occ32(K kern, size_t smem) {
  raise_smem_limit((const void*)kern, smem);
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, STEP_THREADS, smem);
  return b < 1 ? 1 : b;
}

template <typename VT, bool MAT, int KW>
void launch_mat32(const StepLaunch& L, const CycleDev& cd, cudaStream_t st) {
  const size_t smem = s32_mat_smem(L.s, L.sk_copies, KW, sizeof(VT));
  auto k = (L.sk_copies == 32)
               ? ((L.zeta == 8) ? s32_mat_tma_kernel<VT, MAT, KW, 32, 8> : s32_mat_tma_kernel<VT, MAT, KW, 32, 0>)
               : ((L.zeta == 8) ? s32_mat_tma_kernel<VT, MAT, KW, 16, 8> : s32_mat_tma_kernel<VT, MAT, KW, 16, 0>);
  raise_smem_limit((const void*)k, smem);
  launch_pdl(k, L.grid, smem, st, L, cd);
}

template <typename VT, int KW>
void launch_spmv32(const StepLaunch& L, const CycleDev& cd, cudaStream_t st) {
  if (L.sell_col != nullptr) {
    auto k = s32_spmv_sell_kernel<VT, KW>;
    const size_t smem = SP32_STAGES * SELL32_STAGE;
    raise_smem_limit((const void*)k, smem);
    launch_pdl(k, L.grid_spmv, smem, st, L, cd);
    return;
  }
  if (L.dcol != nullptr) {
    auto k = s32_spmv_tma_kernel<VT, KW, true>;
    const size_t smem = SP32_STAGES * sp32_stage_bytes<true>(L.tma_cap);
    raise_smem_limit((const void*)k, smem);
    launch_pdl(k, L.grid_spmv, smem, st, L, cd);
  } else {
    auto k = s32_spmv_tma_kernel<VT, KW, false>;
    const size_t smem = SP32_STAGES * sp32_stage_bytes<false>(L.tma_cap);
    raise_smem_limit((const void*)k, smem);
    launch_pdl(k, L.grid_spmv, smem, st, L, cd);
  }
}

template <typename VT>
void launch_step32_t(const StepLaunch& L, const CycleDev& cd, cudaStream_t st) {
  const bool w2 = L.k <= 2;
  if (L.mat) {
    if (w2) launch_mat32<VT, true, 2>(L, cd, st);
    else launch_mat32<VT, true, MAX_WINDOW>(L, cd, st);
  } else {
    if (w2) launch_mat32<VT, false, 2>(L, cd, st);
    else launch_mat32<VT, false, MAX_WINDOW>(L, cd, st);
  }
  if (L.spmv) {
    if (w2) launch_spmv32<VT, 2>(L, cd, st);
    else launch_spmv32<VT, MAX_WINDOW>(L, cd, st);
  }
}

}  // namespace

size_t s32_mat_smem(int s, int copies, int kw, int vt_bytes) {
  const size_t stage = (size_t)R32 * (4 + (size_t)kw * vt_bytes + 9);
  return align16((size_t)2 * s * copies * sizeof(int)) + MT32_STAGES * stage;
}

int s32_ctas_per_sm(int basis, int s, int copies) {
  const size_t smem = s32_mat_smem(s, copies, 2, basis == 1 ? 4 : 2);
  if (basis == 1)
    return copies == 32 ? occ32(s32_mat_tma_kernel<float, true, 2, 32, 8>, smem)
                        : occ32(s32_mat_tma_kernel<float, true, 2, 16, 8>, smem);
  return copies == 32 ? occ32(s32_mat_tma_kernel<__nv_bfloat16, true, 2, 32, 8>, smem)
                      : occ32(s32_mat_tma_kernel<__nv_bfloat16, true, 2, 16, 8>, smem);
}

int s32_sell_ctas_per_sm() { return occ32(s32_spmv_sell_kernel<float, 2>, SP32_STAGES * SELL32_STAGE); }

int s32_spmv_ctas_per_sm(int tma_cap, int di) {
  return di ? occ32(s32_spmv_tma_kernel<float, 2, true>, SP32_STAGES * sp32_stage_bytes<true>(tma_cap))
            : occ32(s32_spmv_tma_kernel<float, 2, false>, SP32_STAGES * sp32_stage_bytes<false>(tma_cap));
}

void launch_step32(int basis, const StepLaunch& L, const CycleDev& cd, cudaStream_t st) {
  if (basis == 1) launch_step32_t<float>(L, cd, st);
  else launch_step32_t<__nv_bfloat16>(L, cd, st);
}

}  // namespace krylov
