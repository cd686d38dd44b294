// step_kernels.cu -- the Arnoldi-step kernels of one restart cycle.
//
// A step handles basis column j (Algorithm 1's loop body, with the truncated
// orthogonalization of Sec. 5 "incomplete" and the sketch of Sec. 2.1):
//
//   materialize   w_j = rho_j (p_{j-1} - sum_{q in win(j-1)} h_q w_q), the
//                 orthogonalization of the previous product, rounded to the
//                 basis storage type and stored in slot j
//   sketch        u_j += S e_i w_j[i] for the zeta entries of column i of S,
//                 accumulated exactly as fixed-point integer words (a scale
//                 from a bound on |w_j[i]|) with shared-memory integer atomics
//                 into lane-private copies of the bins: deterministic in any
//                 arrival order
//   product       p_j = A w_j, each row's products summed in storage order
//                 (CSR tiles staged in shared memory by bulk asynchronous
//                 copies, or a warp-cooperative CSR stream)
//   dots          <w_q, p_j> for the window of the next column, ||p_j||^2,
//                 ||w_j||^2
//
// step_kernel (float64 / float32 / bfloat16 bases) fuses all four in one
// pass: w_j at a neighbour column c is recomputed from p_{j-1}[c] and the
// window vectors at c with the same rounded arithmetic, so w_j is written
// once and never re-read.  The float-float basis splits a step into
// ff_mat_kernel (materialize + sketch) and ff_spmv_kernel (product + dots):
// recomputing a float-float orthogonalization at every neighbour would make
// the step arithmetic-bound.
//
// Basis vectors are stored unnormalized: rho_j only keeps ||w_j|| near 1
// (from ||p||^2 - sum h_q^2 ||w_q||^2); the exact norm is reduced here and
// h_q = <w_q, p_j> / ||w_q||^2 are projection coefficients, so the
// Arnoldi-like relation A w_{j-1} = sum h_q w_q + w_j / rho_j (Eq. 5) holds
// for whatever rho_j was used.  The whitening absorbs the column scaling.
//
// Reductions are deterministic: per-CTA partials in fixed slots, summed in a
// fixed order.  In the fused kernel the last CTA to arrive (atomic ticket)
// sums them and writes the next column's coefficients, and the sketch
// partials stay per CTA until sketch_reduce_kernel sums them once per cycle.
// The staged float-float pair has no reducer between its kernels: every CTA
// of the next materialize kernel sums the partials and forms the
// coefficients itself (only the last column of a cycle, which no
// materialize kernel follows, and ||p_j||^2 in a randomized Gram-Schmidt
// cycle keep a last-CTA sum), and the sketch of a column is an exact int64
// sum over the CTAs (sketch_finish_kernel forms U once per cycle).
#include <algorithm>
#include <cmath>

#include <type_traits>

#include "internal.h"
#include "kernels.cuh"
#include "step_common.cuh"

namespace krylov {
namespace {

template <typename VT> struct Types {
  using A = float;   // arithmetic
  using P = float;   // raw product storage
  using Sk = float;  // sketch bins / partials
};
template <> struct Types<double> {
  using A = double;
  using P = double;
  using Sk = double;
};

constexpr int STAGE = 512;          // staged nonzeros per warp in the CSR stream

// Products of the CSR stream are formed in batches of U nonzeros per lane:
// all column indices and values of a batch are loaded first, then all the
// gathers, so each lane keeps many independent loads in flight.
constexpr int U_FUSED = 4;

// ---------------------------------------------------------------------------
template <typename VT, typename AT, bool MAT, bool SPMV, int SKM>
__global__ void __launch_bounds__(STEP_THREADS, 3) step_kernel(const StepLaunch L, const CycleDev cd) {
  using A = typename Types<VT>::A;
  using P = typename Types<VT>::P;
  using Sk = typename Types<VT>::Sk;
  constexpr int NW = (sizeof(A) == 8) ? 3 : 2;  // fixed-point words per contribution
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int C = L.sk_copies;
  int* bins = reinterpret_cast<int*>(smem);  // [NW][s][C]
  A* stage = reinterpret_cast<A*>(smem + align16((size_t)NW * L.s * C * sizeof(int)));
  __shared__ A red[32];
  __shared__ double tot[NQ];
  __shared__ int s_last;

  __shared__ FxScale s_fx;
  __shared__ A s_h[MAX_WINDOW + 1];

  const int j = L.j;
  if (cd.flags[0] < j) return;  // an earlier column broke down
  const int lo = MAT ? max(0, j - L.k) : j;
  const int nl = j - lo;
  for (int e = threadIdx.x; e < NW * L.s * C; e += blockDim.x) bins[e] = 0;
  if (threadIdx.x == 0) {  // per-CTA prologue (float64 work done once)
    s_fx = fx_scale(L, cd, MAT ? 1 : 0);
    const double* c = cd.coef + (size_t)(j > 0 ? j - 1 : 0) * (MAX_WINDOW + 1);
    for (int q = 0; q < MAX_WINDOW; ++q) s_h[q] = (MAT && q < nl) ? A(c[q]) : A(0);
    s_h[MAX_WINDOW] = MAT ? A(c[MAX_WINDOW]) : A(1);
  }
  __syncthreads();
  const FxScale fxs = s_fx;
  const int cp = lane & (C - 1);
  const int sC = L.s * C;

  const VT* W = static_cast<const VT*>(L.W);
  VT* Wj = static_cast<VT*>(L.W) + (int64_t)j * L.ldw;
  const P* pprev = static_cast<const P*>(L.p_prev);
  const AT* val = static_cast<const AT*>(L.val);
  A h[MAX_WINDOW];
  const VT* Wq[MAX_WINDOW];
#pragma unroll
  for (int q = 0; q < MAX_WINDOW; ++q) {
    h[q] = s_h[q];
    Wq[q] = W + (int64_t)(lo + (q < nl ? q : 0)) * L.ldw;
  }
  const A rho = s_h[MAX_WINDOW];
  const int dlo = max(0, j - L.k + 1);
  const int nd = L.rgs ? 0 : j - dlo + 1;  // window dots (none in a randomized Gram-Schmidt cycle)
  const int off = dlo - lo;
  const SketchSpec sp = spec_of(L);
  const uint32_t inv_s = sketch_inv_s(L.s);

  // value of w_j at row c, exactly as its owner thread rounds and stores it
  auto wj_at = [&](int c) -> A {
    if (MAT) {
      A t = A(__ldg(pprev + c));
#pragma unroll
      for (int q = 0; q < MAX_WINDOW; ++q)
        if (q < nl) t = fma_rn(-h[q], A(Store<VT>::load(Wq[q] + c)), t);
      return stored<VT, A>(mul_rn(t, rho));
    }
    return A(Store<VT>::load(Wj + c));
  };
  A acc_sig = A(0), acc_pi = A(0);
  A acc_dot[MAX_WINDOW];
#pragma unroll
  for (int q = 0; q < MAX_WINDOW; ++q) acc_dot[q] = A(0);
  int bad = 0;
  A* mystage = stage + wid * STAGE;

  const int r0 = blockIdx.x * L.rows_per_cta;
  const int r1 = min(L.n, r0 + L.rows_per_cta);
  for (int t0 = r0; t0 < r1; t0 += STEP_THREADS) {
    const int i0 = t0 + wid * 32;
    if (i0 >= r1) continue;  // warp-uniform
    const int i = i0 + lane;
    const bool valid = i < r1;
    const int nval = min(32, r1 - i0);
    // ---- own row: loads first ----
    int rb = 0, re = 0;
    A pv0 = A(0);
    A wl[MAX_WINDOW];
#pragma unroll
    for (int q = 0; q < MAX_WINDOW; ++q) wl[q] = A(0);
    typename SkColOf<SKM>::type col;
    if (valid) {
      if (SPMV) {
        rb = __ldg(L.row_ptr + i);
        re = __ldg(L.row_ptr + i + 1);
      }
      if (MAT) {
        pv0 = A(__ldg(pprev + i));
#pragma unroll
        for (int q = 0; q < MAX_WINDOW; ++q)
          if (q < nl) wl[q] = Store<VT>::load(Wq[q] + i);
      }
      col.load(L, sp, inv_s, i);
    }
    A wj = A(0);
    if (valid) {
      if (MAT) {
        A acc = pv0;
#pragma unroll
        for (int q = 0; q < MAX_WINDOW; ++q)
          if (q < nl) acc = fma_rn(-h[q], wl[q], acc);
        wj = stored<VT, A>(mul_rn(acc, rho));
        Store<VT>::put(Wj + i, wj);
      } else {
        wj = Store<VT>::load(Wj + i);
      }
      acc_sig = fma_rn(wj, wj, acc_sig);
      bad |= (col.got < L.zeta);
    }
    // ---- sketch: exact fixed-point contributions ----
    if (valid) {
      float vh, vl;
      if constexpr (sizeof(A) == 8) {
        vh = __double2float_rn((double)wj);
        vl = __double2float_rn((double)wj - (double)vh);
      } else {
        vh = (float)wj;
        vl = 0.f;
      }
      const FxWords<NW> xw = fx_split<NW>(vh, vl, fxs);
      for (int e = 0; e < col.got; ++e) fx_emit<NW>(bins, sC, col.row(e), cp, xw, col.neg(e), C);
    }
    // ---- product: warp-cooperative CSR stream ----
    if (SPMV) {
      const int ebeg = __shfl_sync(FULL, rb, 0);
      const int eend = __shfl_sync(FULL, re, nval - 1);
      const int nent = eend - ebeg;
      A accp = A(0);
      if (nent <= STAGE) {
        for (int kb = 0; kb < nent; kb += 32 * U_FUSED) {
          int cc[U_FUSED];
          A av[U_FUSED];
#pragma unroll
          for (int u = 0; u < U_FUSED; ++u) {
            const int k = kb + u * 32 + lane;
            cc[u] = 0;
            av[u] = A(0);
            if (k < nent) {
              cc[u] = __ldg(L.col + ebeg + k);
              av[u] = A(__ldg(val + ebeg + k));
            }
          }
#pragma unroll
          for (int u = 0; u < U_FUSED; ++u) {
            const int k = kb + u * 32 + lane;
            if (k < nent) mystage[k] = mul_rn(av[u], wj_at(cc[u]));
          }
        }
        __syncwarp();
        if (valid)
          for (int k = rb - ebeg; k < re - ebeg; ++k) accp += mystage[k];
        __syncwarp();
      } else if (valid) {
        for (int e = rb; e < re; ++e) accp = fma_rn(A(__ldg(val + e)), wj_at(__ldg(L.col + e)), accp);
      }
      if (valid) {
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
  double* out = static_cast<double*>(L.sk_part) + (size_t)blockIdx.x * L.s;
  for (int b = threadIdx.x; b < L.s; b += blockDim.x) out[b] = fx_value<NW>(bins, L.s, C, b, fxs, L.fx_wb);
  if (bad) atomicOr(&cd.flags[2], ERR_SKETCH);

  if (!last_block_flag(cd.counter, &s_last)) return;
  for (int q = (int)(threadIdx.x >> 5); q < NQ; q += (int)(blockDim.x >> 5)) {
    const double acc = warp_sum_partials(L.part, (int)gridDim.x, NQ, q);
    if ((threadIdx.x & 31) == 0) tot[q] = acc;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    int brk = 0;
    if (threadIdx.x == 0) brk = reduce_mat(L, cd, tot[0], MAT ? 1 : 0) ? 1 : 0;
    brk = __shfl_sync(FULL, brk, 0);
    if (SPMV) reduce_spmv(L, cd, tot, brk != 0, tot[0]);  // reduce_mat stored ||w_j||^2 = tot[0]
    if (threadIdx.x == 0) *cd.counter = 0u;
  }
}

// ---------------------------------------------------------------------------
// Float-float basis ("df64"): (hi, lo) float pairs, arithmetic on the FP32
// pipes.  The sums that define the Arnoldi relation (products and
// orthogonalization), the sketch and the dots are float-float accurate.

// Inputs of one row of ff_mat_kernel, loaded before any use so that two rows
// per thread have their loads in flight together.
template <int KW, int SKM> struct FfRow {
  ff pv, wl[KW];
  typename SkColOf<SKM>::type col;
};

template <bool MAT, int SKM, int KW>
__global__ void __launch_bounds__(STEP_THREADS, 4) ff_mat_kernel(const StepLaunch L, const CycleDev cd) {
  constexpr int NW = 3;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int C = L.sk_copies;
  int* bins = reinterpret_cast<int*>(smem);  // [NW][s][C]
  __shared__ float red[64];
  __shared__ MatCoef s_c;
  const int j = L.j;
  if (cd.flags[0] < j) return;
  const int lo = MAT ? max(0, j - L.k) : j;
  const int nl = j - lo;
  {
    const int nb = NW * L.s * C;
    int4* b4 = reinterpret_cast<int4*>(bins);
    for (int e = threadIdx.x; e < nb / 4; e += blockDim.x) b4[e] = make_int4(0, 0, 0, 0);
    for (int e = (nb / 4) * 4 + threadIdx.x; e < nb; e += blockDim.x) bins[e] = 0;
  }
  if (MAT) {  // the coefficients, from the partials of the kernels before (every CTA)
    if (!mat_coefficients<KW>(L, cd, s_c)) return;  // column j - 1 ended the cycle
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
  const int cp = lane & (C - 1);
  const int sC = L.s * C;

  const float2* W = static_cast<const float2*>(L.W);
  float2* Wj = static_cast<float2*>(L.W) + (int64_t)j * L.ldw;
  const float2* pprev = static_cast<const float2*>(L.p_prev);
  ff h[KW];
  const float2* Wq[KW];
#pragma unroll
  for (int q = 0; q < KW; ++q) {
    h[q] = s_c.h[q];
    Wq[q] = W + (int64_t)(lo + (q < nl ? q : 0)) * L.ldw;
  }
  const ff rho = s_c.rho;
  const SketchSpec sp = spec_of(L);
  const uint32_t inv_s = sketch_inv_s(L.s);
  ffacc acc_sig;
  int bad = 0;

  auto load_row = [&](FfRow<KW, SKM>& r, int i) {
    if (MAT) {
      r.pv = ld_ff(pprev + i);
#pragma unroll
      for (int q = 0; q < KW; ++q)
        if (q < nl) r.wl[q] = ld_ff(Wq[q] + i);
    } else {
      r.pv = ld_ff(Wj + i);
    }
    r.col.load(L, sp, inv_s, i);
  };
  auto do_row = [&](const FfRow<KW, SKM>& r, int i) {
    ff wj;
    if (MAT) {
      ff acc = r.pv;
#pragma unroll
      for (int q = 0; q < KW; ++q)
        if (q < nl) acc = ff_add(acc, ff_mul(h[q], r.wl[q]));
      wj = ff_mul(acc, rho);
      st_ff(Wj + i, wj);
    } else {
      wj = r.pv;
    }
    acc_sig.add_prod(wj, wj);
    bad |= (r.col.got < L.zeta);
    const FxWords<NW> xw = fx_split<NW>(wj.hi, wj.lo, fxs);
    if constexpr (SKM == SK_TAB8 || SKM == SK_GEN8) {
#pragma unroll
      for (int e = 0; e < 8; ++e)
        if (e < r.col.got) fx_emit<NW>(bins, sC, r.col.row(e), cp, xw, r.col.neg(e), C);
    } else {
      for (int e = 0; e < r.col.got; ++e) fx_emit<NW>(bins, sC, r.col.row(e), cp, xw, r.col.neg(e), C);
    }
  };

  const int r0 = blockIdx.x * L.rows_per_cta;
  const int r1 = min(L.n, r0 + L.rows_per_cta);
  const int T = blockDim.x;
  for (int i = r0 + (int)threadIdx.x; i < r1; i += 2 * T) {
    const int i2 = i + T;
    FfRow<KW, SKM> a, b;
    load_row(a, i);
    if (i2 < r1) load_row(b, i2);
    do_row(a, i);
    if (i2 < r1) do_row(b, i2);
  }
  const ff v = block_sum_ff_pair(acc_sig.result(), red, red + 32);
  if (threadIdx.x == 0) st_part_ff(part_w_of(L, j) + blockIdx.x, v);
  __syncthreads();
  unsigned long long* acc = fx_acc_of(L, j);
  fx_accumulate([&](int b, int c, int w) { return (long long)bins[(w * L.s + b) * C + c]; }, L.s, C, acc);
  if (bad) atomicOr(&cd.flags[2], ERR_SKETCH);
  if (blockIdx.x == 0) {
    if (threadIdx.x == 0) reinterpret_cast<long long*>(acc)[3 * L.s] = fxs.E;
    if (MAT) mat_coefficients_store(L, cd, s_c);
  }
  if (j == L.m) ff_mat_finish(L, cd, MAT ? 1 : 0);  // else the next materialize kernel sums the partials
}

// Materialize + sketch with the row streams staged in shared memory (packed
// sketch table).  Tiles of MT_ROWS rows: the producer thread copies the
// tile's slices of p_{j-1} (or w_0), the window vectors and the sketch table
// (8 row bytes and a sign byte per column) with bulk asynchronous copies
// completing on an mbarrier, MT_STAGES tiles ahead; each row thread then
// handles MT_RPT rows from shared memory with the arithmetic of
// ff_mat_kernel.  Row slices start at multiples of 256 rows (16-byte aligned:
// a CTA's rows are a multiple of 256) and a partial last tile is copied
// rounded up to 16 rows (the row arrays are padded to the slot stride).
constexpr uint64_t TMA_WAIT_NS = 1000000000ull;  // 1 s bound on one staged-tile wait
// One CTA per SM (two CTAs per SM drifted apart as the product kernel's did:
// the second finished ~3.5 us after the first, its SM half idle meanwhile):
// MT_THREADS row threads (MT_RPT rows per thread in a tile of MT_ROWS rows)
// and one producer warp, which refills a stage once every row warp has
// released it (a per-stage "empty" barrier), so that no CTA-wide barrier per
// tile holds the row warps together.
constexpr int MT_THREADS = 512;
constexpr int MT_RPT = 2;  // rows per thread and tile: two independent float-float chains
constexpr int MT_ROWS = MT_THREADS * MT_RPT;
constexpr int MT_BLOCK = MT_THREADS + 32;  // + the producer warp
constexpr int MT_PRODUCER = MT_THREADS;    // the thread that issues the copies
#ifndef KRYLOV_MT_STAGES
#define KRYLOV_MT_STAGES 3
#endif
constexpr int MT_STAGES = KRYLOV_MT_STAGES;
__host__ __device__ constexpr size_t mt_stage_bytes(int kw) {
  return (size_t)MT_ROWS * 8 * (2 + kw) + MT_ROWS;
}

// Bins of this kernel keep the three words of a (bin, copy) next to each other,
// [s][C][3] ints, so the three atomic adds of a sketch entry share one address
// computation (immediate offsets); lane l works in copy l mod C, and with 32
// copies the words a warp adds at one time sit in 32 different banks (word
// stride 3 is odd).  C (copies) and Z (zeta, 0 = runtime value <= 8) are
// compile-time so that the entry loop carries no parameter loads.

template <bool MAT, int KW, int C, int Z>
__global__ void __launch_bounds__(MT_BLOCK, 1) ff_mat_tma_kernel(const StepLaunch L, const CycleDev cd) {
  constexpr int NW = 3;
  static_assert(C == 16 || C == 32, "lane copies of the bins");
  constexpr size_t SB = mt_stage_bytes(KW);
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[MT_STAGES];   // tile landed (bulk-copy bytes)
  __shared__ __align__(8) uint64_t empty[MT_STAGES];  // every row warp is done with the stage
  __shared__ float red[64];
  __shared__ MatCoef s_c;
  const bool producer = threadIdx.x == MT_PRODUCER;
  const int lane = threadIdx.x & 31;
  int* bins = reinterpret_cast<int*>(smem);  // [s][C][NW]
  unsigned char* stages = smem + align16(bins_bytes(3, L.s, C));
  const int j = L.j;
  const int lo = MAT ? max(0, j - L.k) : j;
  const int nl = j - lo;
  const int r0 = blockIdx.x * L.rows_mat;
  const int r1 = min(L.n, r0 + L.rows_mat);
  const int ntiles = (r1 > r0) ? (r1 - r0 + MT_ROWS - 1) / MT_ROWS : 0;

  const float2* W = static_cast<const float2*>(L.W);
  float2* Wj = static_cast<float2*>(L.W) + (int64_t)j * L.ldw;
  const float2* src0 = MAT ? static_cast<const float2*>(L.p_prev) : Wj;
  const float2* Wq[KW];
#pragma unroll
  for (int q = 0; q < KW; ++q) Wq[q] = W + (int64_t)(lo + (q < nl ? q : 0)) * L.ldw;
  auto st_p = [&](int st) { return reinterpret_cast<const float2*>(stages + st * SB); };
  auto st_w = [&](int st, int q) { return reinterpret_cast<const float2*>(stages + st * SB + (size_t)MT_ROWS * 8 * (1 + q)); };
  auto st_r = [&](int st) { return reinterpret_cast<const uint2*>(stages + st * SB + (size_t)MT_ROWS * 8 * (1 + KW)); };
  auto st_n = [&](int st) { return stages + st * SB + (size_t)MT_ROWS * 8 * (2 + KW); };
  // Tile t's copies come in two parts: the window columns and the sketch
  // table (written two or more kernels back, or never) and the product p_{j-1}
  // (written by the kernel just before).  The first part of the first tiles is
  // issued before the programmatic-launch wait, overlapping the previous
  // kernel's reduction tail; the phase completes only once the second part
  // has arrived as well (its arrive carries the last byte count).
  auto rows_of = [&](int t) { return (uint32_t)((min(MT_ROWS, r1 - (r0 + t * MT_ROWS)) + 15) & ~15); };
  auto issue_static = [&](int t) {  // the producer: expects its bytes, does not arrive
    const int st = t % MT_STAGES;
    const int ts = r0 + t * MT_ROWS;
    const uint32_t rc = rows_of(t);
    unsigned char* base = stages + st * SB;
    mbar_expect_tx(&bars[st], rc * 8u * (MAT ? 1u + (uint32_t)nl : 1u) + rc);
    if (MAT) {
#pragma unroll
      for (int q = 0; q < KW; ++q)
        if (q < nl) bulk_g2s(base + (size_t)MT_ROWS * 8 * (1 + q), Wq[q] + ts, rc * 8u, &bars[st]);
    }
    bulk_g2s_stream(base + (size_t)MT_ROWS * 8 * (1 + KW), L.sk_tab.rows8 + ts, rc * 8u, &bars[st]);
    bulk_g2s_stream(base + (size_t)MT_ROWS * 8 * (2 + KW), L.sk_tab.neg8 + ts, rc, &bars[st]);
  };
  auto issue_p = [&](int t) {  // the producer: arrives with the product's bytes
    const int st = t % MT_STAGES;
    const uint32_t rc = rows_of(t);
    mbar_arrive_expect_tx(&bars[st], rc * 8u);
    bulk_g2s(stages + st * SB, src0 + r0 + t * MT_ROWS, rc * 8u, &bars[st]);
  };
  auto issue = [&](int t) {
    issue_static(t);
    issue_p(t);
  };
  if (producer) {
    for (int q = 0; q < MT_STAGES; ++q) {
      mbar_init(&bars[q], 1);
      mbar_init(&empty[q], MT_THREADS / 32);
    }
    fence_mbar_init();
  }
  {
    const int nb = NW * L.s * C;
    int4* b4 = reinterpret_cast<int4*>(bins);
    for (int e = threadIdx.x; e < nb / 4; e += blockDim.x) b4[e] = make_int4(0, 0, 0, 0);
    for (int e = (nb / 4) * 4 + threadIdx.x; e < nb; e += blockDim.x) bins[e] = 0;
  }
  const int npre = min(ntiles, MT_STAGES);
  if (producer)
    for (int t = 0; t < npre; ++t) issue_static(t);
  // everything above is independent of the kernel just before; p_{j-1} and
  // the coefficients are not
  pdl_wait();
  if (!MAT && cd.flags[0] < j) {  // the cycle ended before column j (breakdown)
    if (producer)  // complete the phases and let the copies land before leaving
      for (int t = 0; t < npre; ++t) {
        mbar_arrive(&bars[t]);
        (void)mbar_wait_bounded(&bars[t], 0u, TMA_WAIT_NS);
      }
    return;
  }
  // p_{j-1} is read even if the cycle has ended (mat_coefficients tells):
  // the copies are harmless and start early
  if (producer)
    for (int t = 0; t < npre; ++t) issue_p(t);
  // the coefficients, from the partials of the kernels before (every CTA,
  // while the first tiles land)
  if (MAT) {
    if (!mat_coefficients<KW>(L, cd, s_c)) {  // the cycle ended before column j
      if (producer)  // let the issued copies land before leaving
        for (int t = 0; t < npre; ++t) (void)mbar_wait_bounded(&bars[t], 0u, TMA_WAIT_NS);
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
  ff h[KW];
#pragma unroll
  for (int q = 0; q < KW; ++q) h[q] = s_c.h[q];
  const ff rho = s_c.rho;
  ffacc acc_sig;
  bool timed_out = false;
  if (producer) {
    // refill stage t % MT_STAGES with tile t once every row warp has released
    // tile t - MT_STAGES (phase t / MT_STAGES - 1 of its empty barrier) and
    // that tile's copies have landed (already so, unless a row warp gave up
    // waiting for them)
    int last_issued = npre - 1;
    for (int t = MT_STAGES; t < ntiles; ++t) {
      const int st = t % MT_STAGES;
      const uint32_t prev = (uint32_t)(t / MT_STAGES - 1) & 1u;
      if (!mbar_wait_bounded(&empty[st], prev, TMA_WAIT_NS) || !mbar_wait_bounded(&bars[st], prev, TMA_WAIT_NS)) {
        timed_out = true;
        break;
      }
      fence_proxy_async();
      issue(t);
      last_issued = t;
    }
    // the copies in flight land before the CTA leaves (at once, unless a row
    // warp gave up waiting for them)
    for (int t = max(0, last_issued - MT_STAGES + 1); t <= last_issued; ++t)
      (void)mbar_wait_bounded(&bars[t % MT_STAGES], (uint32_t)(t / MT_STAGES) & 1u, TMA_WAIT_NS);
  } else if (threadIdx.x < MT_THREADS) {
    for (int t = 0; t < ntiles; ++t) {
      const int st = t % MT_STAGES;
      const uint32_t par = (uint32_t)(t / MT_STAGES) & 1u;
      if (!timed_out && !mbar_wait_bounded(&bars[st], par, TMA_WAIT_NS)) timed_out = true;
      // rows k and k + MT_THREADS of the tile: both rows' materialization and
      // fixed-point words first (independent chains), then their sketch entries
      FxWords<NW> xw[MT_RPT];
      uint2 rr[MT_RPT];
      uint32_t ng[MT_RPT];
      bool ok[MT_RPT];
#pragma unroll
      for (int u = 0; u < MT_RPT; ++u) {
        const int k = (int)threadIdx.x + u * MT_THREADS;
        const int i = r0 + t * MT_ROWS + k;
        ok[u] = i < r1 && !timed_out;
        if (ok[u]) {
          const float2 p2 = st_p(st)[k];
          ff wj{p2.x, p2.y};
          if (MAT) {
            ff acc = wj;
#pragma unroll
            for (int q = 0; q < KW; ++q)
              if (q < nl) {
                const float2 w2 = st_w(st, q)[k];
                acc = ff_add(acc, ff_mul(h[q], ff{w2.x, w2.y}));
              }
            wj = ff_mul(acc, rho);
            st_ff(Wj + i, wj);
          }
          acc_sig.add_prod(wj, wj);
          rr[u] = st_r(st)[k];
          ng[u] = st_n(st)[k];
          xw[u] = fx_split<NW>(wj.hi, wj.lo, fxs);
        }
      }
#pragma unroll
      for (int u = 0; u < MT_RPT; ++u) {
        if (!ok[u]) continue;
        const int q0 = xw[u].q[0], q1 = xw[u].q[1], q2 = xw[u].q[2];
        const int n0 = -q0, n1 = -q1, n2 = -q2;
#pragma unroll
        for (int e = 0; e < 8; ++e)
          if (Z == 8 || e < zeta) {
            const int row = (int)__byte_perm(e < 4 ? rr[u].x : rr[u].y, 0u, 0x4440u | (uint32_t)(e & 3));
            int* b = mybins + row * (C * NW);
            const bool neg = (ng[u] >> e) & 1u;
            atomicAdd(b, neg ? n0 : q0);
            atomicAdd(b + 1, neg ? n1 : q1);
            atomicAdd(b + 2, neg ? n2 : q2);
          }
      }
      __syncwarp();  // the warp is done with stage st
      if (lane == 0) mbar_arrive(&empty[st]);
    }
  }
  pdl_trigger();
  if (timed_out) atomicOr(&cd.flags[2], ERR_TIMEOUT);
  const ff v = block_sum_ff_pair(acc_sig.result(), red, red + 32);
  if (threadIdx.x == 0) st_part_ff(part_w_of(L, j) + blockIdx.x, v);
  __syncthreads();
  unsigned long long* acc = fx_acc_of(L, j);
  fx_accumulate([&](int b, int c, int w) { return (long long)bins[(b * C + c) * NW + w]; }, L.s, C, acc);
  if (blockIdx.x == 0) {
    if (threadIdx.x == 0) reinterpret_cast<long long*>(acc)[3 * L.s] = fxs.E;
    if (MAT) mat_coefficients_store(L, cd, s_c);
  }
  if (j == L.m) ff_mat_finish(L, cd, MAT ? 1 : 0);  // else the next materialize kernel sums the partials
}

// Four consecutive matrix values, read as one aligned 16-byte (float) or two
// 16-byte (float-float pair) loads.
template <typename AT> struct Vals4;
template <> struct Vals4<float> {
  float4 v;
  __device__ __forceinline__ void load(const float* p, int c4) { v = __ldg(reinterpret_cast<const float4*>(p) + c4); }
  __device__ __forceinline__ float get(int q) const { return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w)); }
};
template <> struct Vals4<float2> {
  float4 a, b;
  __device__ __forceinline__ void load(const float2* p, int c4) {
    const float4* q4 = reinterpret_cast<const float4*>(p) + 2 * c4;
    a = __ldg(q4);
    b = __ldg(q4 + 1);
  }
  __device__ __forceinline__ float2 get(int q) const {
    return q == 0 ? make_float2(a.x, a.y)
                  : (q == 1 ? make_float2(a.z, a.w) : (q == 2 ? make_float2(b.x, b.y) : make_float2(b.z, b.w)));
  }
};
__device__ __forceinline__ int comp(const int4& v, int q) { return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w)); }

constexpr int UC_FF = 1;  // 16-byte chunks (4 nonzeros) per lane per batch

template <typename AT, int KW>
__global__ void __launch_bounds__(STEP_THREADS, 4) ff_spmv_kernel(const StepLaunch L, const CycleDev cd) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* stage = reinterpret_cast<float2*>(smem);  // [warps][STAGE] (p, e)
  const int j = L.j;
  if (cd.flags[1] != 0) return;  // breakdown in this cycle: no further products
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const float2* W = static_cast<const float2*>(L.W);
  const float2* Wj = W + (int64_t)j * L.ldw;
  const AT* val = static_cast<const AT*>(L.val);
  const int4* col4 = reinterpret_cast<const int4*>(L.col);
  const int dlo = max(0, j - L.k + 1);
  const int nd = L.rgs ? 0 : j - dlo + 1;  // window dots (none in a randomized Gram-Schmidt cycle)
  const float2* Wd[KW];
#pragma unroll
  for (int q = 0; q < KW; ++q) Wd[q] = W + (int64_t)(dlo + (q < nd ? q : 0)) * L.ldw;
  ffacc acc_pi;
  ffacc acc_dot[KW];
  float2* mystage = stage + wid * STAGE;
  const int r0 = blockIdx.x * L.rows_spmv;
  const int r1 = min(L.n, r0 + L.rows_spmv);
  for (int t0 = r0; t0 < r1; t0 += STEP_THREADS) {
    const int i0 = t0 + wid * 32;
    if (i0 >= r1) continue;  // warp-uniform
    const int i = i0 + lane;
    const bool valid = i < r1;
    const int nval = min(32, r1 - i0);
    int rb = 0, re = 0;
    ff wq[KW];
    if (valid) {
      rb = __ldg(L.row_ptr + i);
      re = __ldg(L.row_ptr + i + 1);
#pragma unroll
      for (int q = 0; q < KW; ++q)
        if (q < nd) wq[q] = ld_ff(Wd[q] + i);
    }
    const int ebeg = __shfl_sync(FULL, rb, 0);
    const int eend = __shfl_sync(FULL, re, nval - 1);
    const int nent = eend - ebeg;
    ffacc acc;
    if (nent <= STAGE - 4) {
      // 16-byte chunks of the warp's nonzero range, starting at the aligned
      // chunk that contains ebeg (arrays are padded past nnz)
      const int cbase = ebeg >> 2;
      const int nch = ((eend + 3) >> 2) - cbase;
      for (int cb = 0; cb < nch; cb += 32 * UC_FF) {
        int4 cc[UC_FF];
        Vals4<AT> av[UC_FF];
#pragma unroll
        for (int u = 0; u < UC_FF; ++u) {
          const int ch = cb + u * 32 + lane;
          cc[u] = make_int4(0, 0, 0, 0);
          if (ch < nch) {
            cc[u] = __ldg(col4 + cbase + ch);
            av[u].load(val, cbase + ch);
          }
        }
        ff wv[UC_FF][4];
#pragma unroll
        for (int u = 0; u < UC_FF; ++u) {
          const int e0 = (cbase + cb + u * 32 + lane) * 4;
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (e0 + q >= ebeg && e0 + q < eend) wv[u][q] = ld_ff(Wj + comp(cc[u], q));
        }
#pragma unroll
        for (int u = 0; u < UC_FF; ++u) {
          const int e0 = (cbase + cb + u * 32 + lane) * 4;
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (e0 + q >= ebeg && e0 + q < eend) mystage[e0 + q - ebeg] = prod_pe(av[u].get(q), wv[u][q]);
        }
      }
      __syncwarp();
      if (valid)
        for (int k = rb - ebeg; k < re - ebeg; ++k) {
          const float2 pe = mystage[k];
          acc.add_pe(pe.x, pe.y);
        }
      __syncwarp();
    } else if (valid) {
      for (int e = rb; e < re; ++e) {
        const float2 pe = prod_pe(__ldg(val + e), ld_ff(Wj + __ldg(L.col + e)));
        acc.add_pe(pe.x, pe.y);
      }
    }
    if (valid) {
      const ff p = acc.result();
      st_ff(static_cast<float2*>(L.p_out) + i, p);
      acc_pi.add_prod(p, p);
#pragma unroll
      for (int q = 0; q < KW; ++q)
        if (q < nd) acc_dot[q].add_prod(wq[q], p);
    }
  }
  ff_spmv_finish<KW>(L, cd, acc_pi, acc_dot, nd, L.part + (size_t)blockIdx.x * NQ, L.rgs && L.n_long == 0,
                     L.part, (int)gridDim.x, nullptr, 0);
}

// ---------------------------------------------------------------------------
// Product kernel with bulk-copy staging of the CSR stream (float-float basis).
// The CTA walks its rows in tiles of 256; for tile t the row_ptr slice and the
// tile's column/value slices are brought into shared memory by one thread with
// cp.async.bulk (completion tracked by an mbarrier), two tiles ahead in a
// double buffer, so the CSR bytes stream while the previous tile computes.
// Each thread then forms its row's product from shared memory; only the
// gathers of w_j stay on the critical path.  Waits are bounded: on timeout the
// kernel sets ERR_TIMEOUT and keeps going (the host reports it).
constexpr int TMA_ROWS = STEP_THREADS;     // rows per staged tile
constexpr int TMA_RP = TMA_ROWS + 4;       // staged row_ptr entries (16-byte multiple)
constexpr int TMA_ROW_FAST = 8;            // rows up to this length issue all gathers together
#ifndef KRYLOV_SPMV_STAGES
#define KRYLOV_SPMV_STAGES 2
#endif
constexpr int TMA_STAGES = KRYLOV_SPMV_STAGES;  // CSR tiles in flight per CTA of the staged product
// a stage holds at most 260 row_ptr entries and 4104 (int, float2) nonzeros
// (50.3 KB): four of them still fit the 227 KB of shared memory of a CTA
static_assert(TMA_STAGES >= 2 && TMA_STAGES <= 4, "staged CSR tiles in flight");

// Stage of the staged product kernel: row_ptr slice, columns (4-byte indices,
// or 2-byte offsets col - row when DI), values.  cap is a multiple of 8.
template <typename AT, bool DI = false>
__host__ __device__ __forceinline__ size_t tma_stage_bytes(int cap) {
  return (size_t)TMA_RP * 4 + (size_t)cap * (DI ? 2 : 4) + (size_t)cap * sizeof(AT);
}

__device__ __forceinline__ void acc_val(ffacc& acc, float a, ff w) {
  const float2 pe = prod_pe(a, w);
  acc.add_pe(pe.x, pe.y);
}
__device__ __forceinline__ void acc_val(ffacc& acc, float2 a, ff w) {
  const float2 pe = prod_pe(a, w);
  acc.add_pe(pe.x, pe.y);
}

template <typename AT, int KW, bool DI>
__global__ void __launch_bounds__(STEP_THREADS, 3) ff_spmv_tma_kernel(const StepLaunch L, const CycleDev cd) {
  using CT = typename std::conditional<DI, int16_t, int>::type;  // staged column entry
  constexpr int EA = DI ? 8 : 4;  // staged nonzero ranges start on 16-byte boundaries
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[TMA_STAGES];
  const int j = L.j;
  const int cap = L.tma_cap;
  const size_t sb = tma_stage_bytes<AT, DI>(cap);
  // stage st: row_ptr slice (TMA_RP ints), columns (cap CT), values (cap AT)
  auto rp_st = [&](int st) { return reinterpret_cast<int*>(smem + (size_t)st * sb); };
  auto col_st = [&](int st) { return reinterpret_cast<CT*>(rp_st(st) + TMA_RP); };
  auto val_st = [&](int st) { return reinterpret_cast<AT*>(col_st(st) + cap); };
  const CT* colsrc = DI ? reinterpret_cast<const CT*>(L.dcol) : reinterpret_cast<const CT*>(L.col);
  const float2* W = static_cast<const float2*>(L.W);
  const float2* Wj = W + (int64_t)j * L.ldw;
  const AT* val = static_cast<const AT*>(L.val);
  const int dlo = max(0, j - L.k + 1);
  const int nd = L.rgs ? 0 : j - dlo + 1;  // window dots (none in a randomized Gram-Schmidt cycle)
  const float2* Wd[KW];
#pragma unroll
  for (int q = 0; q < KW; ++q) Wd[q] = W + (int64_t)(dlo + (q < nd ? q : 0)) * L.ldw;
  const int r0 = blockIdx.x * L.rows_spmv;
  const int r1 = min(L.n, r0 + L.rows_spmv);
  const int ntiles = (r1 > r0) ? (r1 - r0 + TMA_ROWS - 1) / TMA_ROWS : 0;
  if (threadIdx.x == 0) {
    for (int q = 0; q < TMA_STAGES; ++q) mbar_init(&bars[q], 1);
    fence_mbar_init();
  }
  __syncthreads();
  // thread 0: stage tile t given its nonzero range [e0, e1)
  auto issue = [&](int t, int e0, int e1) {
    const int st = t % TMA_STAGES;
    const int ts = r0 + t * TMA_ROWS;
    const int ea = e0 & ~(EA - 1), eb = (e1 + EA - 1) & ~(EA - 1);
    const uint32_t brp = TMA_RP * 4u, bcol = (uint32_t)(eb - ea) * (uint32_t)sizeof(CT),
                   bval = (uint32_t)(eb - ea) * sizeof(AT);
    mbar_arrive_expect_tx(&bars[st], brp + bcol + bval);
    bulk_g2s_stream(rp_st(st), L.row_ptr + ts, brp, &bars[st]);
    if (eb > ea) {
      bulk_g2s_stream(col_st(st), colsrc + ea, bcol, &bars[st]);
      bulk_g2s_stream(val_st(st), val + ea, bval, &bars[st]);
    }
  };
  auto tile_end = [&](int t) { return min(r0 + (t + 1) * TMA_ROWS, r1); };
  if (threadIdx.x == 0)
    for (int t = 0; t < min(ntiles, TMA_STAGES); ++t)
      issue(t, __ldg(L.row_ptr + r0 + t * TMA_ROWS), __ldg(L.row_ptr + tile_end(t)));
  // the CSR stream does not depend on earlier kernels: its first tiles are on
  // their way before waiting for the kernel that produced w_j
  pdl_wait();
  if (cd.flags[1] != 0) {  // breakdown in this cycle: no further products
    if (threadIdx.x == 0)
      for (int t = 0; t < min(ntiles, TMA_STAGES); ++t) (void)mbar_wait_bounded(&bars[t], 0u, TMA_WAIT_NS);
    return;
  }
  ffacc acc_pi;
  ffacc acc_dot[KW];
  bool timed_out = false;
  int last_issued = min(ntiles, TMA_STAGES) - 1;  // thread 0: last tile whose copies were issued
  for (int t = 0; t < ntiles; ++t) {
    const int st = t % TMA_STAGES;
    const uint32_t par = (uint32_t)(t / TMA_STAGES) & 1u;
    const int ts = r0 + t * TMA_ROWS;
    const int i = ts + (int)threadIdx.x;
    const bool valid = i < tile_end(t);
    int nb0 = 0, nb1 = 0;
    if (threadIdx.x == 0 && t + TMA_STAGES < ntiles) {  // boundaries of the next tile to issue, loaded early
      nb0 = __ldg(L.row_ptr + ts + TMA_STAGES * TMA_ROWS);
      nb1 = __ldg(L.row_ptr + tile_end(t + TMA_STAGES));
    }
    ff wq[KW];
    if (valid) {
#pragma unroll
      for (int q = 0; q < KW; ++q)
        if (q < nd) wq[q] = ld_ff(Wd[q] + i);
    }
    if (!timed_out && !mbar_wait_bounded(&bars[st], par, TMA_WAIT_NS)) timed_out = true;
    if (valid && !timed_out) {
      const int* rps = rp_st(st);
      const CT* cs = col_st(st);
      const AT* vs = val_st(st);
      const int ea = rps[0] & ~(EA - 1);
      const int rb = rps[threadIdx.x] - ea, re = rps[threadIdx.x + 1] - ea;
      const int cbase = DI ? i : 0;  // column = cbase + staged entry
      ffacc acc;
      if (re - rb <= TMA_ROW_FAST) {
        // short rows: every gather of the row in flight at once
        float2 wv[TMA_ROW_FAST];
#pragma unroll
        for (int q = 0; q < TMA_ROW_FAST; ++q)
          if (rb + q < re) wv[q] = __ldg(Wj + (cbase + (int)cs[rb + q]));
#pragma unroll
        for (int q = 0; q < TMA_ROW_FAST; ++q)
          if (rb + q < re) acc_val(acc, vs[rb + q], ff{wv[q].x, wv[q].y});
      } else {
#pragma unroll 4
        for (int e = rb; e < re; ++e) acc_val(acc, vs[e], ld_ff(Wj + (cbase + (int)cs[e])));
      }
      const ff p = acc.result();
      st_ff(static_cast<float2*>(L.p_out) + i, p);
      acc_pi.add_prod(p, p);
#pragma unroll
      for (int q = 0; q < KW; ++q)
        if (q < nd) acc_dot[q].add_prod(wq[q], p);
    }
    __syncthreads();  // every thread is done with stage st
    if (threadIdx.x == 0 && t + TMA_STAGES < ntiles && !timed_out) {
      fence_proxy_async();
      issue(t + TMA_STAGES, nb0, nb1);
      last_issued = t + TMA_STAGES;
    }
  }
  pdl_trigger();
  if (timed_out) atomicOr(&cd.flags[2], ERR_TIMEOUT);
  if (threadIdx.x == 0 && timed_out) {
    // let copies still in flight land before the CTA exits (bounded again)
    for (int t = max(0, last_issued - TMA_STAGES + 1); t <= last_issued; ++t)
      (void)mbar_wait_bounded(&bars[t % TMA_STAGES], (uint32_t)(t / TMA_STAGES) & 1u, TMA_WAIT_NS);
  }
  ff_spmv_finish<KW>(L, cd, acc_pi, acc_dot, nd, L.part + (size_t)blockIdx.x * NQ, L.rgs && L.n_long == 0,
                     L.part, (int)gridDim.x, nullptr, 0);
}

// Product kernel on the sliced layout: a 256-row tile's entries padded to the
// tile's longest row L and stored slot-major (entry q of row r at q * 256 + r,
// column offsets col - row, padding offset 0 and value 0), so a tile is two
// contiguous bulk copies, entry q of every thread is one conflict-free shared
// load, and a row needs neither row_ptr nor a per-entry bound test: the
// entry loop is unrolled for the tile's L (uniform over a 256-thread group).
// Padding adds exact zeros after a row's own entries, so every row's sum
// equals the CSR kernels' (storage order).
//
// A stage holds SELL_GROUPS consecutive tiles (two bulk copies, the tiles
// being contiguous) and group g of the CTA's 256-thread groups forms the
// rows of tile g; stages are sized by the operator's longest tile row.
// Resident CTAs of one SM drift apart (the warp scheduler favours the
// oldest: with four 256-thread CTAs per SM the last finished ~5 us after the
// first), and groups that meet at every stage finish together but wait for
// each other at the barrier.  Measured per Arnoldi step on the 128^3
// convection-diffusion operator: four CTAs of one group 54.9 us, one CTA of
// four groups 54.3 us, two CTAs of two groups 53.4 us.
constexpr int SELL_GROUPS = 2;
constexpr int SELL_THREADS = SELL_GROUPS * TMA_ROWS;
constexpr int SELL_STAGES = 2;

// bytes of one stage for an operator whose longest tile row is maxl
template <typename AT>
__host__ __device__ constexpr size_t sell_stage_bytes(int maxl) {
  return align16((size_t)SELL_GROUPS * maxl * TMA_ROWS * 2) + (size_t)SELL_GROUPS * maxl * TMA_ROWS * sizeof(AT);
}

template <int NL, typename AT>
__device__ __forceinline__ ff sell_row(const int16_t* cs, const AT* vs, const float2* Wj, int i, int k) {
  float2 wv[NL];
  AT av[NL];
#pragma unroll
  for (int q = 0; q < NL; ++q) {
    av[q] = vs[q * TMA_ROWS + k];
    wv[q] = __ldg(Wj + (i + (int)cs[q * TMA_ROWS + k]));
  }
  ffacc acc;
#pragma unroll
  for (int q = 0; q < NL; ++q) acc_val(acc, av[q], ff{wv[q].x, wv[q].y});
  return acc.result();
}

template <typename AT, int KW>
__global__ void __launch_bounds__(SELL_THREADS, SELL_GROUPS == 1 ? 3 : 4 / SELL_GROUPS) ff_spmv_sell_kernel(const StepLaunch L, const CycleDev cd) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[SELL_STAGES];
  const size_t SB = sell_stage_bytes<AT>(L.sell_maxl);
  const size_t VOFF = align16((size_t)SELL_GROUPS * L.sell_maxl * TMA_ROWS * 2);  // value part of a stage
  const int j = L.j;
  const float2* W = static_cast<const float2*>(L.W);
  const float2* Wj = W + (int64_t)j * L.ldw;
  const AT* sval = static_cast<const AT*>(L.sell_val);
  const int dlo = max(0, j - L.k + 1);
  const int nd = L.rgs ? 0 : j - dlo + 1;
  const float2* Wd[KW];
#pragma unroll
  for (int q = 0; q < KW; ++q) Wd[q] = W + (int64_t)(dlo + (q < nd ? q : 0)) * L.ldw;
  const int r0 = blockIdx.x * L.rows_spmv;
  const int r1 = min(L.n, r0 + L.rows_spmv);
  const int ntiles = (r1 > r0) ? (r1 - r0 + TMA_ROWS - 1) / TMA_ROWS : 0;
  const int nst = (ntiles + SELL_GROUPS - 1) / SELL_GROUPS;  // stages of SELL_GROUPS tiles
  const int g0 = r0 / TMA_ROWS;  // global tile of the CTA's first tile
  const int grp = (int)threadIdx.x / TMA_ROWS, k = (int)threadIdx.x % TMA_ROWS;
  if (threadIdx.x == 0) {
    for (int q = 0; q < SELL_STAGES; ++q) mbar_init(&bars[q], 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto issue = [&](int t) {  // thread 0: the tiles of stage t, two copies
    const int st = t % SELL_STAGES;
    const int ta = g0 + t * SELL_GROUPS, tb = g0 + min(ntiles, (t + 1) * SELL_GROUPS);
    const int e0 = __ldg(L.sell_off + ta), e1 = __ldg(L.sell_off + tb);
    const uint32_t bc = (uint32_t)(e1 - e0) * 2u, bv = (uint32_t)(e1 - e0) * (uint32_t)sizeof(AT);
    mbar_arrive_expect_tx(&bars[st], bc + bv);
    if (e1 > e0) {
      unsigned char* base = smem + (size_t)st * SB;
      bulk_g2s_stream(base, L.sell_col + e0, bc, &bars[st]);
      bulk_g2s_stream(base + VOFF, sval + e0, bv, &bars[st]);
    }
  };
  if (threadIdx.x == 0)
    for (int t = 0; t < min(nst, SELL_STAGES); ++t) issue(t);
  pdl_wait();
  if (cd.flags[1] != 0) {
    if (threadIdx.x == 0)
      for (int t = 0; t < min(nst, SELL_STAGES); ++t) (void)mbar_wait_bounded(&bars[t], 0u, TMA_WAIT_NS);
    return;
  }
  ffacc acc_pi;
  ffacc acc_dot[KW];
  bool timed_out = false;
  int last_issued = min(nst, SELL_STAGES) - 1;
  for (int t = 0; t < nst; ++t) {
    const int st = t % SELL_STAGES;
    const uint32_t par = (uint32_t)(t / SELL_STAGES) & 1u;
    const int tl = t * SELL_GROUPS + grp;  // this group's tile (local index)
    const int i = r0 + tl * TMA_ROWS + k;
    const bool valid = tl < ntiles && i < r1;
    // this tile's place in the stage and its row length (uniform over the group)
    const int ea = __ldg(L.sell_off + g0 + t * SELL_GROUPS);
    const int eg = valid ? __ldg(L.sell_off + g0 + tl) : ea;
    const int nl = valid ? (__ldg(L.sell_off + g0 + tl + 1) - eg) / TMA_ROWS : 0;
    ff wq[KW];
    if (valid) {
#pragma unroll
      for (int q = 0; q < KW; ++q)
        if (q < nd) wq[q] = ld_ff(Wd[q] + i);
    }
    if (!timed_out && !mbar_wait_bounded(&bars[st], par, TMA_WAIT_NS)) timed_out = true;
    if (valid && !timed_out) {
      const int16_t* cs = reinterpret_cast<const int16_t*>(smem + (size_t)st * SB) + (eg - ea);
      const AT* vs = reinterpret_cast<const AT*>(smem + (size_t)st * SB + VOFF) + (eg - ea);
      ff p;
      switch (nl) {  // the same for every thread of the group
        case 1: p = sell_row<1>(cs, vs, Wj, i, k); break;
        case 2: p = sell_row<2>(cs, vs, Wj, i, k); break;
        case 3: p = sell_row<3>(cs, vs, Wj, i, k); break;
        case 4: p = sell_row<4>(cs, vs, Wj, i, k); break;
        case 5: p = sell_row<5>(cs, vs, Wj, i, k); break;
        case 6: p = sell_row<6>(cs, vs, Wj, i, k); break;
        case 7: p = sell_row<7>(cs, vs, Wj, i, k); break;
        case 8: p = sell_row<8>(cs, vs, Wj, i, k); break;
        default: {
          ffacc acc;
          for (int q = 0; q < nl; ++q)
            acc_val(acc, vs[q * TMA_ROWS + k], ld_ff(Wj + (i + (int)cs[q * TMA_ROWS + k])));
          p = acc.result();
        }
      }
      st_ff(static_cast<float2*>(L.p_out) + i, p);
      acc_pi.add_prod(p, p);
#pragma unroll
      for (int q = 0; q < KW; ++q)
        if (q < nd) acc_dot[q].add_prod(wq[q], p);
    }
    __syncthreads();  // every group is done with stage st
    if (threadIdx.x == 0 && t + SELL_STAGES < nst && !timed_out) {
      fence_proxy_async();
      issue(t + SELL_STAGES);
      last_issued = t + SELL_STAGES;
    }
  }
  pdl_trigger();
  if (timed_out) atomicOr(&cd.flags[2], ERR_TIMEOUT);
  if (threadIdx.x == 0 && timed_out) {
    for (int t = max(0, last_issued - SELL_STAGES + 1); t <= last_issued; ++t)
      (void)mbar_wait_bounded(&bars[t % SELL_STAGES], (uint32_t)(t / SELL_STAGES) & 1u, TMA_WAIT_NS);
  }
  ff_spmv_finish<KW>(L, cd, acc_pi, acc_dot, nd, L.part + (size_t)blockIdx.x * NQ, L.rgs && L.n_long == 0,
                     L.part, (int)gridDim.x, nullptr, 0);
}

// ---------------------------------------------------------------------------

size_t fused_smem(int basis, int s, int copies) {
  const size_t a = (basis == 0) ? 8 : 4;
  return align16(bins_bytes(basis, s, copies)) + (size_t)(STEP_THREADS / 32) * STAGE * a;
}

template <typename VT, typename AT, bool MAT, bool SPMV, int SKM>
void launch_fused(const StepLaunch& L, const CycleDev& cd, int basis, cudaStream_t st) {
  const size_t smem = fused_smem(basis, L.s, L.sk_copies);
  auto k = step_kernel<VT, AT, MAT, SPMV, SKM>;
  raise_smem_limit((const void*)k, smem);
  k<<<L.grid, STEP_THREADS, smem, st>>>(L, cd);
}

template <typename VT, typename AT, bool MAT, bool SPMV>
void fused_sk(const StepLaunch& L, const CycleDev& cd, int basis, cudaStream_t st) {
  switch (L.sk_mode) {
    case SK_TAB8: launch_fused<VT, AT, MAT, SPMV, SK_TAB8>(L, cd, basis, st); break;
    case SK_TAB16: launch_fused<VT, AT, MAT, SPMV, SK_TAB16>(L, cd, basis, st); break;
    case SK_GEN8: launch_fused<VT, AT, MAT, SPMV, SK_GEN8>(L, cd, basis, st); break;
    default: launch_fused<VT, AT, MAT, SPMV, SK_GEN>(L, cd, basis, st); break;
  }
}

template <typename VT, typename AT>
void fused_dispatch(const StepLaunch& L, const CycleDev& cd, int basis, cudaStream_t st) {
  if (L.mat && L.spmv) fused_sk<VT, AT, true, true>(L, cd, basis, st);
  else if (L.mat) fused_sk<VT, AT, true, false>(L, cd, basis, st);
  else if (L.spmv) fused_sk<VT, AT, false, true>(L, cd, basis, st);
  else fused_sk<VT, AT, false, false>(L, cd, basis, st);
}

template <bool MAT, int SKM>
void launch_ff_mat_t(const StepLaunch& L, const CycleDev& cd, cudaStream_t st) {
  const size_t smem = bins_bytes(3, L.s, L.sk_copies);
  auto k = (L.k <= 2) ? ff_mat_kernel<MAT, SKM, 2> : ff_mat_kernel<MAT, SKM, MAX_WINDOW>;
  raise_smem_limit((const void*)k, smem);
  k<<<L.grid, STEP_THREADS, smem, st>>>(L, cd);
}

size_t mt_smem(int s, int copies, int kw) { return align16(bins_bytes(3, s, copies)) + MT_STAGES * mt_stage_bytes(kw); }

template <bool MAT>
void launch_ff_mat(const StepLaunch& L, const CycleDev& cd, cudaStream_t st) {
  switch (L.sk_mode) {
    case SK_TAB8: {  // packed table: row streams staged by bulk copies
      const int kw = (L.k <= 2) ? 2 : MAX_WINDOW;
      const size_t smem = mt_smem(L.s, L.sk_copies, kw);
      auto pick = [&](auto kw2, auto kw4) { return (L.k <= 2) ? kw2 : kw4; };
      auto k = (L.sk_copies == 32)
                   ? ((L.zeta == 8) ? pick(ff_mat_tma_kernel<MAT, 2, 32, 8>, ff_mat_tma_kernel<MAT, MAX_WINDOW, 32, 8>)
                                    : pick(ff_mat_tma_kernel<MAT, 2, 32, 0>, ff_mat_tma_kernel<MAT, MAX_WINDOW, 32, 0>))
                   : ((L.zeta == 8) ? pick(ff_mat_tma_kernel<MAT, 2, 16, 8>, ff_mat_tma_kernel<MAT, MAX_WINDOW, 16, 8>)
                                    : pick(ff_mat_tma_kernel<MAT, 2, 16, 0>, ff_mat_tma_kernel<MAT, MAX_WINDOW, 16, 0>));
      raise_smem_limit((const void*)k, smem);
      launch_pdl_threads(k, L.grid_mat, MT_BLOCK, smem, st, L, cd);
      break;
    }
    case SK_TAB16: launch_ff_mat_t<MAT, SK_TAB16>(L, cd, st); break;
    case SK_GEN8: launch_ff_mat_t<MAT, SK_GEN8>(L, cd, st); break;
    default: launch_ff_mat_t<MAT, SK_GEN>(L, cd, st); break;
  }
}

// ---------------------------------------------------------------------------
// Product kernel with the w_j gathers served from shared memory (float-float
// basis, operators with a segment plan).  For each 256-row tile a plan built
// at create lists the few contiguous pieces of w_j that the tile's columns
// touch (a stencil tile touches three: its own neighbourhood and the two
// planes at +-N^2) and stores, per nonzero, the 16-bit position of its column
// among the staged pieces.  Thread 0 copies the tile's row_ptr slice, its
// 16-bit positions, its values and the pieces of w_j into shared memory with
// bulk asynchronous copies (two tiles in flight); each thread then forms its
// row with shared-memory loads only.  The CSR parts do not depend on earlier
// kernels and are issued before the dependent-launch wait, the pieces of w_j
// after it.
template <typename AT>
__host__ __device__ __forceinline__ size_t seg_stage_bytes(int lcap, int seg_cap) {
  return (size_t)TMA_RP * 4 + (size_t)lcap * (2 + sizeof(AT)) + (size_t)seg_cap * sizeof(float2);
}

template <typename AT, int KW>
__global__ void __launch_bounds__(STEP_THREADS, 3) ff_spmv_seg_kernel(const StepLaunch L, const CycleDev cd) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[2];
  const int j = L.j;
  const int lcap = L.lcap;
  const size_t sb = seg_stage_bytes<AT>(lcap, L.seg_cap);
  auto rp_st = [&](int st) { return reinterpret_cast<int*>(smem + (size_t)st * sb); };
  auto lc_st = [&](int st) { return reinterpret_cast<uint16_t*>(smem + (size_t)st * sb + (size_t)TMA_RP * 4); };
  auto val_st = [&](int st) {
    return reinterpret_cast<AT*>(smem + (size_t)st * sb + (size_t)TMA_RP * 4 + (size_t)lcap * 2);
  };
  auto w_st = [&](int st) {
    return reinterpret_cast<float2*>(smem + (size_t)st * sb + (size_t)TMA_RP * 4 + (size_t)lcap * (2 + sizeof(AT)));
  };
  const float2* W = static_cast<const float2*>(L.W);
  const float2* Wj = W + (int64_t)j * L.ldw;
  const AT* val = static_cast<const AT*>(L.val);
  const int dlo = max(0, j - L.k + 1);
  const int nd = L.rgs ? 0 : j - dlo + 1;  // window dots (none in a randomized Gram-Schmidt cycle)
  const float2* Wd[KW];
#pragma unroll
  for (int q = 0; q < KW; ++q) Wd[q] = W + (int64_t)(dlo + (q < nd ? q : 0)) * L.ldw;
  const int r0 = blockIdx.x * L.rows_spmv;
  const int r1 = min(L.n, r0 + L.rows_spmv);
  const int ntiles = (r1 > r0) ? (r1 - r0 + TMA_ROWS - 1) / TMA_ROWS : 0;
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto tile_end = [&](int t) { return min(r0 + (t + 1) * TMA_ROWS, r1); };
  // thread 0: announce all bytes of tile t and copy its CSR parts
  auto issue_csr = [&](int t) {
    const int st = t & 1;
    const int ts = r0 + t * TMA_ROWS;
    const int g = ts / TMA_ROWS;
    const int e0 = __ldg(L.row_ptr + ts), e1 = __ldg(L.row_ptr + tile_end(t));
    const int ea = e0 & ~7, eb = (e1 + 7) & ~7;
    const int ns = __ldg(L.seg_n + g);
    uint32_t wbytes = 0;
    for (int q = 0; q < ns; ++q) wbytes += (uint32_t)__ldg(&L.seg[(size_t)g * SEG_MAX + q].y) * 8u;
    const uint32_t brp = TMA_RP * 4u, blc = (uint32_t)(eb - ea) * 2u, bval = (uint32_t)(eb - ea) * sizeof(AT);
    mbar_arrive_expect_tx(&bars[st], brp + blc + bval + wbytes);
    bulk_g2s(rp_st(st), L.row_ptr + ts, brp, &bars[st]);
    if (eb > ea) {
      bulk_g2s(lc_st(st), L.lcol + ea, blc, &bars[st]);
      bulk_g2s(val_st(st), val + ea, bval, &bars[st]);
    }
  };
  // thread 0: copy the pieces of w_j of tile t (after w_j is complete)
  auto issue_w = [&](int t) {
    const int st = t & 1;
    const int g = (r0 + t * TMA_ROWS) / TMA_ROWS;
    const int ns = __ldg(L.seg_n + g);
    for (int q = 0; q < ns; ++q) {
      const int4 sg = __ldg(&L.seg[(size_t)g * SEG_MAX + q]);
      bulk_g2s(w_st(st) + sg.z, Wj + sg.x, (uint32_t)sg.y * 8u, &bars[st]);
    }
  };
  if (threadIdx.x == 0)
    for (int t = 0; t < min(ntiles, 2); ++t) issue_csr(t);
  pdl_wait();
  if (threadIdx.x == 0)
    for (int t = 0; t < min(ntiles, 2); ++t) issue_w(t);  // also on breakdown: the phases must complete
  if (cd.flags[1] != 0) {  // breakdown in this cycle: no further products
    if (threadIdx.x == 0)
      for (int t = 0; t < min(ntiles, 2); ++t) (void)mbar_wait_bounded(&bars[t], 0u, TMA_WAIT_NS);
    return;
  }
  ffacc acc_pi;
  ffacc acc_dot[KW];
  bool timed_out = false;
  int last_issued = min(ntiles, 2) - 1;
  for (int t = 0; t < ntiles; ++t) {
    const int st = t & 1;
    const uint32_t par = (uint32_t)(t >> 1) & 1u;
    const int ts = r0 + t * TMA_ROWS;
    const int i = ts + (int)threadIdx.x;
    const bool valid = i < tile_end(t);
    ff wq[KW];
    if (valid) {
#pragma unroll
      for (int q = 0; q < KW; ++q)
        if (q < nd) wq[q] = ld_ff(Wd[q] + i);
    }
    if (!timed_out && !mbar_wait_bounded(&bars[st], par, TMA_WAIT_NS)) timed_out = true;
    if (valid && !timed_out) {
      const int* rps = rp_st(st);
      const uint16_t* lcs = lc_st(st);
      const AT* vs = val_st(st);
      const float2* ws = w_st(st);
      const int ea = rps[0] & ~7;
      const int rb = rps[threadIdx.x] - ea, re = rps[threadIdx.x + 1] - ea;
      ffacc acc;
#pragma unroll 4
      for (int e = rb; e < re; ++e) {
        const float2 w2 = ws[lcs[e]];
        acc_val(acc, vs[e], ff{w2.x, w2.y});
      }
      const ff p = acc.result();
      st_ff(static_cast<float2*>(L.p_out) + i, p);
      acc_pi.add_prod(p, p);
#pragma unroll
      for (int q = 0; q < KW; ++q)
        if (q < nd) acc_dot[q].add_prod(wq[q], p);
    }
    __syncthreads();  // every thread is done with stage st
    if (threadIdx.x == 0 && t + 2 < ntiles && !timed_out) {
      fence_proxy_async();
      issue_csr(t + 2);
      issue_w(t + 2);
      last_issued = t + 2;
    }
  }
  pdl_trigger();
  if (timed_out) atomicOr(&cd.flags[2], ERR_TIMEOUT);
  if (threadIdx.x == 0 && timed_out) {
    for (int t = max(0, last_issued - 1); t <= last_issued; ++t)
      (void)mbar_wait_bounded(&bars[t & 1], (uint32_t)(t >> 1) & 1u, TMA_WAIT_NS);
  }
  ff_spmv_finish<KW>(L, cd, acc_pi, acc_dot, nd, L.part + (size_t)blockIdx.x * NQ, L.rgs && L.n_long == 0,
                     L.part, (int)gridDim.x, nullptr, 0);
}

// ---------------------------------------------------------------------------
// Long rows of a power-law operator (float-float basis).  Runs after the
// product kernel of the emptied operator (which gave p_i = 0 on these rows
// and kept its partials).  The rows come longest first: each of the first
// n_big (more than 1024 nonzeros) takes a whole CTA in turn (rows
// blockIdx.x, blockIdx.x + grid, ...), its threads striding over the row's
// nonzeros and a fixed block tree summing them; every other row takes a warp
// (rows n_big + blockIdx.x * warps + warp, stepping by grid * warps) with a
// fixed shuffle tree.  p_i overwrites the zero and the thread that holds it
// adds its shares of ||p||^2 and of the window dots; a fixed block sum makes
// the CTA's partials.  The next materialize kernel's CTAs sum both kernels'
// partials (the emptied operator's CTAs, then these, each in CTA order); in a
// randomized Gram-Schmidt cycle the last CTA here sums ||p||^2 the same way.
template <typename AT, int KW>
__global__ void __launch_bounds__(STEP_THREADS) ff_spmv_long_kernel(const StepLaunch L, const CycleDev cd) {
  __shared__ float rhi[32], rlo[32];
  pdl_wait();  // w_j and the products of the other rows are complete
  if (cd.flags[1] != 0) return;  // breakdown in this cycle: no further products
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int j = L.j;
  const float2* W = static_cast<const float2*>(L.W);
  const float2* Wj = W + (int64_t)j * L.ldw;
  const AT* val = static_cast<const AT*>(L.val_full);
  const int dlo = max(0, j - L.k + 1);
  const int nd = L.rgs ? 0 : j - dlo + 1;
  const float2* Wd[KW];
#pragma unroll
  for (int q = 0; q < KW; ++q) Wd[q] = W + (int64_t)(dlo + (q < nd ? q : 0)) * L.ldw;
  ffacc acc_pi;
  ffacc acc_dot[KW];
  auto finish_row = [&](int i, ff p) {
    st_ff(static_cast<float2*>(L.p_out) + i, p);
    acc_pi.add_prod(p, p);
#pragma unroll
    for (int q = 0; q < KW; ++q)
      if (q < nd) acc_dot[q].add_prod(ld_ff(Wd[q] + i), p);
  };
  for (int r = blockIdx.x; r < L.n_big; r += gridDim.x) {  // a CTA per row
    const int i = __ldg(L.long_rows + r);
    const int e0 = __ldg(L.rp_full + i), e1 = __ldg(L.rp_full + i + 1);
    ffacc acc;
#pragma unroll 4
    for (int e = e0 + (int)threadIdx.x; e < e1; e += (int)blockDim.x)
      acc_val(acc, val[e], ld_ff(Wj + __ldg(L.col_full + e)));
    const ff p = block_sum_ff_pair(acc.result(), rhi, rlo);
    if (threadIdx.x == 0) finish_row(i, p);
  }
  for (int r = L.n_big + (int)blockIdx.x * nwarp + wid; r < L.n_long; r += (int)gridDim.x * nwarp) {  // a warp per row
    const int i = __ldg(L.long_rows + r);
    const int e0 = __ldg(L.rp_full + i), e1 = __ldg(L.rp_full + i + 1);
    ffacc acc;
#pragma unroll 4
    for (int e = e0 + lane; e < e1; e += 32) acc_val(acc, val[e], ld_ff(Wj + __ldg(L.col_full + e)));
    ff p = acc.result();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) p = ff_add(p, ff{__shfl_xor_sync(FULL, p.hi, o), __shfl_xor_sync(FULL, p.lo, o)});
    if (lane == 0) finish_row(i, p);
  }
  pdl_trigger();
  // per-CTA partials: only the threads that finished rows hold nonzero sums
  ff_spmv_finish<KW>(L, cd, acc_pi, acc_dot, nd, L.part_long + (size_t)blockIdx.x * NQ, L.rgs != 0, L.part, L.grid_spmv,
                     L.part_long, (int)gridDim.x);
}

constexpr size_t FF_STAGE_SMEM = (size_t)(STEP_THREADS / 32) * STAGE * sizeof(float2);

template <typename AT, int KW>
void launch_ff_spmv_main(const StepLaunch& L, const CycleDev& cd, cudaStream_t st);

// The product of a step: the kernel of the (possibly emptied) operator, then,
// for a power-law operator, the long-row kernel that completes and reduces it.
template <typename AT, int KW>
void launch_ff_spmv_t(const StepLaunch& L, const CycleDev& cd, cudaStream_t st) {
  launch_ff_spmv_main<AT, KW>(L, cd, st);
  if (L.n_long > 0) launch_pdl(ff_spmv_long_kernel<AT, KW>, L.grid_long, 0, st, L, cd);
}

template <typename AT, int KW>
void launch_ff_spmv_main(const StepLaunch& L, const CycleDev& cd, cudaStream_t st) {
  if (L.seg != nullptr) {
    auto k = ff_spmv_seg_kernel<AT, KW>;
    const size_t smem = 2 * seg_stage_bytes<AT>(L.lcap, L.seg_cap);
    raise_smem_limit((const void*)k, smem);
    launch_pdl(k, L.grid_spmv, smem, st, L, cd);
    return;
  }
  if (L.sell_col != nullptr) {
    auto k = ff_spmv_sell_kernel<AT, KW>;
    const size_t smem = SELL_STAGES * sell_stage_bytes<AT>(L.sell_maxl);
    raise_smem_limit((const void*)k, smem);
    launch_pdl_threads(k, L.grid_spmv, SELL_THREADS, smem, st, L, cd);
    return;
  }
  if (L.tma_cap > 0 && L.dcol != nullptr) {
    auto k = ff_spmv_tma_kernel<AT, KW, true>;
    const size_t smem = TMA_STAGES * tma_stage_bytes<AT, true>(L.tma_cap);
    raise_smem_limit((const void*)k, smem);
    launch_pdl(k, L.grid_spmv, smem, st, L, cd);
    return;
  }
  if (L.tma_cap > 0) {
    auto k = ff_spmv_tma_kernel<AT, KW, false>;
    const size_t smem = TMA_STAGES * tma_stage_bytes<AT>(L.tma_cap);
    raise_smem_limit((const void*)k, smem);
    launch_pdl(k, L.grid_spmv, smem, st, L, cd);
    return;
  }
  auto k = ff_spmv_kernel<AT, KW>;
  raise_smem_limit((const void*)k, FF_STAGE_SMEM);
  k<<<L.grid_spmv, STEP_THREADS, FF_STAGE_SMEM, st>>>(L, cd);
}

void launch_ff_prod(const StepLaunch& L, const CycleDev& cd, cudaStream_t st) {
  if (L.val_f32) {
    if (L.k <= 2 || L.rgs) launch_ff_spmv_t<float, 2>(L, cd, st);
    else launch_ff_spmv_t<float, MAX_WINDOW>(L, cd, st);
  } else {
    if (L.k <= 2 || L.rgs) launch_ff_spmv_t<float2, 2>(L, cd, st);
    else launch_ff_spmv_t<float2, MAX_WINDOW>(L, cd, st);
  }
}

void launch_ff_step(const StepLaunch& L, const CycleDev& cd, cudaStream_t st) {
  if (L.mat) launch_ff_mat<true>(L, cd, st);
  else launch_ff_mat<false>(L, cd, st);
  if (L.spmv) {
    if (L.val_f32) {
      if (L.k <= 2) launch_ff_spmv_t<float, 2>(L, cd, st);
      else launch_ff_spmv_t<float, MAX_WINDOW>(L, cd, st);
    } else {
      if (L.k <= 2) launch_ff_spmv_t<float2, 2>(L, cd, st);
      else launch_ff_spmv_t<float2, MAX_WINDOW>(L, cd, st);
    }
  }
}

template <typename K>
int occ(K kern, size_t smem, int threads = STEP_THREADS) {
  raise_smem_limit((const void*)kern, smem);
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, threads, smem);
  return b < 1 ? 1 : b;
}

}  // namespace

int sketch_bin_copies(int basis, int s) {
  // lane-private copies: the largest power of two <= 32 whose bins fit in
  // 48 KB, or 64 KB for the float-float materialize kernel, where 32 copies
  // (one per lane: the bank of every atomic is its lane) remove the conflicts
  // of lanes l and l + 16 that 16 copies leave (2.35 wavefronts per shared
  // atomic); that costs resident CTAs and still wins 1.5 % per step
  int c = 32;
  while (c > 1 && bins_bytes(basis, s, c) > (basis == 3 ? 64 : 48) * 1024) c >>= 1;
  return c;
}

// Bits per fixed-point word so that no bin column can overflow: a column
// receives at most ceil(rows_per_cta / copies) contributions of magnitude
// below 1.2 * 2^(wb-1), so per * 2^(wb+1) < 2^31 (wb = 30 - log2 per) leaves
// room, and the rounding trick needs wb <= 22.
int sketch_word_bits(int rows_per_cta, int copies) {
  const long long per = (rows_per_cta + copies - 1) / copies + 1;
  int lg = 0;
  while ((1ll << lg) < per) ++lg;
  return std::max(12, std::min(21, 30 - lg));
}

// Resident CTAs per SM of the main step kernel(s) (one persistent wave).
// Resident CTAs per SM of the float-float product kernel for this operator.
int spmv_ctas_per_sm(int vals_f32, int tma_cap, int seg_cap, int lcap) {
  if (seg_cap > 0)
    return vals_f32 ? occ(ff_spmv_seg_kernel<float, 2>, 2 * seg_stage_bytes<float>(lcap, seg_cap))
                    : occ(ff_spmv_seg_kernel<float2, 2>, 2 * seg_stage_bytes<float2>(lcap, seg_cap));
  if (tma_cap > 0)
    return vals_f32 ? occ(ff_spmv_tma_kernel<float, 2, false>, TMA_STAGES * tma_stage_bytes<float>(tma_cap))
                    : occ(ff_spmv_tma_kernel<float2, 2, false>, TMA_STAGES * tma_stage_bytes<float2>(tma_cap));
  return vals_f32 ? occ(ff_spmv_kernel<float, 2>, FF_STAGE_SMEM) : occ(ff_spmv_kernel<float2, 2>, FF_STAGE_SMEM);
}

size_t sell_smem_bytes(int vals_f32, int maxl) {
  return SELL_STAGES * (vals_f32 ? sell_stage_bytes<float>(maxl) : sell_stage_bytes<float2>(maxl));
}

int sell_ctas_per_sm(int vals_f32, int maxl) {
  return vals_f32 ? occ(ff_spmv_sell_kernel<float, 2>, SELL_STAGES * sell_stage_bytes<float>(maxl), SELL_THREADS)
                  : occ(ff_spmv_sell_kernel<float2, 2>, SELL_STAGES * sell_stage_bytes<float2>(maxl), SELL_THREADS);
}

// Resident CTAs per SM of the float-float materialize kernel with the row
// streams staged by bulk copies (MT_BLOCK threads per CTA).
int mat_ctas_per_sm(int s, int copies) {
  return (copies == 32) ? occ(ff_mat_tma_kernel<true, 2, 32, 8>, mt_smem(s, copies, 2), MT_BLOCK)
                        : occ(ff_mat_tma_kernel<true, 2, 16, 8>, mt_smem(s, copies, 2), MT_BLOCK);
}

// CTAs per SM of the 256-thread step kernels (for the float-float basis: of
// the materialize kernel without staged row streams; the persistent wave of
// the other per-row kernels of a cycle is sized from it).
int step_ctas_per_sm(int basis, int sk_mode, int s, int copies, int vals_f32) {
  (void)sk_mode;
  if (basis == 3) return occ(ff_mat_kernel<true, SK_TAB8, 2>, bins_bytes(3, s, copies));
  const size_t smem = fused_smem(basis, s, copies);
  if (basis == 0)
    return vals_f32 ? occ(step_kernel<double, float, true, true, SK_TAB8>, smem)
                    : occ(step_kernel<double, double, true, true, SK_TAB8>, smem);
  if (basis == 1) return occ(step_kernel<float, float, true, true, SK_TAB8>, smem);
  return occ(step_kernel<__nv_bfloat16, float, true, true, SK_TAB8>, smem);
}

void launch_ff_product(const StepLaunch& L, const CycleDev& cd, cudaStream_t st) { launch_ff_prod(L, cd, st); }

void launch_step(int basis, const StepLaunch& L, const CycleDev& cd, int m, cudaStream_t st) {
  (void)m;
  if (basis == 3) {
    launch_ff_step(L, cd, st);
  } else if (basis == 0) {
    if (L.val_f32) fused_dispatch<double, float>(L, cd, basis, st);
    else fused_dispatch<double, double>(L, cd, basis, st);
  } else if (L.tma_cap > 0 && L.sk_mode == SK_TAB8 && !L.rgs) {  // staged pair (float32 / bfloat16)
    launch_step32(basis, L, cd, st);
  } else if (basis == 1) {
    fused_dispatch<float, float>(L, cd, basis, st);
  } else {
    fused_dispatch<__nv_bfloat16, float>(L, cd, basis, st);
  }
}

}  // namespace krylov
