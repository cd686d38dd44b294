// part_kernels.cu -- the Arnoldi steps of a row-partitioned solve: the kernels
// one rank runs on its own contiguous block of rows (float64 basis, truncated
// orthogonalization).
//
// Every n-length reduction of a step (||p||^2 and the window dots of the
// product, ||w_j||^2 of a new basis vector) is split in two: the kernel sums
// its rows' contributions in a fixed order into a small buffer, the host sums
// the buffers of all ranks (an all-reduce of at most k + 2 doubles), and a
// one-warp kernel turns the global sums into the next coefficients with the
// same reducers as the single-GPU step kernels (Algorithm 1's loop body with
// the truncated window).  Every rank therefore holds the same coefficients,
// R, and the same small projected problem, which it solves redundantly.
//
// The sketch columns are keyed by global row, so the sketch of a vector is the
// sum over ranks of the sketches of its row blocks (Eq. 3 applied
// columnwise).  Each rank accumulates its rows' contributions as exact
// fixed-point integer words (one power-of-two scale per basis column, taken
// from a bound that every rank computes from the same global sums), so the
// all-reduced sketch is the same integer sum whatever the partition.
//
// The product needs w_j at the columns a rank's rows reference outside its
// block (its halo): the rank packs the entries its neighbours need, the host
// exchanges them, and the received entries are written behind the local part
// of slot j, where the product's remapped column indices find them.
#include <algorithm>
#include <cmath>

#include "internal.h"
#include "kernels.cuh"
#include "step_common.cuh"

namespace krylov {
namespace {

__global__ void part_pack_kernel(const double* w, const int* idx, int count, double* out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) out[e] = w[idx[e]];
}

__global__ void part_unpack_kernel(const double* in, int count, double* w_halo) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) w_halo[e] = in[e];
}

// ||b|| from the all-reduced ||b||^2 (scal[4]): the scalars norm_b_kernel sets
// on one GPU.
__global__ void part_norm_finish_kernel(CycleDev cd) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const double t = cd.scal[4];
    const double eta = sqrt(t);
    cd.scal[0] = eta;
    cd.scal[1] = (eta > 0.0) ? 1.0 / eta : 0.0;
    cd.scal[5] = 1.0;  // w_1 = b / ||b||
    if (!isfinite(t)) cd.flags[2] |= ERR_NONFINITE;
  }
}

// Column j of the basis: w_j = rho_j (p_{j-1} - sum_q h_q w_q) over this
// rank's rows (MAT), or the start vector already in slot 0; its rows' share
// of ||w_j||^2 (into red[NQ]) and of the sketch S w_j (into the exact word
// sums acc[j][3][s]).
template <bool MAT, int SKM>
__global__ void __launch_bounds__(STEP_THREADS) part_mat_kernel(const PartLaunch P, const StepLaunch L,
                                                                const CycleDev cd) {
  constexpr int NW = 3;
  extern __shared__ __align__(16) unsigned char smem[];
  int* bins = reinterpret_cast<int*>(smem);  // [NW][s]
  __shared__ double red[32];
  __shared__ int s_last;
  __shared__ FxScale s_fx;
  __shared__ double s_c[MAX_WINDOW + 1];
  const int j = L.j;
  if (cd.flags[0] < j) return;  // the cycle ended before column j (breakdown)
  const int lo = MAT ? max(0, j - L.k) : j;
  const int nl = j - lo;
  for (int e = threadIdx.x; e < NW * L.s; e += blockDim.x) bins[e] = 0;
  if (threadIdx.x == 0) {
    s_fx = fx_scale(L, cd, MAT ? 1 : 0);
    const double* c = cd.coef + (size_t)(j > 0 ? j - 1 : 0) * (MAX_WINDOW + 1);
    for (int q = 0; q <= MAX_WINDOW; ++q) s_c[q] = c[q];
    if (blockIdx.x == 0) P.E[j] = s_fx.E;
  }
  __syncthreads();
  const FxScale fxs = s_fx;
  double* Wj = P.W + (int64_t)j * P.ldw;
  const SketchSpec sp = spec_of(L);
  const uint32_t inv_s = sketch_inv_s(L.s);
  double acc = 0.0;
  int bad = 0;
  const int r0 = blockIdx.x * P.rows_per_cta;
  const int r1 = min(P.n, r0 + P.rows_per_cta);
  for (int i = r0 + (int)threadIdx.x; i < r1; i += blockDim.x) {
    double w;
    if (MAT) {
      double a = P.p[i];
      for (int q = 0; q < nl; ++q) a = fma(-s_c[q], P.W[(int64_t)(lo + q) * P.ldw + i], a);
      w = a * s_c[MAX_WINDOW];
      Wj[i] = w;
    } else {
      w = Wj[i];
    }
    acc = fma(w, w, acc);
    const float vh = __double2float_rn(w);
    const float vl = __double2float_rn(w - (double)vh);
    const FxWords<NW> xw = fx_split<NW>(vh, vl, fxs);
    typename SkColOf<SKM>::type col;
    col.load(L, sp, inv_s, i);
    bad |= (col.got < L.zeta);
    for (int e = 0; e < col.got; ++e) fx_emit<NW>(bins, L.s, col.row(e), 0, xw, col.neg(e), 1);
  }
  if (bad) atomicOr(&cd.flags[2], ERR_SKETCH);
  const double v = block_sum(acc, red);
  if (threadIdx.x == 0) P.part[blockIdx.x] = v;
  __syncthreads();
  unsigned long long* colacc = reinterpret_cast<unsigned long long*>(P.acc) + (size_t)j * NW * L.s;
  for (int e = threadIdx.x; e < NW * L.s; e += blockDim.x) {
    const int q = bins[e];
    if (q != 0) atomicAdd(colacc + e, (unsigned long long)(long long)q);  // two's complement: exact signed sum
  }
  if (!last_block_flag(cd.counter, &s_last)) return;
  if (threadIdx.x < 32) {
    const double t = warp_sum_partials(P.part, (int)gridDim.x, 1, 0);
    if (threadIdx.x == 0) {
      P.red[NQ] = t;
      *cd.counter = 0u;
    }
  }
}

// p_j = A w_j over this rank's rows (columns past n are the halo entries of
// w_j), and its rows' shares of ||p_j||^2 (red[1]) and of the window dots
// <w_q, p_j> (red[2 + q]).
__global__ void __launch_bounds__(STEP_THREADS) part_product_kernel(const PartLaunch P, const StepLaunch L,
                                                                    const CycleDev cd) {
  __shared__ double red[32];
  __shared__ int s_last;
  __shared__ double tot[NQ];
  const int j = L.j;
  if (cd.flags[1] != 0) return;  // breakdown in this cycle: no further products
  const int dlo = max(0, j - L.k + 1);
  const int nd = j - dlo + 1;
  const double* Wj = P.W + (int64_t)j * P.ldw;
  double accp = 0.0, accd[MAX_WINDOW] = {0.0, 0.0, 0.0, 0.0};
  const int r0 = blockIdx.x * P.rows_per_cta;
  const int r1 = min(P.n, r0 + P.rows_per_cta);
  for (int i = r0 + (int)threadIdx.x; i < r1; i += blockDim.x) {
    double y = 0.0;
    for (int e = P.rp[i]; e < P.rp[i + 1]; ++e) y = fma(P.val[e], Wj[P.ci[e]], y);
    P.p[i] = y;
    accp = fma(y, y, accp);
#pragma unroll
    for (int q = 0; q < MAX_WINDOW; ++q)
      if (q < nd) accd[q] = fma(P.W[(int64_t)(dlo + q) * P.ldw + i], y, accd[q]);
  }
  double* part = P.part + (size_t)blockIdx.x * NQ;
  double v = block_sum(accp, red);
  if (threadIdx.x == 0) part[1] = v;
#pragma unroll
  for (int q = 0; q < MAX_WINDOW; ++q) {
    if (q >= nd) break;  // uniform over the block
    __syncthreads();
    v = block_sum(accd[q], red);
    if (threadIdx.x == 0) part[2 + q] = v;
  }
  if (!last_block_flag(cd.counter, &s_last)) return;
  for (int q = (int)(threadIdx.x >> 5); q < NQ; q += (int)(blockDim.x >> 5)) {
    const double t = (q >= 1 && q < 2 + nd) ? warp_sum_partials(P.part, (int)gridDim.x, NQ, q) : 0.0;
    if ((threadIdx.x & 31) == 0) tot[q] = t;
  }
  __syncthreads();
  if (threadIdx.x < NQ) P.red[threadIdx.x] = tot[threadIdx.x];
  if (threadIdx.x == 0) *cd.counter = 0u;
}

// The step kernels' reducers, on the all-reduced sums.
__global__ void part_reduce_mat_kernel(const StepLaunch L, const CycleDev cd, const double* red, int mat) {
  if (threadIdx.x == 0 && cd.flags[0] >= L.j) (void)reduce_mat(L, cd, red[NQ], mat);
}

__global__ void part_reduce_product_kernel(const StepLaunch L, const CycleDev cd, const double* red) {
  if (cd.flags[1] != 0) return;
  double tot[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) tot[q] = red[q];
  reduce_spmv(L, cd, tot, false);
}

// U[:, j] = (1/sqrt(zeta)) S w_j from the all-reduced exact word sums of
// column j, whose fixed-point exponent is E[j].
__global__ void part_sketch_u_kernel(const long long* acc, const int* E, int ncols, int s, int wb, double scale,
                                     double* U) {
  const int j = blockIdx.y;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ncols || b >= s) return;
  const long long* a = acc + (size_t)j * 3 * s;
  const int e = E[j];
  const double v = fma((double)a[b], pow2d(e - wb), fma((double)a[s + b], pow2d(e - 2 * wb),
                                                        (double)a[2 * s + b] * pow2d(e - 3 * wb)));
  U[(size_t)j * s + b] = scale * v;
}

}  // namespace

void launch_part_pack(const double* w, const int* idx, int count, double* out, cudaStream_t st) {
  if (count > 0) part_pack_kernel<<<std::min(1024, (count + 255) / 256), 256, 0, st>>>(w, idx, count, out);
}

void launch_part_unpack(const double* in, int count, double* w_halo, cudaStream_t st) {
  if (count > 0) part_unpack_kernel<<<std::min(1024, (count + 255) / 256), 256, 0, st>>>(in, count, w_halo);
}

void launch_part_norm_finish(const CycleDev& cd, cudaStream_t st) { part_norm_finish_kernel<<<1, 32, 0, st>>>(cd); }

size_t part_mat_smem(int s) { return (size_t)3 * s * sizeof(int); }

void launch_part_mat(const PartLaunch& P, const StepLaunch& L, const CycleDev& cd, int mat, cudaStream_t st) {
  const size_t smem = part_mat_smem(L.s);
  if (L.sk_mode == SK_TAB8) {
    auto k = mat ? part_mat_kernel<true, SK_TAB8> : part_mat_kernel<false, SK_TAB8>;
    raise_smem_limit((const void*)k, smem);
    k<<<P.grid, STEP_THREADS, smem, st>>>(P, L, cd);
  } else {
    auto k = mat ? part_mat_kernel<true, SK_TAB16> : part_mat_kernel<false, SK_TAB16>;
    raise_smem_limit((const void*)k, smem);
    k<<<P.grid, STEP_THREADS, smem, st>>>(P, L, cd);
  }
}

void launch_part_product(const PartLaunch& P, const StepLaunch& L, const CycleDev& cd, cudaStream_t st) {
  part_product_kernel<<<P.grid, STEP_THREADS, 0, st>>>(P, L, cd);
}

void launch_part_reduce_mat(const StepLaunch& L, const CycleDev& cd, const double* red, int mat, cudaStream_t st) {
  part_reduce_mat_kernel<<<1, 32, 0, st>>>(L, cd, red, mat);
}

void launch_part_reduce_product(const StepLaunch& L, const CycleDev& cd, const double* red, cudaStream_t st) {
  part_reduce_product_kernel<<<1, 32, 0, st>>>(L, cd, red);
}

void launch_part_sketch_u(const long long* acc, const int* E, int ncols, int s, int zeta, int wb, double* U,
                          cudaStream_t st) {
  dim3 g((s + 127) / 128, ncols);
  part_sketch_u_kernel<<<g, 128, 0, st>>>(acc, E, ncols, s, wb, 1.0 / std::sqrt((double)zeta), U);
}

}  // namespace krylov
