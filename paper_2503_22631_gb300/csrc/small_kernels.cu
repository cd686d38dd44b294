// small_kernels.cu -- the FP64 projected problem of one restart cycle.
//
// whiten_kernel   thin Householder QR of the sketched basis U = S W_{m+1}
//                 (only T is formed; diag(T) > 0), T_m^{-1}, the projected
//                 matrix X = T_m R_m T_m^{-1} + (r_{m+1,m} / T_m[m,m]) t e_m^T
//                 (App. A, Eq. A.1), g = T_m^{-1} t, tau = T[m+1,m+1], and the
//                 restart coupling of Algorithm 2 for the whitened basis:
//                 gamma = rho_prev T[1,1] with rho = r_{m+1,m} tau / T_m[m,m].
// exp kernels     the last block row of exp(-t H_{cm}) for the block lower
//                 bidiagonal H_{cm} of Algorithm 2, by scaling and squaring:
//                 B = -t H / 2^s, Taylor polynomial of degree q in Horner form
//                 for block row c, then s squarings that reuse the stored block
//                 rows of earlier cycles at every scale level.  Block row c of a
//                 square of a block lower triangular matrix needs only block
//                 rows <= c, so each cycle adds one block row per level instead
//                 of recomputing f(H_{cm}) from scratch; the result equals the
//                 last block row of the full scaling-and-squaring evaluation up
//                 to the order of the floating-point sums.
// inv_block       f(z) = 1/z: block forward substitution for H_{cm}^{-1} e_1,
//                 which needs only the last entry of the previous block.
// z_kernel        z = beta T_m^{-1} F[(c-1)m+1 : cm, 1] (Algorithm 2, update y).
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>

#include <cooperative_groups.h>

#include "internal.h"
#include "kernels.cuh"

namespace krylov {
namespace {

namespace cg = cooperative_groups;

constexpr int SMALL_THREADS = 256;
// the whitening QR works in shared memory when s x (m+1) doubles fit in this
constexpr int WHITEN_SMEM_DOUBLES = 20 * 1024;  // 160 KB
size_t whiten_smem(int s, int nc) {
  const size_t d = (size_t)s * nc;
  return d <= (size_t)WHITEN_SMEM_DOUBLES ? d * sizeof(double) : 0;
}

__device__ __forceinline__ double& Tat(double* Tw, int s, int a, int b) { return Tw[(size_t)b * s + a]; }

// Small dense products on GB300 are bound by the FP64 pipe (about two FMAs
// per clock per SM): each FP64 warp instruction occupies its SM sub-partition
// for many cycles, so a product is spread over as many SMs as possible and
// the dependent chain of each output is kept short.  One CTA forms 32
// consecutive entries e = col m + r of L R (m x m, column-major); the sum over
// p is cut into KS_WARPS contiguous ranges, one per warp, and warp 0 adds the
// partial sums in warp order (a fixed order: the result is deterministic).
constexpr int KS_WARPS = 4;
constexpr int KS_THREADS = 32 * KS_WARPS;

// Every thread of the CTA calls this (it holds a barrier); the sum is
// returned in warp 0, other warps get 0.
__device__ __forceinline__ double ks_product(const double* __restrict__ L, const double* __restrict__ R, int M,
                                             int e, double (*red)[32]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int chunk = (M + KS_WARPS - 1) / KS_WARPS;
  const int p0 = w * chunk, p1 = min(M, p0 + chunk);
  double acc = 0.0;
  if (e < M * M) {
    const int r = e % M, col = e / M;
    const double* Lr = L + r;
    const double* Rc = R + (size_t)col * M;
#pragma unroll 4
    for (int p = p0; p < p1; ++p) acc = fma(Lr[(size_t)p * M], Rc[p], acc);
  }
  red[w][lane] = acc;
  __syncthreads();
  double sum = 0.0;
  if (w == 0) {
    sum = red[0][lane];
#pragma unroll
    for (int q = 1; q < KS_WARPS; ++q) sum += red[q][lane];
  }
  return sum;
}

__global__ void __launch_bounds__(SMALL_THREADS) whiten_kernel(SmallDev sd, CycleDev cd, int s, int M,
                                                               int nc, int me, int has_next, int cycle,
                                                               double t, double* scratch, const BatchStride bs) {
  // problem blockIdx.x of a batch (strides are zero for a single problem)
  sd = offset_sd(sd, bs, blockIdx.x);
  cd = offset_cd(cd, bs, blockIdx.x);
  scratch += bs.S0 * blockIdx.x;
  extern __shared__ double sA[];  // the sketched basis in shared memory when it fits
  __shared__ double red[32];
  __shared__ double sh_beta_h;
  __shared__ double diag[1024];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarp = blockDim.x >> 5;
  const bool in_smem = (size_t)s * nc <= (size_t)WHITEN_SMEM_DOUBLES;
  double* A = in_smem ? sA : sd.Tw;  // s x nc, leading dimension s

  for (size_t e = tid; e < (size_t)s * nc; e += blockDim.x) A[e] = sd.U[e];
  __syncthreads();

  // ---- Householder QR, T only ----
  // Two barriers per column: the reflector of column jj is formed by thread 0
  // from the squared norm that the warp updating column jj (in the previous
  // pass) left in sh_nrm2; the trailing update then applies it, and the warp
  // that updates column jj + 1 also forms that column's squared norm below
  // the diagonal for the next pass.
  __shared__ double sh_nrm2;
  {
    double acc = 0.0;
    for (int r = tid; r < s; r += blockDim.x) acc = fma(A[r], A[r], acc);
    const double v = block_sum(acc, red);
    if (tid == 0) sh_nrm2 = v;
  }
  __syncthreads();
  for (int jj = 0; jj < nc; ++jj) {
    if (tid == 0) {
      const double nrm2 = sh_nrm2;
      const double x0 = A[(size_t)jj * s + jj];
      const double nx = sqrt(nrm2);
      const double alpha = (x0 >= 0.0) ? -nx : nx;
      const double v0 = x0 - alpha;
      const double vn2 = nrm2 - x0 * x0 + v0 * v0;
      A[(size_t)jj * s + jj] = v0;
      sh_beta_h = (vn2 > 0.0) ? 2.0 / vn2 : 0.0;
      diag[jj] = alpha;
    }
    __syncthreads();
    const double bh = sh_beta_h;
    for (int l = jj + 1 + wid; l < nc; l += nwarp) {
      double d = 0.0;
      for (int r = jj + lane; r < s; r += 32) d = fma(A[(size_t)jj * s + r], A[(size_t)l * s + r], d);
      d = warp_sum(d) * bh;
      if (l == jj + 1) {  // also the squared norm of the updated column below row jj
        double q = 0.0;
        for (int r = jj + lane; r < s; r += 32) {
          const double u = fma(-d, A[(size_t)jj * s + r], A[(size_t)l * s + r]);
          A[(size_t)l * s + r] = u;
          if (r > jj) q = fma(u, u, q);
        }
        q = warp_sum(q);
        if (lane == 0) sh_nrm2 = q;
      } else {
        for (int r = jj + lane; r < s; r += 32) A[(size_t)l * s + r] = fma(-d, A[(size_t)jj * s + r], A[(size_t)l * s + r]);
      }
    }
    __syncthreads();
  }
  // sign fix: row a of T times sign(diag[a]); write diagonal
  for (int e = tid; e < nc * nc; e += blockDim.x) {
    const int a = e % nc, b = e / nc;
    if (a < b) {
      const double sg = (diag[a] < 0.0) ? -1.0 : 1.0;
      Tat(A, s, a, b) *= sg;
    }
  }
  __syncthreads();
  for (int a = tid; a < nc; a += blockDim.x) Tat(A, s, a, a) = fabs(diag[a]);
  __syncthreads();
  if (in_smem) {  // T (upper nc x nc of A) stays readable in global memory
    for (size_t e = tid; e < (size_t)s * nc; e += blockDim.x) sd.Tw[e] = A[e];
  }

  // ---- T_m^{-1} (upper triangular), one column per thread ----
  double* Ti = sd.Tinv;  // me x me, leading dimension M
  for (int b = tid; b < me; b += blockDim.x) {
    for (int a = me - 1; a > b; --a) Ti[(size_t)b * M + a] = 0.0;
    Ti[(size_t)b * M + b] = 1.0 / Tat(A, s, b, b);
    for (int a = b - 1; a >= 0; --a) {
      double acc = 0.0;
      for (int l = a + 1; l <= b; ++l) acc = fma(Tat(A, s, a, l), Ti[(size_t)b * M + l], acc);
      Ti[(size_t)b * M + a] = -acc / Tat(A, s, a, a);
    }
  }
  __syncthreads();

  // ---- TR = T_m R_m (R banded upper Hessenberg) into scratch ----
  const int ldr = M + 1;
  for (int e = tid; e < me * me; e += blockDim.x) {
    const int a = e % me, b = e / me;
    double acc = 0.0;
    const int l1 = min(b + 1, me - 1);
    for (int l = a; l <= l1; ++l) acc = fma(Tat(A, s, a, l), cd.R[(size_t)b * ldr + l], acc);
    scratch[(size_t)b * M + a] = acc;
  }
  __syncthreads();
  // ---- X = TR T_m^{-1} + (r / T_mm) t e_m^T, zero padded to M x M ----
  double* X = sd.Xblk + (size_t)(cycle - 1) * M * M;
  const double r = has_next ? cd.R[(size_t)(me - 1) * ldr + me] : 0.0;
  const double rt = has_next ? r / Tat(A, s, me - 1, me - 1) : 0.0;
  for (int e = tid; e < M * M; e += blockDim.x) {
    const int a = e % M, b = e / M;
    double acc = 0.0;
    if (a < me && b < me) {
      for (int l = 0; l <= b; ++l) acc = fma(scratch[(size_t)l * M + a], Ti[(size_t)b * M + l], acc);
      if (b == me - 1 && has_next) acc = fma(rt, Tat(A, s, a, me), acc);
    }
    X[e] = acc;
  }
  __syncthreads();
  // ---- g = T_m^{-1} t, tau, norms ----
  for (int a = tid; a < me; a += blockDim.x) {
    double acc = 0.0;
    if (has_next)
      for (int l = a; l < me; ++l) acc = fma(Ti[(size_t)l * M + a], Tat(A, s, l, me), acc);
    sd.zg[M + a] = acc;
  }
  // column sums of |X| for ||tX||_1, and ||T||_1 ||T^{-1}||_1 for the condition estimate
  double cmax = 0.0, tmax = 0.0, timax = 0.0;
  for (int b = tid; b < me; b += blockDim.x) {
    double cs = 0.0, ts = 0.0, tis = 0.0;
    for (int a = 0; a < me; ++a) {
      cs += fabs(X[(size_t)b * M + a]);
      if (a <= b) {
        ts += fabs(Tat(A, s, a, b));
        tis += fabs(Ti[(size_t)b * M + a]);
      }
    }
    cmax = fmax(cmax, cs);
    tmax = fmax(tmax, ts);
    timax = fmax(timax, tis);
  }
  for (int o = 16; o > 0; o >>= 1) {
    cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
    tmax = fmax(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
    timax = fmax(timax, __shfl_xor_sync(0xffffffffu, timax, o));
  }
  __shared__ double wmax[3][32];
  if (lane == 0) {
    wmax[0][wid] = cmax;
    wmax[1][wid] = tmax;
    wmax[2][wid] = timax;
  }
  __syncthreads();
  if (tid == 0) {
    double c0 = 0, c1 = 0, c2 = 0;
    for (int w = 0; w < nwarp; ++w) {
      c0 = fmax(c0, wmax[0][w]);
      c1 = fmax(c1, wmax[1][w]);
      c2 = fmax(c2, wmax[2][w]);
    }
    const double T11 = Tat(A, s, 0, 0);
    double* misc = sd.misc;
    if (cycle == 1) {
      misc[0] = cd.scal[0] * T11;  // beta = ||b|| T[1,1]
      misc[3] = 0.0;
    } else {
      const double gam = misc[1] * T11;  // gamma of the previous coupling
      sd.gam[cycle - 2] = gam;
      misc[3] = fabs(t * gam);
    }
    if (has_next) {
      const double tau = Tat(A, s, me, me);
      misc[1] = r * tau / Tat(A, s, me - 1, me - 1);
      sd.zg[2 * M] = 1.0 / tau;
    } else {
      misc[1] = 0.0;
      sd.zg[2 * M] = 0.0;
    }
    misc[2] = fabs(t) * c0;
    misc[4] = c1 * c2;
    bool ok = isfinite(c0) && isfinite(c1) && isfinite(c2) && isfinite(misc[0]) && isfinite(misc[1]);
    if (!ok) cd.flags[2] |= ERR_NONFINITE;
  }
}

// ---- whitening on a thread-block cluster ----
// The whitening is a chain of nc Householder reflectors whose FP64 work
// (each FP64 warp instruction holds its SM sub-partition for many cycles on
// this part) overwhelms one SM.  Here the columns of U are dealt round-robin
// to the CL CTAs of a cluster (column l lives in the shared memory of CTA
// l mod CL); reflector jj is formed by the warp that owns column jj, every
// CTA reads it from the owner's shared memory (distributed shared memory)
// and applies it to its own columns, one cluster barrier per column.  The
// warp that updates column jj + 1 also forms its squared norm below the
// diagonal and the next reflector, so the chain between two barriers is one
// column update.  Then every CTA gathers T (signs fixed so that diag(T) > 0)
// and each warp takes one column b: the column sweep of T x = e_b gives
// column b of T_m^{-1}, and column b of T_m R_m comes from the band of R_m
// (rows b - k + 1 .. b + 1 of column b hold the only nonzeros of the
// truncated recurrence); the extra column b = me solves T_m g = t.  After a
// cluster barrier each warp forms its columns of X = (T_m R_m) T_m^{-1} +
// (r / T_mm) t e_m^T in that association (the product T_m R_m first, then
// the inverse), the order of the definition in App. A.
constexpr int WC_THREADS = 256;
constexpr size_t WC_SMEM_MAX = 200 * 1024;

size_t whiten_cluster_smem(int s, int nc, int cl) {
  const size_t ncl = (size_t)((nc + cl - 1) / cl);
  return ((size_t)s * ncl + 4 * (size_t)nc + (size_t)nc * nc + (size_t)(WC_THREADS / 32) * 2 * nc) * sizeof(double);
}

// Householder reflector of column col below row jj: v = x - alpha e_1 written
// over the column (row jj holds v_0), beta = 2 / (v^T v), alpha = -sign(x_0) |x|.
__device__ __forceinline__ void wc_reflector(double* col, int jj, double nrm2, double* sbeta, double* salpha) {
  const double x0 = col[jj];
  const double nx = sqrt(nrm2);
  const double alpha = (x0 >= 0.0) ? -nx : nx;
  const double v0 = x0 - alpha;
  const double vn2 = nrm2 - x0 * x0 + v0 * v0;
  col[jj] = v0;
  sbeta[jj] = (vn2 > 0.0) ? 2.0 / vn2 : 0.0;
  salpha[jj] = alpha;
}

// Back substitution T[0..top][0..top] x = rhs by columns (rhs in x on entry):
// x_l = x_l / T_ll, then x_a -= T_al x_l for every a < l (lanes over a).
__device__ __forceinline__ void wc_sweep(double* x, const double* sT, int ldt, const double* dinv, int top,
                                         int lane) {
  for (int l = top; l >= 0; --l) {
    const double xl = x[l] * dinv[l];
    __syncwarp();
    for (int a = lane; a < l; a += 32) x[a] = fma(-sT[(size_t)l * ldt + a], xl, x[a]);
    if (lane == 0) x[l] = xl;
    __syncwarp();
  }
}

__global__ void __launch_bounds__(WC_THREADS) whiten_cluster_kernel(SmallDev sd, CycleDev cd, int s, int M, int nc,
                                                                    int me, int has_next, int cycle, int kw,
                                                                    double t, double* scratch, const BatchStride bs) {
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int prob = (int)(blockIdx.x / (unsigned)CL);  // problem of a batch (one cluster each)
  sd = offset_sd(sd, bs, prob);
  cd = offset_cd(cd, bs, prob);
  scratch += bs.S0 * prob;  // T_m R_m (leading dimension M)
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarp = blockDim.x >> 5;
  const int ncl = (nc + CL - 1) / CL;
  extern __shared__ double wsm[];
  double* Aloc = wsm;                      // s x ncl: slot q holds column q CL + rank
  double* sbeta = Aloc + (size_t)s * ncl;  // [nc] reflector scalars of own columns
  double* salpha = sbeta + nc;             // [nc] alpha of own columns
  double* diag = salpha + nc;              // [nc] alpha of every column
  double* dinv = diag + nc;                // [nc] 1 / T_aa
  double* sT = dinv + nc;                  // nc x nc, T (upper triangle, leading dimension nc)
  double* xw = sT + (size_t)nc * nc;       // per warp: x [nc], z [nc]
  __shared__ double wmax[3][WC_THREADS / 32];
  __shared__ double cta_max[3];

  for (int q = 0; q < ncl; ++q) {
    const int l = q * CL + rank;
    if (l >= nc) break;
    for (int r = tid; r < s; r += blockDim.x) Aloc[(size_t)q * s + r] = sd.U[(size_t)l * s + r];
  }
  __syncthreads();
  if (rank == 0 && wid == 0) {
    double acc = 0.0;
    for (int r = lane; r < s; r += 32) acc = fma(Aloc[r], Aloc[r], acc);
    acc = warp_sum(acc);
    if (lane == 0) wc_reflector(Aloc, 0, acc, sbeta, salpha);
  }
  // ---- Householder QR, one reflector per cluster barrier ----
  for (int jj = 0; jj < nc; ++jj) {
    cluster.sync();  // reflector jj is formed (and visible) in CTA jj mod CL
    const int o = jj % CL;
    const double* v = cluster.map_shared_rank(Aloc, o) + (size_t)(jj / CL) * s;
    const double beta = cluster.map_shared_rank(sbeta, o)[jj];
    const int q0 = (jj + 1 > rank) ? (jj + 1 - rank + CL - 1) / CL : 0;  // first own column after jj
    for (int q = q0 + wid; q < ncl; q += nwarp) {
      const int l = q * CL + rank;
      if (l >= nc) break;
      double* u = Aloc + (size_t)q * s;
      double d = 0.0;
      for (int r = jj + lane; r < s; r += 32) d = fma(v[r], u[r], d);
      d = warp_sum(d) * beta;
      if (l == jj + 1) {  // the next column: its norm below row jj and its reflector
        double nq = 0.0;
        for (int r = jj + lane; r < s; r += 32) {
          const double x = fma(-d, v[r], u[r]);
          u[r] = x;
          if (r > jj) nq = fma(x, x, nq);
        }
        nq = warp_sum(nq);
        __syncwarp();
        if (lane == 0) wc_reflector(u, l, nq, sbeta, salpha);
      } else {
        for (int r = jj + lane; r < s; r += 32) u[r] = fma(-d, v[r], u[r]);
      }
    }
  }
  // ---- T with diag(T) > 0: gathered by every CTA; own columns to global ----
  for (int a = tid; a < nc; a += blockDim.x) {
    const double al = cluster.map_shared_rank(salpha, a % CL)[a];
    diag[a] = al;
    dinv[a] = 1.0 / fabs(al);
  }
  __syncthreads();
  for (size_t e = tid; e < (size_t)nc * nc; e += blockDim.x) {
    const int a = (int)(e % nc), b = (int)(e / nc);
    double x = 0.0;
    if (a < b) {
      x = cluster.map_shared_rank(Aloc, b % CL)[(size_t)(b / CL) * s + a];
      if (diag[a] < 0.0) x = -x;
    } else if (a == b) {
      x = fabs(diag[a]);
    }
    sT[e] = x;
  }
  for (int q = 0; q < ncl; ++q) {
    const int l = q * CL + rank;
    if (l >= nc) break;
    for (int r = tid; r < s; r += blockDim.x) {
      double x = Aloc[(size_t)q * s + r];
      if (r < l) x = (diag[r] < 0.0) ? -x : x;
      else if (r == l) x = fabs(diag[l]);
      sd.Tw[(size_t)l * s + r] = x;
    }
  }
  __syncthreads();

  // ---- per column b: T_m^{-1} e_b, (T_m R_m) e_b, norms; b = me: g = T_m^{-1} t ----
  const int ldr = M + 1;
  const double r_next = has_next ? cd.R[(size_t)(me - 1) * ldr + me] : 0.0;
  const double rt = has_next ? r_next / sT[(size_t)(me - 1) * nc + me - 1] : 0.0;
  double* X = sd.Xblk + (size_t)(cycle - 1) * M * M;
  double* x = xw + (size_t)wid * 2 * nc;
  double cmax = 0.0, tmax = 0.0, timax = 0.0;
  const int ntask = max(M, me + 1);
  for (int b = rank * nwarp + wid; b < ntask; b += CL * nwarp) {
    if (b < me) {
      for (int a = lane; a <= b; a += 32) x[a] = (a == b) ? 1.0 : 0.0;
      __syncwarp();
      wc_sweep(x, sT, nc, dinv, b, lane);
      double ci = 0.0, ct = 0.0;
      for (int a = lane; a < me; a += 32) {
        const double y = (a <= b) ? x[a] : 0.0;
        sd.Tinv[(size_t)b * M + a] = y;
        ci += fabs(y);
        if (a <= b) ct += fabs(sT[(size_t)b * nc + a]);
        // (T_m R_m)[a, b]: R_m has its nonzeros in rows b - k + 1 .. b + 1 of column b
        const int l0 = max(a, b - kw + 1), l1 = min(b + 1, me - 1);
        double tr = 0.0;
        for (int l = l0; l <= l1; ++l) tr = fma(sT[(size_t)l * nc + a], cd.R[(size_t)b * ldr + l], tr);
        scratch[(size_t)b * M + a] = tr;
      }
      ci = warp_sum(ci);
      ct = warp_sum(ct);
      timax = fmax(timax, ci);
      tmax = fmax(tmax, ct);
      __syncwarp();
    } else if (b == me) {
      if (has_next) {
        for (int a = lane; a < me; a += 32) x[a] = sT[(size_t)me * nc + a];
        __syncwarp();
        wc_sweep(x, sT, nc, dinv, me - 1, lane);
      }
      for (int a = lane; a < me; a += 32) sd.zg[M + a] = has_next ? x[a] : 0.0;
      __syncwarp();
    }
  }
  cluster.sync();  // T_m^{-1} and T_m R_m complete (global memory)
  // ---- X = (T_m R_m) T_m^{-1} + (r / T_mm) t e_m^T, column b per warp ----
  for (int b = rank * nwarp + wid; b < M; b += CL * nwarp) {
    double cs = 0.0;
    for (int a = lane; a < M; a += 32) {
      double acc = 0.0;
      if (a < me && b < me) {
        for (int l = 0; l <= b; ++l)
          acc = fma(__ldcg(scratch + (size_t)l * M + a), __ldcg(sd.Tinv + (size_t)b * M + l), acc);
        if (b == me - 1 && has_next) acc = fma(rt, sT[(size_t)me * nc + a], acc);
      }
      X[(size_t)b * M + a] = acc;
      cs += fabs(acc);
    }
    cs = warp_sum(cs);
    if (b < me) cmax = fmax(cmax, cs);
  }
  if (lane == 0) {
    wmax[0][wid] = cmax;
    wmax[1][wid] = tmax;
    wmax[2][wid] = timax;
  }
  __syncthreads();
  if (tid == 0) {
    double c0 = 0.0, c1 = 0.0, c2 = 0.0;
    for (int w = 0; w < nwarp; ++w) {
      c0 = fmax(c0, wmax[0][w]);
      c1 = fmax(c1, wmax[1][w]);
      c2 = fmax(c2, wmax[2][w]);
    }
    cta_max[0] = c0;
    cta_max[1] = c1;
    cta_max[2] = c2;
  }
  cluster.sync();  // every CTA's maxima are in place
  if (rank == 0 && tid == 0) {
    double c0 = 0.0, c1 = 0.0, c2 = 0.0;
    for (int q = 0; q < CL; ++q) {
      const double* cm = cluster.map_shared_rank(cta_max, q);
      c0 = fmax(c0, cm[0]);
      c1 = fmax(c1, cm[1]);
      c2 = fmax(c2, cm[2]);
    }
    const double T11 = sT[0];
    double* misc = sd.misc;
    if (cycle == 1) {
      misc[0] = cd.scal[0] * T11;  // beta = ||b|| T[1,1]
      misc[3] = 0.0;
    } else {
      const double gam = misc[1] * T11;  // gamma of the previous coupling
      sd.gam[cycle - 2] = gam;
      misc[3] = fabs(t * gam);
    }
    if (has_next) {
      const double tau = sT[(size_t)me * nc + me];
      misc[1] = r_next * tau / sT[(size_t)(me - 1) * nc + me - 1];
      sd.zg[2 * M] = 1.0 / tau;
    } else {
      misc[1] = 0.0;
      sd.zg[2 * M] = 0.0;
    }
    misc[2] = fabs(t) * c0;
    misc[4] = c1 * c2;
    const bool ok = isfinite(c0) && isfinite(c1) && isfinite(c2) && isfinite(misc[0]) && isfinite(misc[1]);
    if (!ok) cd.flags[2] |= ERR_NONFINITE;
  }
  cluster.sync();  // no CTA leaves while rank 0 reads its shared memory
}

// One Horner step for block row a of T_q(B), B = scale * H (scale = -t/2^s):
//   S_new[j] = (S_old[j] X_j scale + S_old[j+1](:,1) scale gamma_j e_m^T) / kdeg + E[j]
// with E the block row of the identity (E[a] = I).  first: S_old = E.
// KSW = KS_WARPS: the CTA forms one chunk of 32 entries with the inner sum
// split over its warps (one problem: latency first).  KSW = 1: each warp forms
// its own chunk with whole inner sums (a batch of problems: the FP64 pipe is
// saturated anyway, and the split's partial sums are extra FP64 work).
//
// phi_1 (gout non-null, last step only): with the augmented matrix
// [[B, w], [0, 0]], w = e_1 2^-s, the Horner recurrence S <- S B / k + I
// carries the extra column S_old w / k, so the Taylor polynomial's extra
// column is S^(2) w: the first column of block (a, 0) of the iterate before
// the last step, times 2^-s (gscale).  It is stored as level 0 of the phi_1
// vector of block row a.
template <int KSW>
__global__ void __launch_bounds__(KS_THREADS) exp_taylor_kernel(const double* __restrict__ Xblk,
                                                                const double* __restrict__ gam, int M, int a,
                                                                double kinv, double scale, int first,
                                                                const double* __restrict__ Sold,
                                                                double* __restrict__ Snew, int64_t sx, int64_t sg,
                                                                int64_t s_old, int64_t s_new,
                                                                double* __restrict__ gout, double gscale) {
  static_assert(KSW == KS_WARPS || KSW == 1, "inner sum split over all warps of the CTA or none");
  // problem blockIdx.z of a batch: X blocks, couplings and the Horner buffers
  // at strides sx, sg, s_old, s_new (zero for a single problem)
  Xblk += sx * blockIdx.z;
  gam += sg * blockIdx.z;
  Sold += s_old * blockIdx.z;
  Snew += s_new * blockIdx.z;
  if (gout != nullptr && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0)
    for (int r = threadIdx.x; r < M; r += blockDim.x) gout[r] = Sold[r] * gscale;
  __shared__ double red[KS_WARPS][32];
  const int j = blockIdx.y;  // j <= a (grid rows)
  const int w = threadIdx.x >> 5;
  const int chunk = (KSW == 1) ? (int)blockIdx.x * KS_WARPS + w : (int)blockIdx.x;
  const int e = chunk * 32 + (threadIdx.x & 31);
  const size_t MM = (size_t)M * M;
  const double* Xj = Xblk + (size_t)j * MM;
  double acc = 0.0;
  if (KSW == 1) {
    if (e >= M * M) return;
    if (!first) {
      const int r = e % M, col = e / M;
      const double* Lr = Sold + (size_t)j * MM + r;
      const double* Rc = Xj + (size_t)col * M;
#pragma unroll 4
      for (int p = 0; p < M; ++p) acc = fma(Lr[(size_t)p * M], Rc[p], acc);
    }
  } else {
    if (!first) acc = ks_product(Sold + (size_t)j * MM, Xj, M, e, red);  // uniform branch: whole CTA
    if (w != 0 || e >= M * M) return;
  }
  const int r = e % M, col = e / M;
  if (first) {
    if (j == a) acc = Xj[(size_t)col * M + r] * scale;
    if (j + 1 == a && col == M - 1 && r == 0) acc += scale * gam[j];
  } else {
    acc *= scale;
    if (col == M - 1 && j < a) acc = fma(Sold[(size_t)(j + 1) * MM + r], scale * gam[j], acc);
  }
  acc *= kinv;
  if (j == a && r == col) acc += 1.0;
  Snew[(size_t)j * MM + e] = acc;
}

// Squaring for block row a: N[j] = sum_{l=j}^{a} G[a][l] G[l][j], blocks of
// the lower triangle stored row-major by (row, col) pairs.
__global__ void exp_square_kernel(const double* __restrict__ Gi, double* __restrict__ Go, int M, int a,
                                  int64_t sgm) {
  Gi += sgm * blockIdx.z;  // problem blockIdx.z of a batch (stride 0 for one problem)
  Go += sgm * blockIdx.z;
  const int j = blockIdx.y;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (j > a || e >= M * M) return;
  const int r = e % M, col = e / M;
  const size_t MM = (size_t)M * M;
  const size_t rowa = (size_t)a * (a + 1) / 2;
  double a4[4] = {0.0, 0.0, 0.0, 0.0};  // four independent chains
  for (int l = j; l <= a; ++l) {
    const double* L = Gi + (rowa + l) * MM;                      // G[a][l]
    const double* Rb = Gi + ((size_t)l * (l + 1) / 2 + j) * MM;  // G[l][j]
    int p = 0;
    for (; p + 3 < M; p += 4)
#pragma unroll
      for (int u = 0; u < 4; ++u) a4[u] = fma(L[(size_t)(p + u) * M + r], Rb[(size_t)col * M + p + u], a4[u]);
    for (; p < M; ++p) a4[0] = fma(L[(size_t)p * M + r], Rb[(size_t)col * M + p], a4[0]);
  }
  Go[(rowa + j) * MM + e] = (a4[0] + a4[1]) + (a4[2] + a4[3]);
}

// The same squaring for one problem with the whole inner sum of an output
// block spread over the warps of a CTA: the flattened index (l - j) m + p over
// the (a - j + 1) m terms of N[j] is cut into SQ_WARPS contiguous ranges, one
// per warp, and warp 0 adds the partial sums in warp order (deterministic).
// One CTA per (j, 32 consecutive entries): the dependent chain of a warp is at
// most (a + 1) m / SQ_WARPS terms and the grid holds every block of the row.
constexpr int SQ_WARPS = 8;

//
// phi_1 (gi non-null): grid row a + 1 squares the augmented matrix's extra
// column as well, [[E, g], [0, 1]]^2 = [[E^2, E g + g], [0, 1]]: block row a
// of the new vector is sum_{l <= a} G[a][l] g[l] + g[a], the same flattened
// (l, p) sum split over the warps (g[l]: the m-vector of block row l at the
// input level, gi; output go).
//
// dbl (cos(t sqrt(z))): the double-angle step C(4A) = 2 C(A)^2 - I instead of
// a plain square: the block sum is doubled and the identity subtracted on the
// diagonal block.
// MODE: SQ_EXP (squaring), SQ_PHI (squaring and the phi_1 vector row),
// SQ_COS (double-angle step); a template parameter, so the squaring of the
// exponential carries no branch for the other two.
enum : int { SQ_EXP = 0, SQ_PHI = 1, SQ_COS = 2 };

template <int MODE>
__global__ void __launch_bounds__(SQ_WARPS * 32) exp_square_row_kernel(const double* __restrict__ Gi,
                                                                     double* __restrict__ Go, int M, int a,
                                                                     const double* __restrict__ gi,
                                                                     double* __restrict__ go) {
  __shared__ double red[SQ_WARPS][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int j = blockIdx.y;
  const int e = blockIdx.x * 32 + lane;
  const size_t MM = (size_t)M * M;
  const size_t rowa = (size_t)a * (a + 1) / 2;
  if (MODE == SQ_PHI && j == a + 1) {  // the phi_1 vector of block row a
    if ((int)blockIdx.x * 32 >= M) return;  // whole CTA
    const int K = (a + 1) * M;
    const int chunk = (K + SQ_WARPS - 1) / SQ_WARPS;
    const int k0 = w * chunk, k1 = min(K, k0 + chunk);
    double acc = 0.0;
    if (e < M) {
      int k = k0;
      while (k < k1) {  // one (l, p-range) segment at a time
        const int l = k / M, p0 = k % M, p1 = min(M, p0 + (k1 - k));
        const double* L = Gi + (rowa + l) * MM + e;  // G[a][l], row e
        const double* gl = gi + (size_t)l * M;
        for (int p = p0; p < p1; ++p) acc = fma(L[(size_t)p * M], gl[p], acc);
        k += p1 - p0;
      }
    }
    red[w][lane] = acc;
    __syncthreads();
    if (w == 0 && e < M) {
      double sum = red[0][lane];
#pragma unroll
      for (int q = 1; q < SQ_WARPS; ++q) sum += red[q][lane];
      go[(size_t)a * M + e] = sum + gi[(size_t)a * M + e];
    }
    return;
  }
  const int K = (a - j + 1) * M;
  const int chunk = (K + SQ_WARPS - 1) / SQ_WARPS;
  const int k0 = w * chunk, k1 = min(K, k0 + chunk);
  double acc = 0.0;
  if (e < M * M && k0 < k1) {
    const int r = e % M, col = e / M;
    int k = k0;
    while (k < k1) {  // one (l, p-range) segment at a time
      const int l = j + k / M, p0 = k % M, p1 = min(M, p0 + (k1 - k));
      const double* L = Gi + (rowa + l) * MM + r;                         // G[a][l], row r
      const double* Rb = Gi + ((size_t)l * (l + 1) / 2 + j) * MM + (size_t)col * M;  // G[l][j], column col
#pragma unroll 4
      for (int p = p0; p < p1; ++p) acc = fma(L[(size_t)p * M], Rb[p], acc);
      k += p1 - p0;
    }
  }
  red[w][lane] = acc;
  __syncthreads();
  if (w == 0 && e < M * M) {
    double sum = red[0][lane];
#pragma unroll
    for (int q = 1; q < SQ_WARPS; ++q) sum += red[q][lane];
    if (MODE == SQ_COS) {
      sum *= 2.0;
      if (j == a && e % M == e / M) sum -= 1.0;
    }
    Go[(rowa + j) * MM + e] = sum;
  }
}

// f(z) = 1/z: y_a = X_a^{-1} rhs, rhs = e_1 (a = 0) or -gamma_{a-1} y_{a-1}[M-1] e_1
// (block forward substitution on the block lower-bidiagonal H).  X_a is me x me
// (me < M only in a cycle that ended in breakdown).  LU with partial pivoting in
// one CTA on a scratch copy of X_a + sigma I (sigma = 0 here).
__device__ void shifted_block_solve(const double* __restrict__ X, int M, int me, double sigma, double rhs0,
                                    double* work, double* y, int* s_piv) {
  const int tid = threadIdx.x;
  for (int e = tid; e < me * me; e += blockDim.x) {
    const int r = e % me, c = e / me;
    work[e] = X[(size_t)c * M + r] + (r == c ? sigma : 0.0);
  }
  for (int r = tid; r < me; r += blockDim.x) y[r] = (r == 0) ? rhs0 : 0.0;
  __syncthreads();
  for (int c = 0; c < me; ++c) {
    if (tid < 32) {  // pivot: largest |entry| of column c at or below the diagonal (ties: first row)
      double best = -1.0;
      int p = c;
      for (int r = c + tid; r < me; r += 32) {
        const double v = fabs(work[(size_t)c * me + r]);
        if (v > best) {
          best = v;
          p = r;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, p, o);
        if (ob > best || (ob == best && op < p)) {
          best = ob;
          p = op;
        }
      }
      if (tid == 0) *s_piv = p;
    }
    __syncthreads();
    const int p = *s_piv;
    if (p != c) {
      for (int l = tid; l < me; l += blockDim.x) {
        const double tmp = work[(size_t)l * me + c];
        work[(size_t)l * me + c] = work[(size_t)l * me + p];
        work[(size_t)l * me + p] = tmp;
      }
      if (tid == 0) {
        const double ty = y[c];
        y[c] = y[p];
        y[p] = ty;
      }
    }
    __syncthreads();
    const double d = work[(size_t)c * me + c];
    for (int r = c + 1 + tid; r < me; r += blockDim.x) {
      const double f = work[(size_t)c * me + r] / d;
      for (int l = c + 1; l < me; ++l)
        work[(size_t)l * me + r] = fma(-f, work[(size_t)l * me + c], work[(size_t)l * me + r]);
      y[r] = fma(-f, y[c], y[r]);
    }
    __syncthreads();
  }
  for (int c = me - 1; c >= 0; --c) {  // back substitution, column by column
    if (tid == 0) y[c] = y[c] / work[(size_t)c * me + c];
    __syncthreads();
    const double yc = y[c];
    for (int r = tid; r < c; r += blockDim.x) y[r] = fma(-work[(size_t)c * me + r], yc, y[r]);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(SMALL_THREADS) inv_block_kernel(SmallDev sd, int M, int me, int a, double* work) {
  __shared__ double y[256];
  __shared__ int piv;
  const double rhs0 = (a == 0) ? 1.0 : -sd.gam[a - 1] * sd.misc[5];
  shifted_block_solve(sd.Xblk + (size_t)a * M * M, M, me, 0.0, rhs0, work, y, &piv);
  if (threadIdx.x == 0) sd.misc[5] = y[me - 1];
  for (int r = threadIdx.x; r < me; r += blockDim.x) sd.fcol[r] = y[r];
}

// f(z) = z^{-1/2}.  Substituting s = e^u in the Stieltjes form
//   z^{-1/2} = (2/pi) int_0^inf (z + s^2)^{-1} ds = (2/pi) int_R e^u (z + e^{2u})^{-1} du,
// the trapezoidal rule with step hq at u_i = u0 + i hq converges geometrically for z
// off the closed negative real axis (the integrand is analytic in the strip
// |Im u| < (pi - |arg z|) / 2).  So the first column of H^{-1/2} is a weighted sum of
// the first columns of (H + sigma_i I)^{-1}, sigma_i = e^{2 u_i}, each found block by
// block exactly as for 1/z: block a solves (X_a + sigma_i I) y = rhs_i with
// rhs_i = e_1 (a = 0) or -gamma_{a-1} carry_i e_1, carry_i = last entry of node i's
// y in block a - 1.  One CTA per node; the work matrix is in shared memory when it
// fits (glob = 0), else in the node's slice of sd.qwork.
constexpr int QN_THREADS = 128;
__global__ void __launch_bounds__(QN_THREADS) invsqrt_nodes_kernel(SmallDev sd, int M, int me, int a, double u0,
                                                                      double hq, int glob) {
  extern __shared__ double qs[];
  __shared__ int piv;
  const int i = blockIdx.x;
  double* y = qs;
  double* work = glob ? sd.qwork + (size_t)i * M * M : qs + 256;
  const double u = u0 + hq * i;
  const double rhs0 = (a == 0) ? 1.0 : -sd.gam[a - 1] * sd.qcarry[i];
  shifted_block_solve(sd.Xblk + (size_t)a * M * M, M, me, exp(2.0 * u), rhs0, work, y, &piv);
  const double w = (2.0 * hq / 3.14159265358979323846) * exp(u);
  for (int r = threadIdx.x; r < me; r += blockDim.x) sd.qpart[(size_t)i * M + r] = w * y[r];
  if (threadIdx.x == 0) sd.qcarry[i] = y[me - 1];
}

// fcol[r] = sum over nodes of qpart[i][r], in node order.
__global__ void invsqrt_sum_kernel(SmallDev sd, CycleDev cd, int M, int me, int nodes) {
  for (int r = threadIdx.x; r < me; r += blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < nodes; ++i) acc += sd.qpart[(size_t)i * M + r];
    sd.fcol[r] = acc;
    if (!isfinite(acc)) atomicOr(&cd.flags[2], ERR_NONFINITE);
  }
}

// f(z) = exp(-t z) with a cost per cycle that does not grow with the cycle
// count: the exponential as a resolvent integral,
//   e^w = (1 / 2 pi i) int_Gamma e^zeta (zeta - w)^{-1} d zeta,
// Gamma winding once around the spectrum of w = -t (H - sigma I), discretized by
// the midpoint rule on two contours published for e^w with w on (-inf, 0]
// (Trefethen, Weideman and Schmelzer, BIT 46, 2006):
//   parabolic   zeta(th) = N (0.1309 - 0.1194 th^2 + 0.2500 i th),
//   hyperbolic  zeta(th) = 2.246 N (1 - sin(1.1721 - 0.3443 i th)),
// N = EQ_N points th_k = -pi + (k - 1/2) h, h = 2 pi / N.  For a real matrix and
// vector the points come in conjugate pairs, so the K = N / 2 points with
// th > 0 give e^w v = (h / pi) sum_k Im(e^{zeta_k} zeta'(th_k) (zeta_k - w)^{-1} v).
// (zeta_k I + t (H - sigma I))^{-1} e_1 is found block by block on the block
// lower-bidiagonal H exactly as for 1/z: block a solves
// ((zeta_k - t sigma) I + t X_a) y = rhs, rhs = e_1 (a = 0) or
// -t gamma_{a-1} carry_k e_1 with carry_k the last entry of point k's solution
// in block a - 1, so a cycle costs 2 K complex m x m LU factorizations and the
// state kept across cycles is one complex number per point.  The shift sigma
// (fixed in the first cycle) brings the largest e^w near 1, so the quadrature's
// absolute error is relative to the result.  The two contours enclose
// different regions; their results agree only when both enclose the spectrum,
// which the host checks every cycle before using the result.
constexpr int EQ_N = 32;
constexpr int EQ_K = EQ_N / 2;  // points per contour used (th > 0)

struct cplx {
  double re, im;
};
__device__ __forceinline__ cplx cmul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
  const double d = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

// point k of contour c: zeta and zeta'(th)
__device__ __forceinline__ void eq_point(int c, int k, cplx* z, cplx* dz) {
  const double h = 2.0 * 3.14159265358979323846 / EQ_N;
  const double th = (k + 0.5) * h;
  if (c == 0) {
    *z = {EQ_N * (0.1309 - 0.1194 * th * th), EQ_N * 0.25 * th};
    *dz = {EQ_N * (-2.0 * 0.1194 * th), EQ_N * 0.25};
  } else {
    // sin(u - i v) = sin u cosh v - i cos u sinh v, cos(u - i v) = cos u cosh v + i sin u sinh v
    const double u = 1.1721, v = 0.3443 * th, A = 2.246 * EQ_N;
    const double su = sin(u), cu = cos(u), chv = cosh(v), shv = sinh(v);
    *z = {A * (1.0 - su * chv), A * (cu * shv)};
    // d/dth [A (1 - sin(u - i 0.3443 th))] = A * 0.3443 i * cos(u - i v)
    const cplx cs{cu * chv, su * shv};
    *dz = cmul({0.0, A * 0.3443}, cs);
  }
}

constexpr int EQ_THREADS = 128;
__global__ void __launch_bounds__(EQ_THREADS) exp_quad_nodes_kernel(SmallDev sd, int M, int me, int a, double t,
                                                                   int glob) {
  extern __shared__ double qs[];
  __shared__ int piv;
  const int node = blockIdx.x;  // contour node / EQ_K, point node % EQ_K
  const int tid = threadIdx.x;
  cplx z, dz;
  eq_point(node / EQ_K, node % EQ_K, &z, &dz);
  const double sigma = sd.qstat[0];
  const cplx shift{z.re - t * sigma, z.im};
  cplx* y = reinterpret_cast<cplx*>(qs);
  cplx* work = glob ? reinterpret_cast<cplx*>(sd.qwork) + (size_t)node * M * M : y + 256;
  const double* X = sd.Xblk + (size_t)a * M * M;
  cplx rhs0{1.0, 0.0};
  if (a > 0) {
    const double g = -t * sd.gam[a - 1];
    rhs0 = {g * sd.qcarry[2 * node], g * sd.qcarry[2 * node + 1]};
  }
  for (int e = tid; e < me * me; e += blockDim.x) {
    const int r = e % me, c = e / me;
    work[e] = {t * X[(size_t)c * M + r] + (r == c ? shift.re : 0.0), r == c ? shift.im : 0.0};
  }
  for (int r = tid; r < me; r += blockDim.x) y[r] = (r == 0) ? rhs0 : cplx{0.0, 0.0};
  __syncthreads();
  for (int c = 0; c < me; ++c) {  // LU with partial pivoting (|re| + |im|; ties: first row)
    if (tid < 32) {
      double best = -1.0;
      int p = c;
      for (int r = c + tid; r < me; r += 32) {
        const cplx v = work[(size_t)c * me + r];
        const double m1 = fabs(v.re) + fabs(v.im);
        if (m1 > best) {
          best = m1;
          p = r;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, p, o);
        if (ob > best || (ob == best && op < p)) {
          best = ob;
          p = op;
        }
      }
      if (tid == 0) piv = p;
    }
    __syncthreads();
    const int p = piv;
    if (p != c) {
      for (int l = tid; l < me; l += blockDim.x) {
        const cplx tmp = work[(size_t)l * me + c];
        work[(size_t)l * me + c] = work[(size_t)l * me + p];
        work[(size_t)l * me + p] = tmp;
      }
      if (tid == 0) {
        const cplx ty = y[c];
        y[c] = y[p];
        y[p] = ty;
      }
    }
    __syncthreads();
    const cplx d = work[(size_t)c * me + c];
    for (int r = c + 1 + tid; r < me; r += blockDim.x) {  // multipliers in place of column c
      const cplx f = cdiv(work[(size_t)c * me + r], d);
      work[(size_t)c * me + r] = f;
      const cplx u = cmul(f, y[c]);
      y[r].re -= u.re;
      y[r].im -= u.im;
    }
    __syncthreads();
    const int w = me - c - 1;  // trailing (w x w) update, every thread on it
    for (int e = tid; e < w * w; e += blockDim.x) {
      const int r = c + 1 + e % w, l = c + 1 + e / w;
      const cplx u = cmul(work[(size_t)c * me + r], work[(size_t)l * me + c]);
      work[(size_t)l * me + r].re -= u.re;
      work[(size_t)l * me + r].im -= u.im;
    }
    __syncthreads();
  }
  for (int c = me - 1; c >= 0; --c) {  // back substitution
    if (tid == 0) y[c] = cdiv(y[c], work[(size_t)c * me + c]);
    __syncthreads();
    const cplx yc = y[c];
    for (int r = tid; r < c; r += blockDim.x) {
      const cplx u = cmul(work[(size_t)c * me + r], yc);
      y[r].re -= u.re;
      y[r].im -= u.im;
    }
    __syncthreads();
  }
  // weight (h / pi) e^zeta zeta'
  const double h = 2.0 * 3.14159265358979323846 / EQ_N;
  const double ez = exp(z.re) * (h / 3.14159265358979323846);
  const cplx w = cmul({ez * cos(z.im), ez * sin(z.im)}, dz);
  for (int r = tid; r < me; r += blockDim.x) sd.qpart[(size_t)node * M + r] = cmul(w, y[r]).im;
  if (tid == 0) {
    sd.qcarry[2 * node] = y[me - 1].re;
    sd.qcarry[2 * node + 1] = y[me - 1].im;
  }
}

// fcol = e^{-t sigma} (sum over the parabolic contour's points, in point
// order); qstat[3] = max |difference to the hyperbolic contour's sum| and
// qstat[2] = max |difference to fsq| (when given: the block row of the
// scaling-and-squaring evaluation), both relative to the largest |entry| of
// the first column met so far (qstat[1]) and kept as running maxima until the
// host clears them.
__global__ void exp_quad_sum_kernel(SmallDev sd, CycleDev cd, int M, int me, double t, const double* fsq) {
  __shared__ double s_d[3][256];
  const double E = exp(-t * sd.qstat[0]);
  double dq = 0.0, dsq = 0.0, mx = 0.0;
  for (int r = threadIdx.x; r < me; r += blockDim.x) {
    double f1 = 0.0, f2 = 0.0;
    for (int k = 0; k < EQ_K; ++k) {
      f1 += sd.qpart[(size_t)k * M + r];
      f2 += sd.qpart[(size_t)(EQ_K + k) * M + r];
    }
    f1 *= E;
    f2 *= E;
    sd.fcol[r] = f1;
    if (!isfinite(f1)) atomicOr(&cd.flags[2], ERR_NONFINITE);
    dq = fmax(dq, fabs(f1 - f2));
    mx = fmax(mx, fabs(f1));
    if (fsq) {
      dsq = fmax(dsq, fabs(f1 - fsq[r]));
      mx = fmax(mx, fabs(fsq[r]));
    }
  }
  s_d[0][threadIdx.x] = dq;
  s_d[1][threadIdx.x] = dsq;
  s_d[2][threadIdx.x] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)blockDim.x; ++i) {
      dq = fmax(dq, s_d[0][i]);
      dsq = fmax(dsq, s_d[1][i]);
      mx = fmax(mx, s_d[2][i]);
    }
    const double scale = fmax(sd.qstat[1], mx);
    sd.qstat[1] = scale;
    // running maxima over the blocks since the host last cleared them
    sd.qstat[2] = fmax(sd.qstat[2], (scale > 0.0) ? dsq / scale : INFINITY);
    sd.qstat[3] = fmax(sd.qstat[3], (scale > 0.0 && isfinite(dq)) ? dq / scale : INFINITY);
  }
}

// sigma from the first cycle's block of the scaling-and-squaring evaluation:
// ||f_1|| ~ e^{-t lambda_min} for the smallest real eigenvalue lambda_min the
// first column meets; sigma = (-ln ||f_1|| - 2) / t puts the largest w near
// -2 plus ln(1 / (the weight of that eigenvector in e_1)): inside both
// contours (their rightmost points are 4.19 and 5.66) for weights down to
// e^-5, and the result within e^2 of the largest contour term.
__global__ void exp_quad_sigma_kernel(SmallDev sd, int me, double t, const double* fsq) {
  if (threadIdx.x == 0) {
    double nrm = 0.0;
    for (int r = 0; r < me; ++r) nrm = fma(fsq[r], fsq[r], nrm);
    nrm = sqrt(nrm);
    sd.qstat[0] = (nrm > 0.0 && isfinite(nrm)) ? (-log(nrm) - 2.0) / t : 0.0;
    sd.qstat[1] = 0.0;
  }
}

__global__ void z_kernel(SmallDev sd, int M, int me, const double* fsrc, const BatchStride bs, int64_t fstride) {
  sd = offset_sd(sd, bs, blockIdx.x);  // problem blockIdx.x of a batch
  fsrc += fstride * blockIdx.x;
  const double beta = sd.misc[0];
  for (int a = threadIdx.x; a < me; a += blockDim.x) {
    double acc = 0.0;
    for (int l = a; l < me; ++l) acc = fma(sd.Tinv[(size_t)l * M + a], fsrc[l], acc);
    sd.zg[a] = beta * acc;
  }
}

}  // namespace

namespace {

// Largest cluster (16, 8, 4, 2 or 1 CTAs) the device schedules for the
// cluster whitening at the largest shared-memory footprint it is given, and
// the SM count; found once per device.
struct WcDevice {
  int cl_max = 1;
  int sms = 1;
};

WcDevice whiten_cluster_device() {
  static std::mutex mu;
  static std::map<int, WcDevice> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return WcDevice{};
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  WcDevice d;
  cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
  const void* kern = (const void*)whiten_cluster_kernel;
  if (raise_smem_limit(kern, WC_SMEM_MAX) == cudaSuccess &&
      cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    for (int cl = 16; cl >= 2; cl >>= 1) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(cl);
      cfg.blockDim = dim3(WC_THREADS);
      cfg.dynamicSmemBytes = WC_SMEM_MAX;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = cl;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n > 0) {
        d.cl_max = cl;
        break;
      }
    }
  }
  cudaGetLastError();  // a refused size leaves no error behind
  cache[dev] = d;
  return d;
}

// Cluster whitening of nb problems (one cluster each): the cluster size is
// the device's largest, cut to about (SM count / problems) when many problems
// run at once (nb in this launch times `concurrent` such launches on other
// streams).  Returns false (nothing launched) when the shared-memory
// footprint does not fit; the single-CTA kernel then runs.
bool launch_whiten_cluster(const SmallDev& sd, const CycleDev& cd, const BatchStride& bs, int nb, int concurrent,
                           int s, int m, int ncols, int m_eff, int has_next, int cycle, int kw, double t,
                           cudaStream_t st) {
  const WcDevice d = whiten_cluster_device();
  int cl = d.cl_max;
  const int target = std::max(1, d.sms / std::max(nb * std::max(concurrent, 1), 1));
  while (cl > 1 && cl > target) cl >>= 1;
  const size_t smem = whiten_cluster_smem(s, ncols, cl);
  if (smem > WC_SMEM_MAX) return false;
  if (raise_smem_limit((const void*)whiten_cluster_kernel, smem) != cudaSuccess) return false;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nb * cl));
  cfg.blockDim = dim3(WC_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  // T_m R_m goes to the Horner buffer area (not in use at this point)
  return cudaLaunchKernelEx(&cfg, whiten_cluster_kernel, sd, cd, s, m, ncols, m_eff, has_next, cycle, kw, t, sd.S0,
                            bs) == cudaSuccess;
}

}  // namespace

void launch_whiten(const SmallDev& sd, const CycleDev& cd, int s, int m, int ncols, int m_eff, int has_next,
                   int cycle, int kw, double t, cudaStream_t st) {
  if (launch_whiten_cluster(sd, cd, BatchStride{}, 1, 1, s, m, ncols, m_eff, has_next, cycle, kw, t, st)) return;
  // scratch for T_m R_m: reuse the Horner buffer area (not in use at this point)
  const size_t smem = whiten_smem(s, ncols);
  raise_smem_limit((const void*)whiten_kernel, smem);
  whiten_kernel<<<1, SMALL_THREADS, smem, st>>>(sd, cd, s, m, ncols, m_eff, has_next, cycle, t, sd.S0,
                                                BatchStride{});
}

void launch_whiten_batched(const SmallDev& sd, const CycleDev& cd, const BatchStride& bs, int nb, int concurrent,
                           int s, int m, int ncols, int m_eff, int has_next, int cycle, int kw, double t,
                           cudaStream_t st) {
  if (launch_whiten_cluster(sd, cd, bs, nb, concurrent, s, m, ncols, m_eff, has_next, cycle, kw, t, st)) return;
  const size_t smem = whiten_smem(s, ncols);
  raise_smem_limit((const void*)whiten_kernel, smem);
  whiten_kernel<<<nb, SMALL_THREADS, smem, st>>>(sd, cd, s, m, ncols, m_eff, has_next, cycle, t, sd.S0, bs);
}

void launch_exp_taylor_batched(const SmallDev& sd, const BatchStride& bs, int nb, int m, int a, int kdeg,
                               double scale, int first, int src, double* dst0, int dst_in_g, cudaStream_t st) {
  const int MM = m * m;
  dim3 g((MM + KS_THREADS - 1) / KS_THREADS, a + 1, nb);
  const double* Sold = sd.S0 + (size_t)src * (size_t)(a + 1) * MM;
  // dst0 lies in problem 0's Horner buffer or (last step) its exp rows
  exp_taylor_kernel<1><<<g, KS_THREADS, 0, st>>>(sd.Xblk, sd.gam, m, a, 1.0 / kdeg, scale, first, Sold, dst0, bs.Xblk, bs.gam,
                                       bs.S0, dst_in_g ? bs.G : bs.S0, nullptr, 0.0);
}

void launch_exp_square_batched(const SmallDev& sd, const BatchStride& bs, int nb, int m, int a, int level,
                               int64_t level_stride, cudaStream_t st) {
  const int MM = m * m;
  dim3 g((MM + 127) / 128, a + 1, nb);
  exp_square_kernel<<<g, 128, 0, st>>>(sd.G + (size_t)level * level_stride, sd.G + (size_t)(level + 1) * level_stride,
                                      m, a, bs.G);
}

void launch_z_batched(const SmallDev& sd, const BatchStride& bs, int nb, int m, int m_eff, const double* fcol0,
                      int64_t fcol_stride, cudaStream_t st) {
  z_kernel<<<nb, 256, 0, st>>>(sd, m, m_eff, fcol0, bs, fcol_stride);
}

void launch_exp_taylor_step(const SmallDev& sd, int m, int a, double kinv, double scale, int first, int last,
                            int src, double* dst, double* gout, double gscale, cudaStream_t st) {
  const int MM = m * m;
  dim3 g((MM + 31) / 32, a + 1);
  const double* Sold = sd.S0 + (size_t)src * (size_t)(a + 1) * MM;
  exp_taylor_kernel<KS_WARPS><<<g, KS_THREADS, 0, st>>>(sd.Xblk, sd.gam, m, a, kinv, scale, first, Sold, dst, 0, 0,
                                                         0, 0, (last && !first) ? gout : nullptr, gscale);
}

void launch_exp_square(const SmallDev& sd, int m, int a, int level, int64_t level_stride, const double* gi,
                       double* go, int dbl, cudaStream_t st) {
  const int MM = m * m;
  const double* Gi = sd.G + (size_t)level * level_stride;
  double* Go = sd.G + (size_t)(level + 1) * level_stride;
  const dim3 block(SQ_WARPS * 32);
  if (gi != nullptr)
    exp_square_row_kernel<SQ_PHI><<<dim3((MM + 31) / 32, a + 2), block, 0, st>>>(Gi, Go, m, a, gi, go);
  else if (dbl)
    exp_square_row_kernel<SQ_COS><<<dim3((MM + 31) / 32, a + 1), block, 0, st>>>(Gi, Go, m, a, nullptr, nullptr);
  else
    exp_square_row_kernel<SQ_EXP><<<dim3((MM + 31) / 32, a + 1), block, 0, st>>>(Gi, Go, m, a, nullptr, nullptr);
}

void launch_inv_block(const SmallDev& sd, int m, int m_eff, int a, cudaStream_t st) {
  inv_block_kernel<<<1, SMALL_THREADS, 0, st>>>(sd, m, m_eff, a, sd.S0);
}

size_t invsqrt_smem(int m) {
  const size_t b = (size_t)(256 + (size_t)m * m) * sizeof(double);
  return b <= INVSQRT_SMEM_MAX ? b : (size_t)256 * sizeof(double);
}

void launch_invsqrt_block(const SmallDev& sd, const CycleDev& cd, int m, int m_eff, int a, double u0, double hq,
                          int nodes, cudaStream_t st) {
  const size_t smem = invsqrt_smem(m);
  const int glob = (smem == (size_t)256 * sizeof(double)) ? 1 : 0;
  raise_smem_limit((const void*)invsqrt_nodes_kernel, smem);
  invsqrt_nodes_kernel<<<nodes, QN_THREADS, smem, st>>>(sd, m, m_eff, a, u0, hq, glob);
  invsqrt_sum_kernel<<<1, 256, 0, st>>>(sd, cd, m, m_eff, nodes);
}

size_t exp_quad_smem(int m) {
  const size_t b = (size_t)(256 + (size_t)m * m) * 2 * sizeof(double);
  return b <= EXP_QUAD_SMEM_MAX ? b : (size_t)256 * 2 * sizeof(double);
}

int exp_quad_nodes() { return 2 * EQ_K; }

void launch_exp_quad_sigma(const SmallDev& sd, int m_eff, double t, const double* fsq, cudaStream_t st) {
  exp_quad_sigma_kernel<<<1, 32, 0, st>>>(sd, m_eff, t, fsq);
}

void launch_exp_quad(const SmallDev& sd, const CycleDev& cd, int m, int m_eff, int a, double t, const double* fsq,
                     cudaStream_t st) {
  const size_t smem = exp_quad_smem(m);
  const int glob = (smem == (size_t)256 * 2 * sizeof(double)) ? 1 : 0;
  raise_smem_limit((const void*)exp_quad_nodes_kernel, smem);
  exp_quad_nodes_kernel<<<2 * EQ_K, EQ_THREADS, smem, st>>>(sd, m, m_eff, a, t, glob);
  exp_quad_sum_kernel<<<1, 256, 0, st>>>(sd, cd, m, m_eff, t, fsq);
}

void launch_z(const SmallDev& sd, int m, int m_eff, const double* fcol_src, cudaStream_t st) {
  z_kernel<<<1, 256, 0, st>>>(sd, m, m_eff, fcol_src, BatchStride{}, 0);
}

}  // namespace krylov
