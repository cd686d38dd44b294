// api.cu -- the C ABI (include/krylov.h): handle management and the host
// driver of Algorithm 2 (restart cycles) on top of the kernels.
//
// Per cycle the host launches m+1 step kernels, the sketch reduction, the
// whitening kernel and the projected-function kernels, then the streaming
// update.  It synchronizes twice per cycle: once to read m_eff, the breakdown
// flag and the norm of the new projected block (to fix the number of
// squarings), once to read ||y|| and ||x|| for the stopping test of Sec. 4.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/krylov.h"
#include "internal.h"
#include "kernels.cuh"

using namespace krylov;

namespace {

constexpr double EXP_THETA = 0.5;  // ||B||_1 bound after scaling
// cos(t sqrt(z)): Taylor degree 14 in A = t^2 H / 4^s with ||A||_1 <= 4: the
// first omitted term is below 4^15 / 30! = 4e-24
constexpr int COS_TAYLOR_DEG = 14;
constexpr double COS_THETA = 4.0;
// Column-index and value arrays get CSR_PAD zeroed elements past nnz so the
// step kernels can read them in aligned 16-byte chunks.
constexpr size_t CSR_PAD = 8;
// row_ptr gets RP_PAD zeroed entries past n+1: staged row_ptr slices of a
// 256-row tile are copied as 260 entries.
constexpr size_t RP_PAD = 272;
constexpr int TMA_MAX_CAP = 4096;  // largest staged tile span (nonzeros)
#ifndef KRYLOV_SELL
#define KRYLOV_SELL 1  // build the sliced layout for the float-float product where it applies
#endif
constexpr int EXP_SQ_CYCLES = 16;              // exp: cycles also evaluated by scaling and squaring
constexpr double QUAD_TOL_CONTOURS = 1e-12;    // exp quadrature: largest difference of the two contours
constexpr double QUAD_TOL_SQUARING = 1e-11;    // ... and to scaling and squaring (relative to the first column)
constexpr int QUAD_RETRIES = 2;                // lower shifts tried after a failed check
constexpr int QUAD_START = 10;                 // first cycle with the quadrature (shorter runs never pay for it)
// z^{-1/2}: trapezoidal nodes in u (s = e^u) with step INVSQRT_H on
// [0.5 ln(alpha * 1e-18) - 38, 0.5 ln(alpha * 1e4) + 38], alpha = ||A||_inf >= |lambda|:
// the two tails are below e^-38 relative for spectra inside [1e-18 alpha, 1e4 alpha], and
// the step gives geometric accuracy exp(-2 pi d / h) with d = (pi - |arg z|) / 2.
constexpr double INVSQRT_H = 0.2;
constexpr int EXP_TAYLOR_DEG = 14; // theta^15/15! e^theta = 3.9e-17 < 2^-53 (each Taylor step is one launch
                                    // per block row, a squaring level one more: 14 steps + 2 levels beat 24 steps)

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

namespace {

// Segment plan of an operator (see ff_spmv_seg_kernel): device arrays and caps.
struct SegPlan {
  int4* seg = nullptr;
  int* seg_n = nullptr;
  uint16_t* lcol = nullptr;
  int seg_cap = 0;
  int lcap = 0;
};

// Rows with more nonzeros than this go to the long-row product kernel
// (power-law operators with the float-float basis): a row per thread would
// leave one thread with a hub's tens of thousands of nonzeros.  48 keeps the
// emptied operator's 256-row tiles within the staged kernel's span on the
// R-MAT graphs (the largest tile: 3512 nonzeros at 2^20 nodes).  Long rows
// with more than LONG_ROW_CTA nonzeros take a CTA each, the others a warp.
constexpr int LONG_ROW = 48;
constexpr int LONG_ROW_CTA = 1024;

struct LongRows {
  int n_long = 0;
  int n_big = 0;            // the first n_big rows have more than LONG_ROW_CTA nonzeros
  int* rows = nullptr;      // [n_long] longest first
  int* rp = nullptr;        // the operator with these rows emptied
  int* ci = nullptr;
  float* val32 = nullptr;
  float2* valff = nullptr;
  int tma_cap = 0;          // staged span per tile of the emptied operator (0: no staging)
  int grid = 0;             // CTAs of the long-row kernel
  double* part = nullptr;   // [grid][8] its scalar partials
};

// Host construction of a segment plan from a host CSR: per 256-row tile the
// sorted distinct columns are cut into pieces wherever two consecutive columns
// are more than SEG_GAP apart; each piece is widened to an even start and an
// even length (16-byte copies of float-float entries) and placed after the
// previous one.  Returns false when some tile needs more than SEG_MAX pieces
// or SEG_CAP_MAX staged entries (the operator then keeps the gather kernel).
bool build_seg_plan(int n, int64_t nnz, const int* rp, const int* ci, std::vector<int4>& seg, std::vector<int>& segn,
                    std::vector<uint16_t>& lcol, int& seg_cap, int& lcap) {
  const int ntiles = (n + STEP_THREADS - 1) / STEP_THREADS;
  seg.assign((size_t)ntiles * SEG_MAX, make_int4(0, 0, 0, 0));
  segn.assign((size_t)ntiles, 0);
  lcol.assign((size_t)nnz + 16, 0);
  std::atomic<bool> ok{true};
  std::atomic<int> cap_w{0}, cap_l{0};
  auto work = [&](int t0, int t1) {
    std::vector<int> cols, starts, ends;
    int my_w = 0, my_l = 0;
    for (int t = t0; t < t1 && ok.load(std::memory_order_relaxed); ++t) {
      const int ts = t * STEP_THREADS, te = std::min(n, ts + STEP_THREADS);
      const int e0 = rp[ts], e1 = rp[te];
      my_l = std::max(my_l, ((e1 + 7) & ~7) - (e0 & ~7));
      cols.assign(ci + e0, ci + e1);
      std::sort(cols.begin(), cols.end());
      cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
      starts.clear();
      ends.clear();
      for (int c : cols) {
        if (starts.empty() || c > ends.back() + SEG_GAP) {
          starts.push_back(c);
          ends.push_back(c);
        } else {
          ends.back() = c;
        }
      }
      if ((int)starts.size() > SEG_MAX) {
        ok = false;
        break;
      }
      int off = 0;
      for (size_t q = 0; q < starts.size(); ++q) {
        const int a = starts[q] & ~1;
        const int len = ((ends[q] + 1 - a) + 1) & ~1;
        seg[(size_t)t * SEG_MAX + q] = make_int4(a, len, off, 0);
        starts[q] = a;
        off += len;
      }
      if (off > SEG_CAP_MAX) {
        ok = false;
        break;
      }
      my_w = std::max(my_w, off);
      segn[(size_t)t] = (int)starts.size();
      for (int e = e0; e < e1; ++e) {
        const int c = ci[e];
        const int q = (int)(std::upper_bound(starts.begin(), starts.end(), c) - starts.begin()) - 1;
        const int4 sg = seg[(size_t)t * SEG_MAX + q];
        lcol[(size_t)e] = (uint16_t)(sg.z + (c - sg.x));
      }
    }
    int w = cap_w.load();
    while (my_w > w && !cap_w.compare_exchange_weak(w, my_w)) {
    }
    int l = cap_l.load();
    while (my_l > l && !cap_l.compare_exchange_weak(l, my_l)) {
    }
  };
  const int nth = std::max(1, std::min(16, (int)std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  const int per = (ntiles + nth - 1) / nth;
  for (int w = 0; w < nth; ++w) {
    const int t0 = w * per, t1 = std::min(ntiles, t0 + per);
    if (t0 < t1) pool.emplace_back(work, t0, t1);
  }
  for (auto& th : pool) th.join();
  seg_cap = cap_w.load();
  lcap = std::max(8, cap_l.load());
  return ok.load();
}

struct BlockWs;

}  // namespace

struct krylov_handle {
  int n = 0;
  int64_t nnz = 0;
  int m = 0, k = 0, s = 0;
  uint64_t seed = 0;
  krylov_func f{};
  krylov_options opt{};
  cudaStream_t st = nullptr;
  int num_sms = 0;
  int device = 0;
  int grid = 0;                    // CTAs of the step kernels (one resident wave)
  int grid_spmv = 0, grid_spmv_t = 0;  // CTAs of the float-float product kernel for A, A^T

  // matrix (and its transpose, built on first adjoint use)
  int* rp = nullptr;
  int* ci = nullptr;
  double* val = nullptr;
  float* val32 = nullptr;
  float2* valff = nullptr;  // (hi, lo) value pairs for the float-float basis
  int vals_exact_f32 = 0;
  int part_cap = 0;                // per-CTA partial slots (8 doubles each)
  double* part_w = nullptr;        // [2][part_cap] ||w_j||^2 partials of the float-float materialize kernels
  int grid_mat = 0;                // CTAs of the float-float materialize kernel with staged row streams
  int sell_maxl = 0;               // longest tile row of the sliced layout
  void* sk_acc = nullptr;          // (m+1) x sk_acc_stride int64: exact sketches of the float-float basis
  int64_t sk_acc_stride = 0;
  long long* rgs_acc = nullptr;    // randomized Gram-Schmidt: exact sketch sums [3][s]
  BlockWs* bk = nullptr;           // block form workspace (allocated on first use)
  int bk_concurrent = 1;           // instances running concurrently in the current batched call
  int grid_update = 0;             // CTAs of the cycle-end update pass
  int q_nodes = 0;                 // z^{-1/2} quadrature nodes
  double q_u0 = 0.0;               // first node
  int tma_cap = 0, tma_cap_t = 0;  // staged span per tile for A and A^T (0: no staging)
  int16_t* dcol = nullptr;         // col - row per nonzero of A (bandwidth < 2^15, staged float-float product)
  int* sell_off = nullptr;         // sliced layout of A (float-float product; null: not built)
  int16_t* sell_col = nullptr;
  void* sell_val = nullptr;
  int grid_sell = 0;
  int16_t* dcolt = nullptr;        // the same for A^T
  SegPlan seg_a, seg_t;            // segment plans of A and A^T (float-float basis)
  LongRows long_a, long_t;         // long rows of A and A^T (float-float basis, power-law operators)
  int* rpt = nullptr;
  int* cit = nullptr;
  double* valt = nullptr;
  float* valt32 = nullptr;
  float2* valtff = nullptr;
  int have_t = 0;

  // cycle workspaces
  void* W = nullptr;
  int64_t ldw = 0;
  void* p[2] = {nullptr, nullptr};
  void* sk_part = nullptr;
  int64_t sk_col_stride = 0;
  double* part = nullptr;
  CycleDev cd{};
  SmallDev sd{};
  int cap_rows = 0;     // block rows of the projected-problem storage (X blocks, couplings)
  int cap_grows = 0;    // block rows of the exponential's scale levels in sd.G
  int cap_levels = 0;   // scale levels allocated in sd.G
  int64_t gphi_stride = 0;  // phi_1 vectors: doubles per scale level in sd.gphi
  int64_t level_stride = 0;
  int* d_flag = nullptr;
  double* d_dot = nullptr;
  double* stage_b = nullptr;  // device staging of krylov_apply_host
  double* stage_x = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // step phase, small problem
  // the m + 1 step launches of a cycle for A (0) and A^T (1), captured once
  // (their arguments do not change between cycles or calls) and replayed
  cudaGraphExec_t step_graph[2] = {nullptr, nullptr};
  int step_runs[2] = {0, 0};
  cudaStream_t cap_stream = nullptr;  // private stream the graphs are captured on
  SketchTable sk_tab{};
  int sk_mode = SK_TAB8;
  int sk_copies = 32;

  // row-partitioned solve (krylov_create_partition); part_mode == 0 otherwise
  int part_mode = 0;
  int staged32 = 0;  // float32 / bfloat16 basis: staged two-kernel step (forward operator)
  int n_halo = 0, n_send = 0;
  int64_t row0 = 0, n_global = 0;
  krylov_comm comm{};
  int* send_idx = nullptr;         // device, n_send local rows to send
  double* sendbuf = nullptr;       // device, n_send
  double* recvbuf = nullptr;       // device, n_halo
  double* red = nullptr;           // device, NQ + 1 all-reduced step sums
  long long* part_acc = nullptr;   // device, [m+1][3][s] exact sketch word sums
  int* part_E = nullptr;           // device, [m+1] fixed-point exponents
  int part_grid = 0, part_rows = 0, part_wb = 0;

  // host mirrors
  int* h_flags = nullptr;     // pinned: flags[4]
  double* h_scal = nullptr;   // pinned: 32 doubles ([0, 8) cycle scalars, [8, 16) misc, [16, 24) quadrature)
  int last_me = 0, last_nc = 0, last_cycle = 0;
  std::vector<void*> allocs;
};

namespace {

int basis_bytes(int basis) { return (basis == 0 || basis == 3) ? 8 : (basis == 1 ? 4 : 2); }
int wide(int basis) { return basis == 0 || basis == 3; }

krylov_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return KRYLOV_OK;
  if (e == cudaErrorMemoryAllocation) return KRYLOV_ENOMEM;
  return KRYLOV_ECUDA;
}

#define CK(call)                                          \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_status(e_);        \
  } while (0)

// Two timing events, destroyed on every path out of the scope that made them
// (the calls below return early on errors).
struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  EventPair() = default;
  EventPair(const EventPair&) = delete;
  EventPair& operator=(const EventPair&) = delete;
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
  cudaError_t create() {
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    return e;
  }
};

// An NVTX range (visible to profilers that attach; a no-op otherwise).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Consecutive NVTX ranges inside one scope: next() closes the open one and
// opens the next; the last one closes with the scope.
struct NvtxPhase {
  bool open = false;
  NvtxPhase() = default;
  NvtxPhase(const NvtxPhase&) = delete;
  NvtxPhase& operator=(const NvtxPhase&) = delete;
  void next(const char* name) {
    if (open) nvtxRangePop();
    nvtxRangePushA(name);
    open = true;
  }
  ~NvtxPhase() {
    if (open) nvtxRangePop();
  }
};

template <typename T>
cudaError_t dalloc(krylov_handle* h, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  h->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return cudaSuccess;
}

void dfree(krylov_handle* h, void* p) {
  if (!p) return;
  for (auto& q : h->allocs)
    if (q == p) {
      cudaFree(q);
      q = nullptr;
    }
}

// Projected-function storage for `rows` block rows and `levels` scale levels.
// Storage of the projected problem: X blocks and couplings for `rows` cycles,
// and the scale levels of the exponential's block rows (sd.G) for `grows`
// rows (grows < 0: as many as rows).  Reallocating G discards its rows; the
// caller recomputes them from the X blocks.
krylov_status ensure_small_capacity(krylov_handle* h, int rows, int levels, int grows = -1) {
  const size_t MM = (size_t)h->m * h->m;
  if (grows < 0) grows = rows;
  if (rows > h->cap_rows) {
    int nr = std::max(rows, std::max(8, 2 * h->cap_rows));
    dfree(h, h->sd.Xblk);
    dfree(h, h->sd.gam);
    dfree(h, h->sd.S0);
    CK(dalloc(h, &h->sd.Xblk, (size_t)nr * MM));
    CK(dalloc(h, &h->sd.gam, (size_t)nr));
    CK(dalloc(h, &h->sd.S0, std::max<size_t>(2 * (size_t)nr * MM, (size_t)h->m * h->m)));
    h->cap_rows = nr;
  }
  grows = std::min(grows, h->cap_rows);
  if (grows > h->cap_grows || levels > h->cap_levels || h->sd.G == nullptr) {
    const int ng = std::max(grows, h->cap_grows);
    const int nl = (levels > h->cap_levels) ? std::max(levels, h->cap_levels + 4) : h->cap_levels;
    dfree(h, h->sd.G);
    h->sd.G = nullptr;
    h->level_stride = (int64_t)ng * (ng + 1) / 2 * (int64_t)MM;
    CK(dalloc(h, &h->sd.G, (size_t)nl * h->level_stride));
    if (h->f.kind == KRYLOV_F_PHI1_NEG) {  // the augmented column: one m-vector per block row and level
      dfree(h, h->sd.gphi);
      h->gphi_stride = (int64_t)ng * h->m;
      CK(dalloc(h, &h->sd.gphi, (size_t)nl * h->gphi_stride));
    }
    h->cap_grows = ng;
    h->cap_levels = nl;
  }
  return KRYLOV_OK;
}

int scale_levels_for(double normH) {
  if (!(normH > EXP_THETA)) return 0;
  return (int)std::ceil(std::log2(normH / EXP_THETA));
}

// cos(t sqrt(H)): double-angle steps s with ||t^2 H|| / 4^s <= COS_THETA
int cos_levels_for(double normA) {
  if (!(normA > COS_THETA)) return 0;
  return (int)std::ceil(0.5 * std::log2(normA / COS_THETA));
}

// Block row a of exp(-t H) at all scale levels 0..sl (scale 2^-sl).
// Returns the number of kernels launched.
int exp_row(krylov_handle* h, int a, int sl) {
  const int M = h->m;
  const size_t MM = (size_t)M * M;
  // exp(-tH) and phi_1(-tH): B = -t H / 2^sl, Taylor-Horner S <- S B / k + I,
  // squarings.  cos(t sqrt(H)): B = -t^2 H / 4^sl, S <- S B / ((2k-1) 2k) + I
  // (the series of cos(sqrt(A)) in Horner form), double-angle steps.
  const bool cosm = (h->f.kind == KRYLOV_F_COS_SQRT);
  const int q = cosm ? COS_TAYLOR_DEG : EXP_TAYLOR_DEG;
  const double scale = cosm ? -(h->f.t * h->f.t) / std::ldexp(1.0, 2 * sl) : -h->f.t / std::ldexp(1.0, sl);
  double* g0row = h->sd.G + (size_t)a * (a + 1) / 2 * MM;
  int src = 0;
  // phi_1: the extra column of exp([[-tH, e_1], [0, 0]]) rides along (level 0
  // from the Taylor steps, then one vector row per squaring)
  const bool phi = (h->f.kind == KRYLOV_F_PHI1_NEG);
  auto gvec = [&](int lv) { return h->sd.gphi + (size_t)lv * h->gphi_stride; };
  for (int kdeg = q; kdeg >= 1; --kdeg) {
    const int first = (kdeg == q);
    const double kinv = cosm ? 1.0 / ((2.0 * kdeg - 1.0) * (2.0 * kdeg)) : 1.0 / kdeg;
    double* dst = (kdeg == 1) ? g0row : h->sd.S0 + (size_t)(1 - src) * (size_t)(a + 1) * MM;
    launch_exp_taylor_step(h->sd, M, a, kinv, scale, first, kdeg == 1, src, dst,
                           phi ? gvec(0) + (size_t)a * M : nullptr, std::ldexp(1.0, -sl), h->st);
    src = 1 - src;
  }
  for (int lv = 0; lv < sl; ++lv)
    launch_exp_square(h->sd, M, a, lv, h->level_stride, phi ? gvec(lv) : nullptr, phi ? gvec(lv + 1) : nullptr,
                      cosm ? 1 : 0, h->st);
  return q + sl;
}

struct Operator {
  const int* rp;
  const int* ci;
  const double* val;
  const float* val32;
  const float2* valff;
};

// Build the segment plan of an operator held on the device (copied to the
// host for the construction) and upload it; no plan when a tile does not fit.
krylov_status install_seg_plan(krylov_handle* h, SegPlan& plan, const int* rp_dev, const int* ci_dev) {
  std::vector<int> rp((size_t)h->n + 1), ci((size_t)std::max<int64_t>(h->nnz, 1));
  CK(cudaStreamSynchronize(h->st));
  CK(cudaMemcpy(rp.data(), rp_dev, sizeof(int) * rp.size(), cudaMemcpyDeviceToHost));
  if (h->nnz > 0) CK(cudaMemcpy(ci.data(), ci_dev, sizeof(int) * (size_t)h->nnz, cudaMemcpyDeviceToHost));
  std::vector<int4> seg;
  std::vector<int> segn;
  std::vector<uint16_t> lcol;
  int seg_cap = 0, lcap = 0;
  if (!build_seg_plan(h->n, h->nnz, rp.data(), ci.data(), seg, segn, lcol, seg_cap, lcap)) return KRYLOV_OK;
  CK(dalloc(h, &plan.seg, seg.size()));
  CK(dalloc(h, &plan.seg_n, segn.size()));
  CK(dalloc(h, &plan.lcol, lcol.size()));
  CK(cudaMemcpy(plan.seg, seg.data(), sizeof(int4) * seg.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(plan.seg_n, segn.data(), sizeof(int) * segn.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(plan.lcol, lcol.data(), sizeof(uint16_t) * lcol.size(), cudaMemcpyHostToDevice));
  plan.seg_cap = std::max(seg_cap, 2);
  plan.lcap = lcap;
  return KRYLOV_OK;
}

krylov_status choose_product_kernel(krylov_handle* h, int transpose);

// Column offsets col - row as 2-byte integers for the staged float-float
// product kernel, when every |col - row| fits (banded operators: stencils and
// meshes in a banded ordering); they replace the 4-byte column indices in
// its copies.  Null otherwise.
krylov_status install_delta16(krylov_handle* h, const int* rp_dev, const int* ci_dev, int16_t** out) {
  *out = nullptr;
  if ((h->opt.basis_dtype != 3 && !h->staged32) || h->nnz == 0) return KRYLOV_OK;
  CK(csr_bandwidth(h->n, rp_dev, ci_dev, h->d_flag, h->h_flags, h->st));
  if (h->h_flags[0] > 32767) return KRYLOV_OK;
  int16_t* d = nullptr;
  CK(dalloc(h, &d, (size_t)h->nnz + CSR_PAD));
  CK(cudaMemsetAsync(d + h->nnz, 0, CSR_PAD * sizeof(int16_t), h->st));
  CK(csr_delta16(h->n, rp_dev, ci_dev, d, h->st));
  *out = d;
  return KRYLOV_OK;
}

// Sliced layout of A for the float-float product kernel (ff_spmv_sell_kernel):
// every 256-row tile padded to its longest row and stored slot-major.  Built
// when the band allows 2-byte offsets, no tile has a row longer than
// SELL_MAXL and the padding adds at most a quarter to the stored entries
// (stencils and meshes; power-law operators keep the CSR kernels).
krylov_status install_sell(krylov_handle* h, int use32) {
  if ((h->opt.basis_dtype != 3 && !h->staged32) || h->long_a.n_long > 0 || h->dcol == nullptr || h->nnz == 0)
    return KRYLOV_OK;
  const int n = h->n;
  const int64_t nnz = h->nnz;
  std::vector<int> rp((size_t)n + 1), ci((size_t)nnz);
  CK(cudaStreamSynchronize(h->st));
  CK(cudaMemcpy(rp.data(), h->rp, sizeof(int) * rp.size(), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(ci.data(), h->ci, sizeof(int) * (size_t)nnz, cudaMemcpyDeviceToHost));
  const int ntiles = (n + STEP_THREADS - 1) / STEP_THREADS;
  std::vector<int> off((size_t)ntiles + 1, 0);
  int64_t total = 0;
  int maxl = 1;
  for (int g = 0; g < ntiles; ++g) {
    int lmax = 0;
    for (int r = g * STEP_THREADS; r < std::min(n, (g + 1) * STEP_THREADS); ++r) lmax = std::max(lmax, rp[r + 1] - rp[r]);
    if (lmax > SELL_MAXL) return KRYLOV_OK;
    maxl = std::max(maxl, lmax);
    total += (int64_t)lmax * STEP_THREADS;
    if (total > 0x7FFFFFF0LL) return KRYLOV_OK;
    off[(size_t)g + 1] = (int)total;
  }
  if ((double)total > 1.25 * (double)nnz) return KRYLOV_OK;
  // the float-float product kernel stages several tiles of the longest row
  if (!h->staged32 && sell_smem_bytes(use32, maxl) > 220 * 1024) return KRYLOV_OK;
  const size_t vb = use32 ? sizeof(float) : sizeof(float2);
  std::vector<unsigned char> vsrc((size_t)nnz * vb), vdst((size_t)total * vb, 0);
  CK(cudaMemcpy(vsrc.data(), use32 ? (const void*)h->val32 : (const void*)h->valff, vsrc.size(),
                cudaMemcpyDeviceToHost));
  std::vector<int16_t> col((size_t)total, 0);
  for (int r = 0; r < n; ++r) {
    const int g = r / STEP_THREADS, k = r % STEP_THREADS;
    for (int q = 0; q < rp[r + 1] - rp[r]; ++q) {
      const size_t e = (size_t)off[g] + (size_t)q * STEP_THREADS + k;
      const int src = rp[r] + q;
      col[e] = (int16_t)(ci[src] - r);
      std::memcpy(vdst.data() + e * vb, vsrc.data() + (size_t)src * vb, vb);
    }
  }
  int16_t* dc = nullptr;
  unsigned char* dv = nullptr;
  CK(dalloc(h, &h->sell_off, off.size()));
  CK(dalloc(h, &dc, (size_t)total));
  CK(dalloc(h, &dv, (size_t)total * vb));
  CK(cudaMemcpy(h->sell_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dc, col.data(), sizeof(int16_t) * col.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dv, vdst.data(), vdst.size(), cudaMemcpyHostToDevice));
  h->sell_col = dc;
  h->sell_val = dv;
  h->sell_maxl = maxl;
  const int per_sm = h->staged32 ? s32_sell_ctas_per_sm() : sell_ctas_per_sm(use32, maxl);
  h->grid_sell = std::max(1, std::min(h->num_sms * per_sm, std::min(h->part_cap, (n + STEP_THREADS - 1) / STEP_THREADS)));
  return KRYLOV_OK;
}

// Long rows of an operator held on the device: if any row has more than
// LONG_ROW nonzeros (float-float basis), build the operator with those rows
// emptied (same row count, so every other kernel keeps its layout), the list
// of long rows (longest first), the staged span of the emptied operator's
// tiles and the long-row kernel's grid and partials.
krylov_status install_long_rows(krylov_handle* h, LongRows& lr, const int* rp_dev, const int* ci_dev,
                                const float* v32_dev, const float2* vff_dev) {
  lr = LongRows{};
  if (h->opt.basis_dtype != 3 || h->nnz == 0) return KRYLOV_OK;
  const int n = h->n;
  const size_t nnz = (size_t)h->nnz;
  std::vector<int> rp((size_t)n + 1);
  CK(cudaStreamSynchronize(h->st));
  CK(cudaMemcpy(rp.data(), rp_dev, sizeof(int) * rp.size(), cudaMemcpyDeviceToHost));
  std::vector<int> longs;
  for (int i = 0; i < n; ++i)
    if (rp[(size_t)i + 1] - rp[i] > LONG_ROW) longs.push_back(i);
  if (longs.empty()) return KRYLOV_OK;
  std::stable_sort(longs.begin(), longs.end(),
                   [&](int a, int b) { return rp[(size_t)a + 1] - rp[a] > rp[(size_t)b + 1] - rp[b]; });
  std::vector<char> is_long((size_t)n, 0);
  for (int i : longs) is_long[i] = 1;
  std::vector<int> ci(nnz);
  CK(cudaMemcpy(ci.data(), ci_dev, sizeof(int) * nnz, cudaMemcpyDeviceToHost));
  std::vector<float> v32(v32_dev ? nnz : 0);
  std::vector<float2> vff(vff_dev ? nnz : 0);
  if (v32_dev) CK(cudaMemcpy(v32.data(), v32_dev, sizeof(float) * nnz, cudaMemcpyDeviceToHost));
  if (vff_dev) CK(cudaMemcpy(vff.data(), vff_dev, sizeof(float2) * nnz, cudaMemcpyDeviceToHost));
  std::vector<int> rps((size_t)n + 1 + RP_PAD, 0);
  std::vector<int> cis;
  std::vector<float> v32s;
  std::vector<float2> vffs;
  cis.reserve(nnz);
  for (int i = 0; i < n; ++i) {
    if (!is_long[i]) {
      for (int e = rp[i]; e < rp[(size_t)i + 1]; ++e) {
        cis.push_back(ci[e]);
        if (v32_dev) v32s.push_back(v32[e]);
        if (vff_dev) vffs.push_back(vff[e]);
      }
    }
    rps[(size_t)i + 1] = (int)cis.size();
  }
  for (size_t q = 0; q < CSR_PAD; ++q) {
    cis.push_back(0);
    if (v32_dev) v32s.push_back(0.f);
    if (vff_dev) vffs.push_back(make_float2(0.f, 0.f));
  }
  lr.n_long = (int)longs.size();
  while (lr.n_big < lr.n_long && rp[(size_t)longs[lr.n_big] + 1] - rp[longs[lr.n_big]] > LONG_ROW_CTA) ++lr.n_big;
  CK(dalloc(h, &lr.rows, longs.size()));
  CK(dalloc(h, &lr.rp, rps.size()));
  CK(dalloc(h, &lr.ci, cis.size()));
  CK(cudaMemcpy(lr.rows, longs.data(), sizeof(int) * longs.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(lr.rp, rps.data(), sizeof(int) * rps.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(lr.ci, cis.data(), sizeof(int) * cis.size(), cudaMemcpyHostToDevice));
  if (v32_dev) {
    CK(dalloc(h, &lr.val32, v32s.size()));
    CK(cudaMemcpy(lr.val32, v32s.data(), sizeof(float) * v32s.size(), cudaMemcpyHostToDevice));
  }
  if (vff_dev) {
    CK(dalloc(h, &lr.valff, vffs.size()));
    CK(cudaMemcpy(lr.valff, vffs.data(), sizeof(float2) * vffs.size(), cudaMemcpyHostToDevice));
  }
  CK(tile_span_max(n, lr.rp, h->d_flag, h->h_flags, h->st));
  lr.tma_cap = (h->h_flags[0] <= TMA_MAX_CAP) ? std::max(h->h_flags[0], 8) : 0;
  lr.grid = std::max(1, std::min(std::max(lr.n_big, (lr.n_long + 7) / 8), h->num_sms * 8));
  CK(dalloc(h, &lr.part, (size_t)lr.grid * 8));
  return KRYLOV_OK;
}

krylov_status build_transpose(krylov_handle* h) {
  if (h->have_t) return KRYLOV_OK;
  int* work = nullptr;
  CK(dalloc(h, &h->rpt, (size_t)h->n + 1 + RP_PAD));
  CK(cudaMemsetAsync(h->rpt + h->n + 1, 0, RP_PAD * sizeof(int), h->st));
  CK(dalloc(h, &h->cit, (size_t)h->nnz + CSR_PAD));
  CK(cudaMemsetAsync(h->cit + h->nnz, 0, CSR_PAD * sizeof(int), h->st));
  CK(dalloc(h, &h->valt, (size_t)h->nnz + CSR_PAD));
  CK(cudaMemsetAsync(h->valt + h->nnz, 0, CSR_PAD * sizeof(double), h->st));
  CK(dalloc(h, &work, 2 * (size_t)h->n));
  CK(transpose_csr(h->n, h->nnz, h->rp, h->ci, h->val, h->rpt, h->cit, h->valt, work, h->st));
  if (h->val32) {
    CK(dalloc(h, &h->valt32, (size_t)h->nnz + CSR_PAD));
    CK(cudaMemsetAsync(h->valt32 + h->nnz, 0, CSR_PAD * sizeof(float), h->st));
    CK(narrow_values(h->nnz, h->valt, h->valt32, h->d_flag, h->h_flags, h->st));
  }
  if (h->valff) {
    CK(dalloc(h, &h->valtff, (size_t)h->nnz + CSR_PAD));
    CK(cudaMemsetAsync(h->valtff + h->nnz, 0, CSR_PAD * sizeof(float2), h->st));
    CK(split_values(h->nnz, h->valt, h->valtff, h->st));
  }
  CK(cudaStreamSynchronize(h->st));
  dfree(h, work);
  CK(tile_span_max(h->n, h->rpt, h->d_flag, h->h_flags, h->st));
  h->tma_cap_t = (h->h_flags[0] <= TMA_MAX_CAP) ? std::max(h->h_flags[0], 8) : 0;
  if (h->opt.basis_dtype == 3) {
    const int vals32 = h->vals_exact_f32 && h->opt.narrow_values_if_exact;
    krylov_status ps = install_long_rows(h, h->long_t, h->rpt, h->cit, h->valt32, h->valtff);
    if (ps != KRYLOV_OK) return ps;
    if (h->long_t.n_long == 0) {  // plans describe the full operator
      ps = install_seg_plan(h, h->seg_t, h->rpt, h->cit);
      if (ps != KRYLOV_OK) return ps;
      ps = install_delta16(h, h->rpt, h->cit, &h->dcolt);
      if (ps != KRYLOV_OK) return ps;
    }
    const SegPlan& sp = h->seg_t;
    const int tcap = h->long_t.n_long ? h->long_t.tma_cap : h->tma_cap_t;
    h->grid_spmv_t = std::max(1, std::min(h->num_sms * spmv_ctas_per_sm(vals32, tcap, sp.seg ? sp.seg_cap : 0,
                                                                        sp.lcap),
                                          std::min(h->part_cap, (h->n + STEP_THREADS - 1) / STEP_THREADS)));
  }
  h->have_t = 1;
  {
    const krylov_status cs = choose_product_kernel(h, 1);
    if (cs != KRYLOV_OK) return cs;
  }
  return KRYLOV_OK;
}

double model_bytes_step(const krylov_handle* h, int use32) {
  const double bv = basis_bytes(h->opt.basis_dtype);
  const double ba = use32 ? 4.0 : 8.0;
  // the lower bound of the roofline model: A read once with 4-byte column
  // indices (also when the product kernel streams 2-byte offsets instead),
  // the current vector and the k-1 other window vectors read once, the new
  // vector written once
  return (double)h->nnz * (ba + 4.0) + 4.0 * (h->n + 1) + (h->k + 1) * (double)h->n * bv;
}

// Randomized Gram-Schmidt step j: read A and w_j, write p; the sketch reads p
// and S's table (9 bytes per column); the materialization reads p and the
// window (min(j + 1, k) vectors) and writes w_{j+1}.
double model_bytes_rgs_step(const krylov_handle* h, int use32, int j) {
  const double bv = basis_bytes(h->opt.basis_dtype);
  const double ba = use32 ? 4.0 : 8.0;
  const double n = (double)h->n;
  const int nwin = std::min(j + 1, h->k);
  return (double)h->nnz * (ba + 4.0) + 4.0 * (n + 1) + n * bv + n * bv + (n * bv + 9.0 * n) +
         (n * bv + nwin * n * bv + n * bv);
}

// Arguments of the step launch for column j of a cycle (the same in every cycle).
StepLaunch step_args(const krylov_handle* h, const Operator& op, int transpose, int use32, double thr, int j) {
  const int n = h->n, M = h->m, basis = h->opt.basis_dtype;
  StepLaunch L{};
  L.n = n;
  L.row_ptr = op.rp;
  L.col = op.ci;
  L.val = use32 ? (const void*)op.val32 : (basis == 3 ? (const void*)op.valff : (const void*)op.val);
  L.val_f32 = use32;
  L.W = h->W;
  L.ldw = h->ldw;
  L.j = j;
  L.k = h->k;
  L.mat = (j > 0);
  L.spmv = (j < M);
  L.p_prev = h->p[(j + 1) & 1];
  L.p_out = h->p[j & 1];
  L.sk_part = (char*)h->sk_part + (size_t)j * h->sk_col_stride * sizeof(double);
  L.part = h->part;
  L.part_w = h->part_w;
  L.part_w_stride = h->part_cap;
  L.sk_acc = h->sk_acc;
  L.sk_acc_stride = h->sk_acc_stride;
  L.thr = thr;
  L.s = h->s;
  L.zeta = h->opt.zeta;
  L.seed = h->seed;
  L.grid = h->grid;
  L.grid_spmv = transpose ? h->grid_spmv_t : h->grid_spmv;
  L.rows_spmv = ((n + L.grid_spmv - 1) / L.grid_spmv + STEP_THREADS - 1) / STEP_THREADS * STEP_THREADS;
  // whole 256-row tiles per CTA (tiles then start at multiples of 256)
  L.rows_per_cta = ((n + h->grid - 1) / h->grid + STEP_THREADS - 1) / STEP_THREADS * STEP_THREADS;
  L.m = M;
  L.grid_mat = L.grid;
  L.rows_mat = L.rows_per_cta;
  if (basis == 3 && h->sk_mode == SK_TAB8 && h->grid_mat > 0) {
    L.grid_mat = h->grid_mat;
    L.rows_mat = ((n + h->grid_mat - 1) / h->grid_mat + STEP_THREADS - 1) / STEP_THREADS * STEP_THREADS;
  }
  // float32 / bfloat16: the staged kernels run on the forward operator only
  const int st32 = h->staged32 && !transpose;
  L.tma_cap = (basis == 3) ? (transpose ? h->tma_cap_t : h->tma_cap) : (st32 ? h->tma_cap : 0);
  L.dcol = (basis == 3) ? (transpose ? h->dcolt : h->dcol) : (st32 ? h->dcol : nullptr);
  if ((basis == 3 || st32) && !transpose && h->sell_col) {  // the sliced layout of A
    L.sell_off = h->sell_off;
    L.sell_col = h->sell_col;
    L.sell_val = h->sell_val;
    L.sell_maxl = h->sell_maxl;
  }
  if (basis == 3) {
    const SegPlan& sp = transpose ? h->seg_t : h->seg_a;
    L.seg = sp.seg;
    L.seg_n = sp.seg_n;
    L.lcol = sp.lcol;
    L.seg_cap = sp.seg_cap;
    L.lcap = sp.lcap;
  }
  if (basis == 3) {
    const LongRows& lr = transpose ? h->long_t : h->long_a;
    if (lr.n_long > 0) {  // the product runs on the emptied operator, then on the long rows
      L.rp_full = L.row_ptr;
      L.col_full = L.col;
      L.val_full = L.val;
      L.row_ptr = lr.rp;
      L.col = lr.ci;
      L.val = use32 ? (const void*)lr.val32 : (const void*)lr.valff;
      L.tma_cap = lr.tma_cap;
      L.dcol = nullptr;
      L.seg = nullptr;
      L.n_long = lr.n_long;
      L.n_big = lr.n_big;
      L.long_rows = lr.rows;
      L.grid_long = lr.grid;
      L.part_long = lr.part;
    }
  }
  L.sk_tab = h->sk_tab;
  L.sk_mode = h->sk_mode;
  L.sk_copies = h->sk_copies;
  L.fx_wb = sketch_word_bits(basis == 3 ? L.rows_mat : L.rows_per_cta, h->sk_copies);
  return L;
}

// The m steps of a randomized Gram-Schmidt cycle (Algorithm 1): sketch and
// normalize the start vector, then per column the product, the sketch-space
// orthogonalization and the materialization of the next column.  Returns the
// number of kernels launched.
int rgs_cycle_steps(krylov_handle* h, const Operator& op, int transpose, int use32, double thr, int cycle,
                    cudaStream_t st) {
  const int M = h->m, basis = h->opt.basis_dtype;
  RgsArgs a{};
  a.n = h->n;
  a.m = M;
  a.k = h->k;
  a.s = h->s;
  a.zeta = h->opt.zeta;
  a.grid = h->grid;
  a.rows_per_cta = ((h->n + h->grid - 1) / h->grid + STEP_THREADS - 1) / STEP_THREADS * STEP_THREADS;
  a.sk_mode = h->sk_mode;
  a.copies = h->sk_copies;
  a.fx_wb = sketch_word_bits(a.rows_per_cta, h->sk_copies);
  a.basis = basis;
  a.ldw = h->ldw;
  a.seed = h->seed;
  a.sk_tab = h->sk_tab;
  a.W = h->W;
  a.part = h->part;
  a.acc = h->rgs_acc;
  a.U = h->sd.U;
  a.misc = h->sd.misc;
  a.thr = thr;
  int launches = 0;
  launch_rgs_start(a, h->cd, cycle, st);
  launches += 2;
  for (int j = 0; j < M; ++j) {
    StepLaunch L = step_args(h, op, transpose, use32, thr, j);
    L.rgs = 1;
    L.spmv = 1;
    L.mat = 0;
    L.p_out = h->p[j & 1];
    if (basis == 3) {
      launch_ff_product(L, h->cd, st);
    } else {
      L.rows_per_cta = (h->n + h->grid - 1) / h->grid;
      launch_rgs_product_f64(L, h->cd, st);
    }
    launch_rgs_orth(a, h->cd, h->p[j & 1], j, st);
    launch_rgs_mat(a, h->cd, h->p[j & 1], j, st);
    launches += 3;
  }
  return launches;
}

// Autotuning of the float-float product kernel for one operator: time the
// kernel that stages the pieces of w_j in shared memory (segment plan) against
// the one that gathers w_j through L1/L2, a few launches each on zeroed
// vectors, and keep the faster (stencils with float32 values favour the
// gathers, wider rows with float-float values the staged pieces).
krylov_status choose_product_kernel(krylov_handle* h, int transpose) {
  SegPlan& sp = transpose ? h->seg_t : h->seg_a;
  int& grid = transpose ? h->grid_spmv_t : h->grid_spmv;
  if (h->opt.basis_dtype != 3 || !sp.seg || h->opt.autotune == 0) return KRYLOV_OK;
  const int use32 = (h->opt.narrow_values_if_exact && h->vals_exact_f32) ? 1 : 0;
  Operator op{transpose ? h->rpt : h->rp, transpose ? h->cit : h->ci, transpose ? h->valt : h->val,
              transpose ? h->valt32 : h->val32, transpose ? h->valtff : h->valff};
  const int n = h->n;
  const int tcap = transpose ? h->tma_cap_t : h->tma_cap;
  const int grid_seg = grid;
  // the alternative to the staged pieces: the sliced-layout kernel where it
  // was built, else the CSR gather kernel
  const int grid_gather =
      (!transpose && h->sell_col)
          ? h->grid_sell
          : std::max(1, std::min(h->num_sms * spmv_ctas_per_sm(use32, tcap, 0, 0),
                                 std::min(h->part_cap, (n + STEP_THREADS - 1) / STEP_THREADS)));
  if (h->opt.autotune == 2) {  // fixed choice: the gather kernel
    sp.seg = nullptr;
    grid = grid_gather;
    return KRYLOV_OK;
  }
  cudaStream_t st = h->st;
  CK(cudaMemsetAsync(h->W, 0, sizeof(float2) * 2 * (size_t)h->ldw, st));
  CK(cudaMemsetAsync(h->cd.flags, 0, 4 * sizeof(int), st));
  EventPair evp;
  CK(evp.create());
  cudaEvent_t e0 = evp.a, e1 = evp.b;
  auto time_variant = [&](bool seg) -> float {
    StepLaunch L = step_args(h, op, transpose, use32, 1e-12, 1);
    L.grid_spmv = seg ? grid_seg : grid_gather;
    L.rows_spmv = ((n + L.grid_spmv - 1) / L.grid_spmv + STEP_THREADS - 1) / STEP_THREADS * STEP_THREADS;
    if (!seg) L.seg = nullptr;
    for (int r = 0; r < 2; ++r) launch_ff_product(L, h->cd, st);
    cudaEventRecord(e0, st);
    for (int r = 0; r < 5; ++r) launch_ff_product(L, h->cd, st);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
  };
  // alternate the variants over a few rounds and keep each one's best time:
  // one round alone flips with the box's state; the segment plan must win by
  // a clear margin over the plain gather kernel to be kept
  float t_seg = 1e30f, t_gather = 1e30f;
  for (int round = 0; round < 3; ++round) {
    t_seg = std::min(t_seg, time_variant(true));
    t_gather = std::min(t_gather, time_variant(false));
  }
  CK(cudaGetLastError());
  if (!(t_seg < 0.97f * t_gather)) {
    sp.seg = nullptr;
    grid = grid_gather;
  }
  return KRYLOV_OK;
}

// ---- row-partitioned solve ---------------------------------------------------
constexpr int PART_NQ = 2 + MAX_WINDOW;  // step sums of the product: [1] ||p||^2, [2..] window dots

krylov_status comm_status(int rc) { return rc == 0 ? KRYLOV_OK : KRYLOV_ECUDA; }

// The m + 1 columns of a cycle on this rank's rows: for column j, the
// materialization (and its rows' share of ||w_j||^2 and of S w_j), the sum of
// ||w_j||^2 over ranks and its reducer; then, for j < m, the halo exchange of
// w_j, the product p_j = A w_j on the rank's rows with its shares of ||p_j||^2
// and of the window dots, their sum over ranks and the coefficient reducer.
// Every rank runs the same sequence of collective calls; a breakdown is seen
// by all ranks alike (the reducers act on the all-reduced sums), and the
// kernels of the columns after it return at once.
krylov_status part_cycle_steps(krylov_handle* h, double thr, cudaStream_t st) {
  const int M = h->m;
  const int64_t nacc = (int64_t)(M + 1) * 3 * h->s;
  CK(cudaMemsetAsync(h->part_acc, 0, sizeof(long long) * (size_t)nacc, st));
  StepLaunch L{};
  L.n = h->n;
  L.k = h->k;
  L.m = M;
  L.s = h->s;
  L.zeta = h->opt.zeta;
  L.seed = h->seed;
  L.thr = thr;
  L.sk_tab = h->sk_tab;
  L.sk_mode = h->sk_mode;
  L.sk_copies = 1;
  L.fx_wb = h->part_wb;
  L.rows_per_cta = h->part_rows;
  L.grid = h->part_grid;
  PartLaunch P{};
  P.n = h->n;
  P.rp = h->rp;
  P.ci = h->ci;
  P.val = h->val;
  P.W = static_cast<double*>(h->W);
  P.ldw = h->ldw;
  P.p = static_cast<double*>(h->p[0]);
  P.part = h->part;
  P.red = h->red;
  P.acc = h->part_acc;
  P.E = h->part_E;
  P.grid = h->part_grid;
  P.rows_per_cta = h->part_rows;
  krylov_status cs = KRYLOV_OK;
  for (int j = 0; j <= M; ++j) {
    L.j = j;
    launch_part_mat(P, L, h->cd, j > 0 ? 1 : 0, st);
    CK(cudaGetLastError());
    if ((cs = comm_status(h->comm.allreduce_sum_f64(h->comm.ctx, h->red + PART_NQ, 1, st))) != KRYLOV_OK) return cs;
    launch_part_reduce_mat(L, h->cd, h->red, j > 0 ? 1 : 0, st);
    if (j == M) break;
    double* Wj = P.W + (int64_t)j * P.ldw;
    launch_part_pack(Wj, h->send_idx, h->n_send, h->sendbuf, st);
    CK(cudaGetLastError());
    if ((cs = comm_status(h->comm.halo_exchange_f64(h->comm.ctx, h->sendbuf, h->recvbuf, st))) != KRYLOV_OK)
      return cs;
    launch_part_unpack(h->recvbuf, h->n_halo, Wj + h->n, st);
    launch_part_product(P, L, h->cd, st);
    CK(cudaGetLastError());
    if ((cs = comm_status(h->comm.allreduce_sum_f64(h->comm.ctx, h->red, PART_NQ, st))) != KRYLOV_OK) return cs;
    launch_part_reduce_product(L, h->cd, h->red, st);
  }
  CK(cudaGetLastError());
  return KRYLOV_OK;
}

krylov_status apply_core(krylov_handle* h, int transpose, const double* b, double* x, double tol,
                         int max_cycles, krylov_stats* stout) {
  if (!h || !b || !x || max_cycles < 1 || !(tol >= 0.0)) return KRYLOV_EINVAL;
  if (transpose) {
    krylov_status s = build_transpose(h);
    if (s != KRYLOV_OK) return s;
  }
  const int basis = h->opt.basis_dtype;
  // float32 matrix values: always for the float32/bfloat16 bases, and for the
  // wide bases only when the narrowing is lossless
  const int use32 = (basis == 1 || basis == 2) || (h->opt.narrow_values_if_exact && h->vals_exact_f32);
  Operator op{transpose ? h->rpt : h->rp, transpose ? h->cit : h->ci, transpose ? h->valt : h->val,
              transpose ? h->valt32 : h->val32, transpose ? h->valtff : h->valff};
  const int n = h->n, M = h->m;
  cudaStream_t st = h->st;
  krylov_stats stats{};
  NvtxRange call_range(transpose ? "krylov_apply_adjoint" : "krylov_apply");
  EventPair evp;
  CK(evp.create());
  cudaEvent_t e0 = evp.a, e1 = evp.b;
  CK(cudaEventRecord(e0, st));

  int levels_needed = 1;
  if (h->f.kind == KRYLOV_F_EXP_NEG || h->f.kind == KRYLOV_F_PHI1_NEG || h->f.kind == KRYLOV_F_COS_SQRT)
    levels_needed = std::max(1, h->cap_levels);
  // exp(-t z), t > 0: the contour quadrature runs from the first cycle; the
  // scaling-and-squaring block rows are formed in the first EXP_SQ_CYCLES
  // cycles (they validate the quadrature) and afterwards only if a check fails
  bool quad = (h->f.kind == KRYLOV_F_EXP_NEG && h->f.t > 0.0 && h->sd.qstat != nullptr && max_cycles > EXP_SQ_CYCLES);
  krylov_status cs =
      ensure_small_capacity(h, max_cycles, levels_needed, quad ? std::min(max_cycles, EXP_SQ_CYCLES) : max_cycles);
  if (cs != KRYLOV_OK) return cs;

  CK(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)n, st));
  CK(cudaMemsetAsync(h->cd.flags, 0, 4 * sizeof(int), st));
  CK(cudaMemsetAsync(h->sd.misc, 0, 8 * sizeof(double), st));
  launch_norm_b(b, n, h->part, h->grid, h->cd, st);
  stats.launches += 1;
  if (h->part_mode) {  // ||b||^2 over all ranks
    CK(cudaGetLastError());
    cs = comm_status(h->comm.allreduce_sum_f64(h->comm.ctx, h->cd.scal + 4, 1, st));
    if (cs != KRYLOV_OK) return cs;
    launch_part_norm_finish(h->cd, st);
    stats.launches += 1;
  }
  CK(cudaMemcpyAsync(h->h_scal, h->cd.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h->h_flags, h->cd.flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h->h_flags[2] & ERR_NONFINITE) return KRYLOV_ENONFINITE;
  if (h->h_scal[0] == 0.0) {  // b = 0: f(A) 0 = 0
    CK(cudaEventRecord(e1, st));
    CK(cudaEventSynchronize(e1));
    if (stout) *stout = stats;
    return KRYLOV_OK;
  }
  launch_start(basis, b, h->W, n, h->cd, h->grid, st);
  stats.launches += 1;

  // breakdown threshold: a few hundred units of the basis arithmetic's roundoff
  const double thr = (basis == 0) ? 1e-14 : (basis == 3 ? 1e-12 : 1e-6);
  int s_lv = -1;        // scale levels in use (exp)
  double maxX = 0.0, maxG = 0.0;
  krylov_status result = KRYLOV_NOT_CONVERGED;
  for (int c = 1; c <= max_cycles; ++c) {
    NvtxRange cycle_range("restart cycle");
    NvtxPhase phase;
    phase.next("arnoldi steps");
    // float-float and staged float32 / bfloat16 materialize kernels: column
    // 0's exact sketch starts from zero
    const bool ff_mat = (basis == 3 || (h->staged32 && !transpose)) && !(h->opt.ortho == KRYLOV_ORTHO_RGS) &&
                        !h->part_mode;
    launch_cycle_reset(h->cd, M, st, ff_mat ? h->sk_acc : nullptr, ff_mat ? 3 * h->s : 0);
    CK(cudaEventRecord(h->ev[0], st));
    const bool rgs = (h->opt.ortho == KRYLOV_ORTHO_RGS);
    if (rgs) {
      stats.launches += rgs_cycle_steps(h, op, transpose, use32, thr, c, st);
    }
    if (h->part_mode) {
      cs = part_cycle_steps(h, thr, st);
      if (cs != KRYLOV_OK) return cs;
      stats.launches += 5 * M + 2;
      stats.step_launches += 2 * M + 1;
    }
    // the first run is eager (it also raises the kernels' shared-memory
    // limits); later cycles replay a graph of the same launches
    const bool use_graph = !rgs && !h->part_mode && h->opt.use_graph && h->step_runs[transpose] > 0;
    if (use_graph && !h->step_graph[transpose]) {
      // captured on a private stream (the caller's may be the legacy default
      // stream, which cannot be captured); the graph is launched on st
      if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
      cudaGraph_t g = nullptr;
      CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
      for (int j = 0; j <= M; ++j)
        launch_step(basis, step_args(h, op, transpose, use32, thr, j), h->cd, M, h->cap_stream);
      const cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &g);
      cudaError_t ie = cudaErrorUnknown;
      if (ce == cudaSuccess) ie = cudaGraphInstantiate(&h->step_graph[transpose], g, 0);
      if (g) cudaGraphDestroy(g);
      if (ie != cudaSuccess) {  // no graph: the same launches stay eager
        h->step_graph[transpose] = nullptr;
        h->opt.use_graph = 0;
        (void)cudaGetLastError();
      }
    }
    if (rgs || h->part_mode) {
      // launched above
    } else if (use_graph && h->step_graph[transpose]) {
      CK(cudaGraphLaunch(h->step_graph[transpose], st));
    } else {
      for (int j = 0; j <= M; ++j) launch_step(basis, step_args(h, op, transpose, use32, thr, j), h->cd, M, st);
      h->step_runs[transpose] += 1;
    }
    CK(cudaEventRecord(h->ev[1], st));
    if (!rgs && !h->part_mode) {
      const bool two = (basis == 3) || (h->staged32 && !transpose);
      stats.launches += (two ? 2 * M + 1 : M + 1) + 1;
      stats.step_launches += (two ? 2 * M + 1 : M + 1);
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h->h_flags, h->cd.flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h->h_flags[2] & ERR_TIMEOUT) return KRYLOV_ETIMEOUT;
    if (h->h_flags[2] & ERR_NONFINITE) return KRYLOV_ENONFINITE;
    if (h->h_flags[2] & ERR_SKETCH) return KRYLOV_ECUDA;
    const int me = std::min(h->h_flags[0], M);
    const int brk = h->h_flags[1];
    if (me < 1) return KRYLOV_ENONFINITE;
    const int has_next = brk ? 0 : 1;
    const int nc = me + has_next;
    stats.steps += me;
    {
      float ms_s = 0.f;
      CK(cudaEventElapsedTime(&ms_s, h->ev[0], h->ev[1]));
      stats.ms_steps += ms_s;
      if (h->opt.ortho == KRYLOV_ORTHO_RGS) {
        for (int j = 0; j < me; ++j) stats.step_bytes += model_bytes_rgs_step(h, use32, j);
      } else {
        stats.step_bytes += me * model_bytes_step(h, use32);
      }
    }
    phase.next("small problem");
    CK(cudaEventRecord(h->ev[2], st));
    if (rgs) {
      launch_rgs_small(h->sd, h->cd, M, me, has_next, c, h->f.t, st);
      stats.launches += 1;
    } else {
      if (h->part_mode) {  // S W_{m+1}: the exact word sums of all ranks
        cs = comm_status(h->comm.allreduce_sum_i64(h->comm.ctx, reinterpret_cast<int64_t*>(h->part_acc),
                                                   (int64_t)nc * 3 * h->s, st));
        if (cs != KRYLOV_OK) return cs;
        launch_part_sketch_u(h->part_acc, h->part_E, nc, h->s, h->opt.zeta, h->part_wb, h->sd.U, st);
      } else if (basis == 3 || (h->staged32 && !transpose)) {  // exact sketches of the staged materialize kernels
        launch_sketch_finish(h->sk_acc, nc, h->s, h->sk_acc_stride, step_args(h, op, transpose, use32, thr, 0).fx_wb,
                             h->opt.zeta, h->sd.U, st);
      } else {
        launch_sketch_reduce(h->sk_part, nc, h->grid, h->s, h->opt.zeta, h->sk_col_stride, h->sd.U, st);
      }
      launch_whiten(h->sd, h->cd, h->s, M, nc, me, has_next, c, h->k, h->f.t, st);
      stats.launches += 2;
    }
    const int a = c - 1;
    if (h->f.kind == KRYLOV_F_EXP_NEG || h->f.kind == KRYLOV_F_PHI1_NEG || h->f.kind == KRYLOV_F_COS_SQRT) {
      CK(cudaMemcpyAsync(h->h_scal, h->sd.misc, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      maxX = std::max(maxX, h->h_scal[2]);
      maxG = std::max(maxG, h->h_scal[3]);
      stats.kappa_T_max = std::max(stats.kappa_T_max, h->h_scal[4]);
      if (!std::isfinite(maxX) || !std::isfinite(maxG)) return KRYLOV_ENONFINITE;
      // ||t X||_1 + |t gamma| bounds ||t H||_1; cos(t sqrt(H)) scales t^2 H
      const int need = (h->f.kind == KRYLOV_F_COS_SQRT) ? cos_levels_for(std::fabs(h->f.t) * (maxX + maxG))
                                                         : scale_levels_for(maxX + maxG);
      const size_t MM = (size_t)M * M;
      // exp: first column of block (a, 0); phi_1: block row a of the extra column
      auto square_row = [&]() -> const double* {
        return (h->f.kind == KRYLOV_F_PHI1_NEG)
                   ? h->sd.gphi + (size_t)s_lv * h->gphi_stride + (size_t)a * M
                   : h->sd.G + (size_t)s_lv * h->level_stride + (size_t)a * (a + 1) / 2 * MM;
      };
      // scaling and squaring of block row a (all earlier rows at a new scale)
      auto squaring = [&](bool all_rows) -> krylov_status {
        if (need > s_lv || all_rows) {
          s_lv = std::max(s_lv, need);
          const krylov_status c2 = ensure_small_capacity(h, max_cycles, s_lv + 1,
                                                         quad ? std::min(max_cycles, EXP_SQ_CYCLES) : max_cycles);
          if (c2 != KRYLOV_OK) return c2;
          for (int ap = 0; ap < a; ++ap) stats.launches += exp_row(h, ap, s_lv);
        }
        stats.launches += exp_row(h, a, s_lv);
        return KRYLOV_OK;
      };
      const bool sq = !quad || c <= EXP_SQ_CYCLES;
      const double* fsq = nullptr;
      if (sq) {
        if ((cs = squaring(false)) != KRYLOV_OK) return cs;
        fsq = square_row();
      }
      const double* fsrc = fsq;
      if (quad && c >= QUAD_START) {
        // fresh check maxima for this cycle (at the start, for every block so far)
        CK(cudaMemsetAsync(h->sd.qstat + 2, 0, 2 * sizeof(double), st));
        if (c == QUAD_START) {  // shift from the first block, then blocks 0 .. a - 1
          const double* f0 = h->sd.G + (size_t)s_lv * h->level_stride;
          launch_exp_quad_sigma(h->sd, M, h->f.t, f0, st);
          for (int ap = 0; ap < a; ++ap)
            launch_exp_quad(h->sd, h->cd, M, M, ap, h->f.t, f0 + (size_t)ap * (ap + 1) / 2 * MM, st);
          stats.launches += 1 + 2 * a;
        }
        launch_exp_quad(h->sd, h->cd, M, me, a, h->f.t, fsq, st);
        stats.launches += 3;
        if (!sq) {  // the contours must agree before the result is used
          CK(cudaMemcpyAsync(h->h_scal + 16, h->sd.qstat, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
          CK(cudaStreamSynchronize(st));
          if (h->h_scal[19] <= QUAD_TOL_CONTOURS) {
            fsrc = h->sd.fcol;
            stats.fquad_cycles += 1;
          } else {  // squaring from here on, all block rows formed now
            quad = false;
            if ((cs = squaring(true)) != KRYLOV_OK) return cs;
            fsrc = square_row();
          }
        }
      }
      launch_z(h->sd, M, me, fsrc, st);
      stats.launches += 1;
    } else if (h->f.kind == KRYLOV_F_INVSQRT) {
      launch_invsqrt_block(h->sd, h->cd, M, me, a, h->q_u0, INVSQRT_H, h->q_nodes, st);
      launch_z(h->sd, M, me, h->sd.fcol, st);
      stats.launches += 3;
    } else if (h->f.kind == KRYLOV_F_INV) {
      launch_inv_block(h->sd, M, me, a, st);
      launch_z(h->sd, M, me, h->sd.fcol, st);
      stats.launches += 2;
    } else {
      return KRYLOV_EUNSUPPORTED;
    }
    CK(cudaEventRecord(h->ev[3], st));
    phase.next("update");
    launch_update(basis, h->W, h->ldw, n, me, has_next, h->sd.zg, x, h->part, h->grid_update, h->cd, M, st);
    stats.launches += 1;
    CK(cudaGetLastError());
    if (h->part_mode) {  // ||y||^2, ||x||^2 and ||v_next||^2 over all ranks
      cs = comm_status(h->comm.allreduce_sum_f64(h->comm.ctx, h->cd.scal + 2, 2, st));
      if (cs == KRYLOV_OK) cs = comm_status(h->comm.allreduce_sum_f64(h->comm.ctx, h->cd.scal + 5, 1, st));
      if (cs != KRYLOV_OK) return cs;
    }
    CK(cudaMemcpyAsync(h->h_scal, h->cd.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h->h_scal + 8, h->sd.misc, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h->h_flags, h->cd.flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    if (quad) CK(cudaMemcpyAsync(h->h_scal + 16, h->sd.qstat, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    // a cycle with both evaluations: the quadrature must match the squaring and
    // its two contours each other, else the squaring continues alone
    if (quad && c >= QUAD_START && c <= EXP_SQ_CYCLES &&
        !(h->h_scal[18] <= QUAD_TOL_SQUARING && h->h_scal[19] <= QUAD_TOL_CONTOURS)) {
      // a Ritz value outside the contours: up to two retries with the shift
      // lowered by 3 / t (the quadrature of every block so far recomputed and
      // checked against the squaring block by block), else squaring alone
      bool fixed = false;
      const size_t MMq = (size_t)M * M;
      for (int attempt = 0; attempt < QUAD_RETRIES && !fixed; ++attempt) {
        h->h_scal[20] = h->h_scal[16] - 3.0 / h->f.t;  // sigma
        for (int q = 21; q < 24; ++q) h->h_scal[q] = 0.0;  // largest entry and check maxima
        CK(cudaMemcpyAsync(h->sd.qstat, h->h_scal + 20, 4 * sizeof(double), cudaMemcpyHostToDevice, st));
        for (int ap = 0; ap <= c - 1; ++ap) {
          const double* fsq_ap = h->sd.G + (size_t)s_lv * h->level_stride + (size_t)ap * (ap + 1) / 2 * MMq;
          launch_exp_quad(h->sd, h->cd, M, ap == c - 1 ? me : M, ap, h->f.t, fsq_ap, st);
          stats.launches += 2;
        }
        CK(cudaMemcpyAsync(h->h_scal + 16, h->sd.qstat, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        fixed = (h->h_scal[18] <= QUAD_TOL_SQUARING && h->h_scal[19] <= QUAD_TOL_CONTOURS);
      }
      if (!fixed) {
        quad = false;
        cs = ensure_small_capacity(h, max_cycles, s_lv + 1, max_cycles);  // rows beyond EXP_SQ_CYCLES
        if (cs != KRYLOV_OK) return cs;
        for (int ap = 0; ap <= c - 1; ++ap) stats.launches += exp_row(h, ap, s_lv);
      }
    }
    {
      float ms_q = 0.f;
      CK(cudaEventElapsedTime(&ms_q, h->ev[2], h->ev[3]));
      stats.ms_small += ms_q;
    }
    if (h->h_flags[2] & ERR_TIMEOUT) return KRYLOV_ETIMEOUT;  // a bounded wait of the small problem
    if (h->h_flags[2] & ERR_NONFINITE) return KRYLOV_ENONFINITE;
    stats.kappa_T_max = std::max(stats.kappa_T_max, h->h_scal[8 + 4]);
    const double ynorm = std::sqrt(h->h_scal[2]);
    const double xnorm = std::sqrt(h->h_scal[3]);
    stats.cycles = c;
    stats.last_update_norm = ynorm;
    stats.x_norm = xnorm;
    h->last_me = me;
    h->last_nc = nc;
    h->last_cycle = c;
    if (!std::isfinite(ynorm) || !std::isfinite(xnorm)) return KRYLOV_ENONFINITE;
    if (brk) {
      stats.breakdown = 1;
      result = KRYLOV_BREAKDOWN_EXACT;
      break;
    }
    // relative test: x must be nonzero (a first cycle whose update underflows
    // to zero has not yet resolved f(A) b and does not stop the method)
    const double lim = h->opt.abs_tol ? tol : tol * xnorm;
    if (ynorm <= lim && (h->opt.abs_tol || xnorm > 0.0)) {
      result = KRYLOV_OK;
      break;
    }
  }
  CK(cudaEventRecord(e1, st));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  stats.ms_total = ms;
  const double bv = basis_bytes(basis);
  stats.bytes_moved = stats.steps * model_bytes_step(h, use32) +
                      stats.cycles * ((M + 1) * (double)n * bv + 16.0 * n + n * bv);
  if (stout) *stout = stats;
  return result;
}

// apply_core with the call's status recorded in the stats (zeroed first, so a
// call that fails early leaves only the status set).
krylov_status apply_impl(krylov_handle* h, int transpose, const double* b, double* x, double tol,
                         int max_cycles, krylov_stats* stout) {
  if (stout) std::memset(stout, 0, sizeof(*stout));
  const krylov_status r = apply_core(h, transpose, b, x, tol, max_cycles, stout);
  if (stout) stout->status = r;
  return r;
}

constexpr int NQ_HOST = 2 + MAX_WINDOW;  // per-CTA scalar slots of the product kernels

// ---- block form (several right-hand sides of one matrix together) ----------

// Workspace of the block form for up to nb_cap right-hand sides: vectors
// row-major n x nb, per-right-hand-side cycle and small-problem state at the
// strides of bs.
struct BlockWs {
  int nb_cap = 0, rows_cap = 0, levels_cap = 0;
  int64_t level_stride = 0;
  void* W = nullptr;                 // float2 pairs, or floats for the float32 basis
  void* P[2] = {nullptr, nullptr};
  double* part = nullptr;
  long long* acc = nullptr;
  int* E = nullptr;
  int* active = nullptr;
  unsigned* counter = nullptr;
  CycleDev cd{};
  SmallDev sd{};
  BatchStride bs{};
  int* h_flags = nullptr;    // pinned: nb x 4
  double* h_scal = nullptr;  // pinned: nb x 8 (scal) then nb x 8 (misc)
  int* h_active = nullptr;   // pinned: nb
  std::vector<void*> allocs;
};

constexpr int BK_NB = 64;
constexpr int BK_MAX_CYCLES = 16;  // block exp rows stored for at most this many cycles

template <typename T>
cudaError_t balloc(BlockWs& b, T** p, size_t count, cudaStream_t st) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  b.allocs.push_back(q);
  *p = static_cast<T*>(q);
  // zeroed on the stream that uses it: the block kernels run on the
  // instance's non-blocking stream, which a plain cudaMemset (legacy default
  // stream) does not order against (the zeroing could land after them)
  return cudaMemsetAsync(q, 0, std::max<size_t>(count, 1) * sizeof(T), st);
}

void free_block_ws(BlockWs& b) {
  for (void* p : b.allocs) cudaFree(p);
  b.allocs.clear();
  if (b.h_flags) cudaFreeHost(b.h_flags);
  if (b.h_scal) cudaFreeHost(b.h_scal);
  if (b.h_active) cudaFreeHost(b.h_active);
  b = BlockWs{};
}

// Can the block kernels run this configuration?
bool block_eligible(const krylov_handle* h, int n_rhs, int max_cycles) {
  return h->opt.block_rhs && n_rhs > 1 &&
         (h->opt.basis_dtype == KRYLOV_BASIS_DF64 || h->opt.basis_dtype == KRYLOV_BASIS_F32) &&
         h->opt.ortho == KRYLOV_ORTHO_TRUNC && h->f.kind == KRYLOV_F_EXP_NEG && h->sk_mode == SK_TAB8 &&
         max_cycles <= BK_MAX_CYCLES && h->m <= 64 && bk_mat_smem(h->s, BK_NB) <= 200 * 1024;
}

krylov_status ensure_block_ws(krylov_handle* h, int levels) {
  BlockWs& b = *h->bk;
  const int M = h->m, s = h->s;
  const size_t MM = (size_t)M * M;
  if (b.nb_cap == 0) {
    const size_t n = (size_t)h->n;
    b.nb_cap = BK_NB;
    b.rows_cap = BK_MAX_CYCLES;
    // float-float pairs take two floats per entry, the float32 basis one
    const size_t fl = (h->opt.basis_dtype == KRYLOV_BASIS_F32) ? 1 : 2;
    float* w = nullptr;
    float* p0 = nullptr;
    float* p1 = nullptr;
    CK(balloc(b, &w, (size_t)(M + 1) * n * BK_NB * fl, h->st));
    CK(balloc(b, &p0, n * BK_NB * fl, h->st));
    CK(balloc(b, &p1, n * BK_NB * fl, h->st));
    b.W = w;
    b.P[0] = p0;
    b.P[1] = p1;
    CK(balloc(b, &b.part, (size_t)h->num_sms * 8 * NQ_HOST * BK_NB, h->st));
    CK(balloc(b, &b.acc, (size_t)(M + 1) * 3 * s * BK_NB, h->st));
    CK(balloc(b, &b.E, (size_t)(M + 1) * BK_NB, h->st));
    CK(balloc(b, &b.active, (size_t)BK_NB, h->st));
    CK(balloc(b, &b.counter, 4, h->st));
    BatchStride& bs = b.bs;
    bs.flags = 4;
    bs.sig2 = M + 1;
    bs.pi = M + 1;
    bs.coef = (int64_t)(M + 1) * (MAX_WINDOW + 1);
    bs.R = (int64_t)(M + 1) * M;
    bs.scal = 8;
    bs.U = (int64_t)s * (M + 1);
    bs.Tw = (int64_t)s * (M + 1);
    bs.Tinv = (int64_t)MM;
    bs.zg = 2 * M + 1;
    bs.Xblk = (int64_t)b.rows_cap * MM;
    bs.gam = b.rows_cap;
    bs.misc = 8;
    bs.S0 = (int64_t)std::max<size_t>(2 * (size_t)b.rows_cap * MM, MM);
    bs.fcol = M;
    CK(balloc(b, &b.cd.flags, (size_t)bs.flags * BK_NB, h->st));
    CK(balloc(b, &b.cd.sig2, (size_t)bs.sig2 * BK_NB, h->st));
    CK(balloc(b, &b.cd.pi, (size_t)bs.pi * BK_NB, h->st));
    CK(balloc(b, &b.cd.coef, (size_t)bs.coef * BK_NB, h->st));
    CK(balloc(b, &b.cd.R, (size_t)bs.R * BK_NB, h->st));
    CK(balloc(b, &b.cd.scal, (size_t)bs.scal * BK_NB, h->st));
    b.cd.counter = b.counter;
    CK(balloc(b, &b.sd.U, (size_t)bs.U * BK_NB, h->st));
    CK(balloc(b, &b.sd.Tw, (size_t)bs.Tw * BK_NB, h->st));
    CK(balloc(b, &b.sd.Tinv, (size_t)bs.Tinv * BK_NB, h->st));
    CK(balloc(b, &b.sd.zg, (size_t)bs.zg * BK_NB, h->st));
    CK(balloc(b, &b.sd.Xblk, (size_t)bs.Xblk * BK_NB, h->st));
    CK(balloc(b, &b.sd.gam, (size_t)bs.gam * BK_NB, h->st));
    CK(balloc(b, &b.sd.misc, (size_t)bs.misc * BK_NB, h->st));
    CK(balloc(b, &b.sd.S0, (size_t)bs.S0 * BK_NB, h->st));
    CK(balloc(b, &b.sd.fcol, (size_t)bs.fcol * BK_NB, h->st));
    if (cudaMallocHost(&b.h_flags, sizeof(int) * 4 * BK_NB) != cudaSuccess) return KRYLOV_ENOMEM;
    if (cudaMallocHost(&b.h_scal, sizeof(double) * 16 * BK_NB) != cudaSuccess) return KRYLOV_ENOMEM;
    if (cudaMallocHost(&b.h_active, sizeof(int) * BK_NB) != cudaSuccess) return KRYLOV_ENOMEM;
  }
  if (levels > b.levels_cap) {
    const int nl = std::max(levels, b.levels_cap + 4);
    if (b.sd.G) {
      cudaFree(b.sd.G);
      b.allocs.erase(std::find(b.allocs.begin(), b.allocs.end(), (void*)b.sd.G));
      b.sd.G = nullptr;
    }
    b.level_stride = (int64_t)b.rows_cap * (b.rows_cap + 1) / 2 * (int64_t)MM;
    b.bs.G = (int64_t)nl * b.level_stride;
    CK(balloc(b, &b.sd.G, (size_t)b.bs.G * BK_NB, h->st));
    b.levels_cap = nl;
  }
  return KRYLOV_OK;
}

// Block row a of exp(-t H_r) for every right-hand side r at scale levels 0..sl.
int exp_row_block(krylov_handle* h, int nb, int a, int sl, cudaStream_t st) {
  BlockWs& b = *h->bk;
  const int M = h->m;
  const size_t MM = (size_t)M * M;
  const double scale = -h->f.t / std::ldexp(1.0, sl);
  double* g0row = b.sd.G + (size_t)a * (a + 1) / 2 * MM;
  int src = 0;
  for (int kdeg = EXP_TAYLOR_DEG; kdeg >= 1; --kdeg) {
    const int first = (kdeg == EXP_TAYLOR_DEG);
    double* dst = (kdeg == 1) ? g0row : b.sd.S0 + (size_t)(1 - src) * (size_t)(a + 1) * MM;
    launch_exp_taylor_batched(b.sd, b.bs, nb, M, a, kdeg, scale, first, src, dst, kdeg == 1 ? 1 : 0, st);
    src = 1 - src;
  }
  for (int lv = 0; lv < sl; ++lv) launch_exp_square_batched(b.sd, b.bs, nb, M, a, lv, b.level_stride, st);
  return EXP_TAYLOR_DEG + sl;
}

// nb (<= 64) right-hand sides of the caller's row-major block B (column c0
// on, leading dimension ldb) through the block kernels; results into X (same
// layout).  Right-hand sides that meet a breakdown are flagged in `redo` and
// solved afterwards by the single-vector path.
krylov_status block_solve(krylov_handle* h, const double* B, double* X, int64_t ldb, int nb, double tol,
                          int max_cycles, krylov_stats* st, std::vector<int>& redo) {
  if (!h->bk) h->bk = new (std::nothrow) BlockWs();
  if (!h->bk) return KRYLOV_ENOMEM;
  BlockWs& b = *h->bk;
  cudaStream_t s_ = h->st;
  const int M = h->m, n = h->n;
  const size_t MM = (size_t)M * M;
  krylov_status cs = ensure_block_ws(h, std::max(1, b.levels_cap));
  if (cs != KRYLOV_OK) return cs;
  const int b32 = (h->opt.basis_dtype == KRYLOV_BASIS_F32) ? 1 : 0;
  const int use32 = (b32 || (h->opt.narrow_values_if_exact && h->vals_exact_f32)) ? 1 : 0;
  BlockLaunch L{};
  L.basis32 = b32;
  L.n = n;
  L.nb = nb;
  L.m = M;
  L.k = h->k;
  L.s = h->s;
  L.zeta = h->opt.zeta;
  L.rp = h->rp;
  L.ci = h->ci;
  L.val = use32 ? (const void*)h->val32 : (const void*)h->valff;
  L.val_f32 = use32;
  L.W = b.W;
  L.slot = (int64_t)n * nb;
  L.part = b.part;
  L.cd = b.cd;
  L.bs = b.bs;
  L.counter = b.counter;
  L.acc = b.acc;
  L.E = b.E;
  L.tab = h->sk_tab;
  // grids from the kernels' occupancy (the materialize kernel holds nb-wide
  // sketch bins in shared memory, the product and update kernels none)
  // (a full wave each for one instance; two CTAs per SM when several
  // instances run concurrently and fill the GPU between them)
  const int part_ctas = h->num_sms * 8;
  const int per_sm_mat = (h->bk_concurrent > 1) ? 2 : bk_ctas_per_sm(0, bk_mat_smem(h->s, nb));
  const int per_sm_p = (h->bk_concurrent > 1) ? 2 : bk_ctas_per_sm(1, 0);
  L.grid = std::max(1, std::min(std::min(part_ctas, h->num_sms * per_sm_mat), (n + 7) / 8));
  L.rows_per_cta = (n + L.grid - 1) / L.grid;
  L.grid_p = std::max(1, std::min(std::min(part_ctas, h->num_sms * per_sm_p), (n + 7) / 8));
  L.rows_p = (n + L.grid_p - 1) / L.grid_p;
  L.fx_wb = sketch_word_bits(L.rows_per_cta, 1);
  L.thr = b32 ? 1e-6 : 1e-12;  // the breakdown thresholds of the single-vector path
  NvtxRange call_range("krylov_apply_batched block");
  EventPair evp;
  CK(evp.create());
  cudaEvent_t e0 = evp.a, e1 = evp.b;
  CK(cudaEventRecord(e0, s_));
  // x = 0 in the block's columns; flags, misc cleared
  launch_zero_columns(X, n, ldb, nb, s_);
  CK(cudaMemsetAsync(b.cd.flags, 0, sizeof(int) * 4 * BK_NB, s_));
  CK(cudaMemsetAsync(b.sd.misc, 0, sizeof(double) * 8 * BK_NB, s_));
  launch_bk_norm_start(L, B, ldb, s_);
  CK(cudaMemcpyAsync(b.h_scal, b.cd.scal, sizeof(double) * 8 * nb, cudaMemcpyDeviceToHost, s_));
  CK(cudaStreamSynchronize(s_));
  std::vector<int> active((size_t)nb, 1), done((size_t)nb, 0);
  std::vector<double> maxX((size_t)nb, 0.0), maxG((size_t)nb, 0.0);
  for (int r = 0; r < nb; ++r) {
    std::memset(&st[r], 0, sizeof(krylov_stats));
    st[r].status = KRYLOV_NOT_CONVERGED;
    if (!(b.h_scal[8 * r] > 0.0) || !std::isfinite(b.h_scal[8 * r])) {  // b_r = 0 (or invalid): one by one
      active[r] = 0;
      redo.push_back(r);
    }
  }
  int s_lv = -1, launches = 2;
  double ms_steps = 0.0, step_bytes = 0.0;
  for (int c = 1; c <= max_cycles; ++c) {
    int n_active = 0;
    for (int r = 0; r < nb; ++r) {
      b.h_active[r] = active[r];
      n_active += active[r];
      b.h_flags[4 * r] = M;
      b.h_flags[4 * r + 1] = 0;
      b.h_flags[4 * r + 2] = 0;
      b.h_flags[4 * r + 3] = 0;
    }
    if (n_active == 0) break;
    CK(cudaMemcpyAsync(b.active, b.h_active, sizeof(int) * nb, cudaMemcpyHostToDevice, s_));
    CK(cudaMemcpyAsync(b.cd.flags, b.h_flags, sizeof(int) * 4 * nb, cudaMemcpyHostToDevice, s_));
    CK(cudaEventRecord(h->ev[0], s_));
    for (int j = 0; j <= M; ++j) {
      L.j = j;
      L.p_prev = b.P[(j + 1) & 1];
      L.p_out = b.P[j & 1];
      launch_bk_step(L, j > 0, j < M, s_);
      launches += (j < M) ? 2 : 1;
    }
    CK(cudaEventRecord(h->ev[1], s_));
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(b.h_flags, b.cd.flags, sizeof(int) * 4 * nb, cudaMemcpyDeviceToHost, s_));
    CK(cudaStreamSynchronize(s_));
    {
      float ms_s = 0.f;
      CK(cudaEventElapsedTime(&ms_s, h->ev[0], h->ev[1]));
      ms_steps += ms_s;
      // per step: A once, and per right-hand side the vectors of a single step
      step_bytes += M * ((double)h->nnz * ((use32 ? 4.0 : 8.0) + 4.0) + 4.0 * (n + 1) +
                         (double)nb * (model_bytes_step(h, use32) - (double)h->nnz * ((use32 ? 4.0 : 8.0) + 4.0) -
                                       4.0 * (n + 1)));
    }
    for (int r = 0; r < nb; ++r) {
      if (!active[r]) continue;
      if (b.h_flags[4 * r + 1] != 0 || (b.h_flags[4 * r + 2] & (ERR_NONFINITE | ERR_SKETCH | ERR_TIMEOUT))) {
        active[r] = 0;  // breakdown (or trouble): this right-hand side is redone alone
        redo.push_back(r);
      }
    }
    launch_bk_sketch_fin(L, b.sd, M + 1, s_);
    launch_whiten_batched(b.sd, b.cd, b.bs, nb, h->bk_concurrent, h->s, M, M + 1, M, 1, c, h->k, h->f.t, s_);
    CK(cudaMemcpyAsync(b.h_scal + 8 * BK_NB, b.sd.misc, sizeof(double) * 8 * nb, cudaMemcpyDeviceToHost, s_));
    CK(cudaStreamSynchronize(s_));
    launches += 2;
    int need = 0;
    for (int r = 0; r < nb; ++r) {
      if (!active[r]) continue;
      const double* mi = b.h_scal + 8 * BK_NB + 8 * r;
      maxX[r] = std::max(maxX[r], mi[2]);
      maxG[r] = std::max(maxG[r], mi[3]);
      st[r].kappa_T_max = std::max(st[r].kappa_T_max, mi[4]);
      if (!std::isfinite(maxX[r]) || !std::isfinite(maxG[r])) {
        active[r] = 0;
        redo.push_back(r);
        continue;
      }
      need = std::max(need, scale_levels_for(maxX[r] + maxG[r]));
    }
    const int a = c - 1;
    if (need > s_lv) {
      s_lv = need;
      cs = ensure_block_ws(h, s_lv + 1);
      if (cs != KRYLOV_OK) return cs;
      for (int ap = 0; ap < a; ++ap) launches += exp_row_block(h, nb, ap, s_lv, s_);
    }
    launches += exp_row_block(h, nb, a, s_lv, s_);
    const double* fsrc = b.sd.G + (size_t)s_lv * b.level_stride + (size_t)a * (a + 1) / 2 * MM;
    launch_z_batched(b.sd, b.bs, nb, M, M, fsrc, b.bs.G, s_);
    for (int r = 0; r < nb; ++r) b.h_active[r] = active[r];
    CK(cudaMemcpyAsync(b.active, b.h_active, sizeof(int) * nb, cudaMemcpyHostToDevice, s_));
    launch_bk_update(L, b.sd, M, 1, X, ldb, b.active, s_);
    launches += 2;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(b.h_scal, b.cd.scal, sizeof(double) * 8 * nb, cudaMemcpyDeviceToHost, s_));
    CK(cudaStreamSynchronize(s_));
    for (int r = 0; r < nb; ++r) {
      if (!active[r]) continue;
      const double yn = std::sqrt(b.h_scal[8 * r + 2]), xn = std::sqrt(b.h_scal[8 * r + 3]);
      st[r].cycles = c;
      st[r].steps += M;
      st[r].last_update_norm = yn;
      st[r].x_norm = xn;
      if (!std::isfinite(yn) || !std::isfinite(xn)) {
        active[r] = 0;
        redo.push_back(r);
        continue;
      }
      const double lim = h->opt.abs_tol ? tol : tol * xn;
      if (yn <= lim && (h->opt.abs_tol || xn > 0.0)) {
        active[r] = 0;
        st[r].status = KRYLOV_OK;
      }
    }
  }
  CK(cudaEventRecord(e1, s_));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  // block-wide figures are reported once, on the block's first right-hand side
  for (int r = 0; r < nb; ++r) {
    st[r].ms_total = ms;
    st[r].launches = (r == 0) ? launches : 0;
    st[r].step_launches = (r == 0) ? launches : 0;
    st[r].ms_steps = (r == 0) ? ms_steps : 0.0;
    st[r].step_bytes = (r == 0) ? step_bytes : 0.0;
  }
  return KRYLOV_OK;
}

// One instance of the batched form: its right-hand sides in order, on a
// stream of its own ordered after (and, at the end, before) the handle's stream.
krylov_status run_instance(krylov_handle* h, int n_rhs, const double* B, double* X, const double* t_new, double tol,
                           int max_cycles, krylov_stats* st) {
  if (cudaSetDevice(h->device) != cudaSuccess) return KRYLOV_ECUDA;
  cudaStream_t orig = h->st, bs = nullptr;
  cudaEvent_t ev = nullptr;
  if (cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) != cudaSuccess) return KRYLOV_ECUDA;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaStreamDestroy(bs);
    return KRYLOV_ECUDA;
  }
  krylov_status worst = KRYLOV_OK;
  const double t_old = h->f.t;
  if (t_new && (h->f.kind == KRYLOV_F_EXP_NEG || h->f.kind == KRYLOV_F_PHI1_NEG || h->f.kind == KRYLOV_F_COS_SQRT))
    h->f.t = *t_new;
  if (cudaEventRecord(ev, orig) != cudaSuccess || cudaStreamWaitEvent(bs, ev, 0) != cudaSuccess) worst = KRYLOV_ECUDA;
  h->st = bs;
  if (worst == KRYLOV_OK && !h->stage_b) {
    if (dalloc(h, &h->stage_b, (size_t)h->n) != cudaSuccess || dalloc(h, &h->stage_x, (size_t)h->n) != cudaSuccess)
      worst = KRYLOV_ENOMEM;
  }
  // block kernels: up to 64 right-hand sides advance together; those that meet
  // a breakdown (or a zero right-hand side) are redone one by one below
  std::vector<char> todo((size_t)n_rhs, 1);
  if (worst == KRYLOV_OK && block_eligible(h, n_rhs, max_cycles)) {
    std::vector<krylov_stats> bst((size_t)n_rhs);
    for (int c0 = 0; c0 < n_rhs && worst == KRYLOV_OK; c0 += BK_NB) {
      const int nb = std::min(BK_NB, n_rhs - c0);
      std::vector<int> redo;
      const krylov_status s = block_solve(h, B + c0, X + c0, n_rhs, nb, tol, max_cycles, bst.data() + c0, redo);
      if (s != KRYLOV_OK) {
        worst = s;
        break;
      }
      for (int r = 0; r < nb; ++r) todo[(size_t)(c0 + r)] = 0;
      for (int r : redo) todo[(size_t)(c0 + r)] = 1;
    }
    for (int r = 0; r < n_rhs; ++r) {
      if (todo[(size_t)r]) continue;
      if (st) st[r] = bst[(size_t)r];
      if (bst[(size_t)r].status == KRYLOV_NOT_CONVERGED && worst == KRYLOV_OK) worst = KRYLOV_NOT_CONVERGED;
    }
  }
  // every right-hand side runs even if an earlier one failed (its status is in
  // its stats); only a CUDA error stops the instance
  for (int r = 0; r < n_rhs && worst != KRYLOV_ECUDA && worst != KRYLOV_ENOMEM; ++r) {
    if (!todo[(size_t)r]) continue;
    launch_gather_column(B, h->n, n_rhs, r, h->stage_b, bs);
    krylov_status s = apply_impl(h, 0, h->stage_b, h->stage_x, tol, max_cycles, st ? st + r : nullptr);
    launch_scatter_column(h->stage_x, h->n, n_rhs, r, X, bs);
    if (cudaGetLastError() != cudaSuccess) s = KRYLOV_ECUDA;
    if (s < 0 && worst >= 0) worst = s;
    if (s == KRYLOV_NOT_CONVERGED && worst == KRYLOV_OK) worst = KRYLOV_NOT_CONVERGED;
  }
  h->st = orig;
  h->f.t = t_old;
  if (cudaEventRecord(ev, bs) != cudaSuccess || cudaStreamWaitEvent(orig, ev, 0) != cudaSuccess) worst = KRYLOV_ECUDA;
  cudaEventDestroy(ev);
  cudaStreamDestroy(bs);
  return worst;
}

}  // namespace

extern "C" {

void krylov_options_default(krylov_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->zeta = 8;
  opt->basis_dtype = KRYLOV_BASIS_F64;
  opt->ortho = KRYLOV_ORTHO_TRUNC;
  opt->narrow_values_if_exact = 1;
  opt->use_graph = 1;
  opt->autotune = 1;
  opt->block_rhs = 1;
  opt->abs_tol = 0;
  opt->stream = nullptr;
}

const char* krylov_status_string(krylov_status s) {
  switch (s) {
    case KRYLOV_OK: return "ok";
    case KRYLOV_NOT_CONVERGED: return "not converged within max_cycles";
    case KRYLOV_BREAKDOWN_EXACT: return "happy breakdown: exact result";
    case KRYLOV_EINVAL: return "invalid argument";
    case KRYLOV_ENOMEM: return "device out of memory";
    case KRYLOV_ECUDA: return "CUDA error";
    case KRYLOV_ENONFINITE: return "non-finite value";
    case KRYLOV_ETIMEOUT: return "device wait timed out";
    case KRYLOV_EUNSUPPORTED: return "unsupported option";
  }
  return "unknown status";
}

void krylov_destroy(krylov_handle* h) {
  if (!h) return;
  for (void* p : h->allocs)
    if (p) cudaFree(p);
  for (auto& e : h->ev)
    if (e) cudaEventDestroy(e);
  for (auto& g : h->step_graph)
    if (g) cudaGraphExecDestroy(g);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->bk) {
    free_block_ws(*h->bk);
    delete h->bk;
  }
  if (h->h_flags) cudaFreeHost(h->h_flags);
  if (h->h_scal) cudaFreeHost(h->h_scal);
  delete h;
}

// what krylov_create_partition adds to krylov_create (null for a whole matrix)
struct PartSpec {
  int64_t n_halo, row0, n_global;
  const int32_t* send_idx;
  int64_t n_send;
  const krylov_comm* comm;
};

static krylov_status create_impl(const krylov_csr* A, krylov_func f, int m, int k, int s, uint64_t seed,
                                 const krylov_options* opt_in, const PartSpec* ps, krylov_handle** out) {
  if (!A || !out) return KRYLOV_EINVAL;
  *out = nullptr;
  krylov_options opt;
  krylov_options_default(&opt);
  if (opt_in) opt = *opt_in;
  if (A->n < 1 || A->n > 0x7FF00000LL || A->nnz < 0 || A->nnz > 0x7FFFFFF0LL) return KRYLOV_EINVAL;
  if (!A->row_ptr || (A->nnz > 0 && (!A->col_idx || !A->val))) return KRYLOV_EINVAL;
  if (m < 1 || m > 256 || k < 1 || s < m + 1 || s > 1024) return KRYLOV_EINVAL;
  if (k > ((opt.ortho == KRYLOV_ORTHO_RGS) ? m : MAX_WINDOW)) return KRYLOV_EINVAL;
  if (opt.zeta < 1 || opt.zeta > std::min(s, MAX_ZETA)) return KRYLOV_EINVAL;
  if (opt.basis_dtype < 0 || opt.basis_dtype > 3) return KRYLOV_EINVAL;
  if (opt.ortho != KRYLOV_ORTHO_TRUNC && opt.ortho != KRYLOV_ORTHO_RGS) return KRYLOV_EINVAL;
  if (opt.autotune < 0 || opt.autotune > 2) return KRYLOV_EINVAL;
  // the randomized Gram-Schmidt cycle runs with the float64 and float-float bases
  if (opt.ortho == KRYLOV_ORTHO_RGS && opt.basis_dtype != KRYLOV_BASIS_F64 && opt.basis_dtype != KRYLOV_BASIS_DF64)
    return KRYLOV_EUNSUPPORTED;
  if (f.kind != KRYLOV_F_EXP_NEG && f.kind != KRYLOV_F_INV && f.kind != KRYLOV_F_INVSQRT &&
      f.kind != KRYLOV_F_PHI1_NEG && f.kind != KRYLOV_F_COS_SQRT)
    return KRYLOV_EINVAL;
  if (!std::isfinite(f.t)) return KRYLOV_EINVAL;
  if (ps) {
    const krylov_comm* cm = ps->comm;
    if (!cm || !cm->allreduce_sum_f64 || !cm->allreduce_sum_i64 || !cm->allreduce_max_f64 ||
        !cm->halo_exchange_f64)
      return KRYLOV_EINVAL;
    if (ps->n_halo < 0 || ps->n_send < 0 || ps->row0 < 0 || ps->n_global < A->n || ps->row0 + A->n > ps->n_global)
      return KRYLOV_EINVAL;
    if (ps->n_global > 0xFFFFFFFFLL || A->n + ps->n_halo > 0x7FF00000LL || ps->n_send > 0x7FF00000LL)
      return KRYLOV_EINVAL;
    if (ps->n_send > 0 && !ps->send_idx) return KRYLOV_EINVAL;
    for (int64_t e = 0; e < ps->n_send; ++e)
      if (ps->send_idx[e] < 0 || ps->send_idx[e] >= A->n) return KRYLOV_EINVAL;
    if (opt.basis_dtype != KRYLOV_BASIS_F64 || opt.ortho != KRYLOV_ORTHO_TRUNC || opt.sketch_regenerate)
      return KRYLOV_EUNSUPPORTED;
  }
  const int64_t ncols = A->n + (ps ? ps->n_halo : 0);  // columns of the stored rows

  krylov_handle* h = new (std::nothrow) krylov_handle();
  if (!h) return KRYLOV_ENOMEM;
  h->n = (int)A->n;
  h->ldw = (ncols + 63) / 64 * 64;  // basis slot stride (also the padded length of row arrays)
  h->nnz = A->nnz;
  h->m = m;
  h->k = k;
  h->s = s;
  h->seed = seed;
  h->f = f;
  h->opt = opt;
  h->st = static_cast<cudaStream_t>(opt.stream);
  auto fail = [&](krylov_status st) {
    krylov_destroy(h);
    return st;
  };
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(KRYLOV_ECUDA);
  h->device = dev;
  if (cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(KRYLOV_ECUDA);
  if (cudaMallocHost(&h->h_flags, 16 * sizeof(int)) != cudaSuccess) return fail(KRYLOV_ENOMEM);
  if (cudaMallocHost(&h->h_scal, 32 * sizeof(double)) != cudaSuccess) return fail(KRYLOV_ENOMEM);

  const int n = h->n;
  const int64_t nnz = h->nnz;
  const cudaMemcpyKind kind = A->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
#define CKF(call)                                     \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return fail(cuda_status(e_)); \
  } while (0)
  CKF(dalloc(h, &h->rp, (size_t)n + 1 + RP_PAD));
  CKF(dalloc(h, &h->ci, (size_t)nnz + CSR_PAD));
  CKF(dalloc(h, &h->val, (size_t)nnz + CSR_PAD));
  CKF(dalloc(h, &h->d_flag, 4));
  CKF(cudaMemcpyAsync(h->rp, A->row_ptr, sizeof(int) * ((size_t)n + 1), kind, h->st));
  if (nnz > 0) {
    CKF(cudaMemcpyAsync(h->ci, A->col_idx, sizeof(int) * (size_t)nnz, kind, h->st));
    CKF(cudaMemcpyAsync(h->val, A->val, sizeof(double) * (size_t)nnz, kind, h->st));
  }
  CKF(cudaMemsetAsync(h->ci + nnz, 0, CSR_PAD * sizeof(int), h->st));
  CKF(cudaMemsetAsync(h->rp + n + 1, 0, RP_PAD * sizeof(int), h->st));
  CKF(cudaMemsetAsync(h->val + nnz, 0, CSR_PAD * sizeof(double), h->st));
  CKF(validate_csr(n, nnz, h->rp, h->ci, h->d_flag, h->h_flags, h->st, (int)ncols));
  if (h->h_flags[0] != 0) return fail(KRYLOV_EINVAL);
  // float32 copy of the values: exact-narrowing test, and the operand of the
  // float32/bfloat16 basis modes
  CKF(dalloc(h, &h->val32, (size_t)nnz + CSR_PAD));
  CKF(cudaMemsetAsync(h->val32 + nnz, 0, CSR_PAD * sizeof(float), h->st));
  CKF(narrow_values(nnz, h->val, h->val32, h->d_flag, h->h_flags, h->st));
  h->vals_exact_f32 = (h->h_flags[0] == 0);
  CKF(tile_span_max(n, h->rp, h->d_flag, h->h_flags, h->st));
  h->tma_cap = (h->h_flags[0] <= TMA_MAX_CAP) ? std::max(h->h_flags[0], 8) : 0;
  if (opt.basis_dtype == KRYLOV_BASIS_DF64 && !(h->vals_exact_f32 && opt.narrow_values_if_exact)) {
    CKF(dalloc(h, &h->valff, (size_t)nnz + CSR_PAD));
    CKF(cudaMemsetAsync(h->valff + nnz, 0, CSR_PAD * sizeof(float2), h->st));
    CKF(split_values(nnz, h->val, h->valff, h->st));
  }

  for (auto& e : h->ev)
    if (cudaEventCreate(&e) != cudaSuccess) return fail(KRYLOV_ECUDA);
  // the sparse sign embedding S: a device table (default) or regenerated in
  // every step kernel
  const bool packed = (s <= 255 && opt.zeta <= 8);
  h->sk_copies = sketch_bin_copies(opt.basis_dtype, s);
  if (opt.sketch_regenerate) {
    h->sk_mode = packed ? SK_GEN8 : SK_GEN;
  } else {
    h->sk_mode = packed ? SK_TAB8 : SK_TAB16;
    h->sk_tab.packed = packed ? 1 : 0;
    if (packed) {
      // padded to the slot stride: staged copies read whole 16-row groups
      CKF(dalloc(h, &h->sk_tab.rows8, (size_t)h->ldw));
      CKF(dalloc(h, &h->sk_tab.neg8, (size_t)h->ldw));
    } else {
      CKF(dalloc(h, &h->sk_tab.rows16, (size_t)n * opt.zeta));
      CKF(dalloc(h, &h->sk_tab.neg32, (size_t)n));
    }
    CKF(cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->st));
    launch_sketch_table(n, s, opt.zeta, seed, h->sk_tab, h->d_flag, h->st, ps ? ps->row0 : 0);
    CKF(cudaGetLastError());
    CKF(cudaMemcpyAsync(h->h_flags, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CKF(cudaStreamSynchronize(h->st));
    if (h->h_flags[0] != 0) return fail(KRYLOV_ECUDA);
  }
  // workspaces: one persistent wave of the step kernel(s)
  const int vals32 = (opt.basis_dtype == 1 || opt.basis_dtype == 2) ||
                     (h->vals_exact_f32 && opt.narrow_values_if_exact);
  // float32 / bfloat16 bases: the staged pair of step kernels when the packed
  // sketch table and the staged CSR tiles apply, else the fused kernel
  h->staged32 = (opt.basis_dtype == 1 || opt.basis_dtype == 2) && h->sk_mode == SK_TAB8 && h->tma_cap > 0 &&
                opt.ortho == KRYLOV_ORTHO_TRUNC && !ps;
  const int cps = h->staged32 ? s32_ctas_per_sm(opt.basis_dtype, s, h->sk_copies)
                              : step_ctas_per_sm(opt.basis_dtype, h->sk_mode, s, h->sk_copies, vals32);
  h->grid = std::max(1, std::min(h->num_sms * cps, (n + STEP_THREADS - 1) / STEP_THREADS));
  if (opt.basis_dtype == 3 && h->sk_mode == SK_TAB8)
    h->grid_mat = std::max(1, std::min(h->num_sms * mat_ctas_per_sm(s, h->sk_copies), (n + STEP_THREADS - 1) / STEP_THREADS));
  const int bb = basis_bytes(opt.basis_dtype);
  CKF(cudaMalloc(&h->W, (size_t)(m + 1) * h->ldw * bb));
  h->allocs.push_back(h->W);
  const int pb = wide(opt.basis_dtype) ? 8 : 4;
  for (int i = 0; i < 2; ++i) {
    CKF(cudaMalloc(&h->p[i], (size_t)h->ldw * pb));
    h->allocs.push_back(h->p[i]);
  }
  h->sk_col_stride = (int64_t)h->grid * s;
  CKF(cudaMalloc(&h->sk_part, (size_t)(m + 1) * h->sk_col_stride * sizeof(double)));
  h->allocs.push_back(h->sk_part);
  h->grid_spmv = h->grid;
  if (opt.basis_dtype == 3) {
    krylov_status ps = install_long_rows(h, h->long_a, h->rp, h->ci, h->val32, h->valff);
    if (ps != KRYLOV_OK) return fail(ps);
    if (h->long_a.n_long == 0) {  // plans describe the full operator
      ps = install_seg_plan(h, h->seg_a, h->rp, h->ci);
      if (ps != KRYLOV_OK) return fail(ps);
      ps = install_delta16(h, h->rp, h->ci, &h->dcol);
      if (ps != KRYLOV_OK) return fail(ps);
    }
    const SegPlan& sp = h->seg_a;
    const int tcap = h->long_a.n_long ? h->long_a.tma_cap : h->tma_cap;
    h->grid_spmv = std::max(1, std::min(h->num_sms * spmv_ctas_per_sm(vals32, tcap, sp.seg ? sp.seg_cap : 0,
                                                                      sp.lcap),
                                        (n + STEP_THREADS - 1) / STEP_THREADS));
  }
  if (h->staged32) {
    const krylov_status ps2 = install_delta16(h, h->rp, h->ci, &h->dcol);
    if (ps2 != KRYLOV_OK) return fail(ps2);
    h->grid_spmv = std::max(1, std::min(h->num_sms * s32_spmv_ctas_per_sm(h->tma_cap, h->dcol != nullptr ? 1 : 0),
                                        (n + STEP_THREADS - 1) / STEP_THREADS));
  }
  h->grid_spmv_t = h->grid_spmv;
  h->part_cap = std::max(h->grid, std::min(h->num_sms * 32, (n + STEP_THREADS - 1) / STEP_THREADS));
  CKF(dalloc(h, &h->part, (size_t)h->part_cap * 8));
  CKF(dalloc(h, &h->part_w, (size_t)h->part_cap * 2));
  if ((opt.basis_dtype == 3 || h->staged32) && KRYLOV_SELL) {
    const krylov_status ps3 = install_sell(h, vals32);
    if (ps3 != KRYLOV_OK) return fail(ps3);
    if (h->sell_col && !h->seg_a.seg) h->grid_spmv = h->grid_sell;
  }
  // the update pass streams m + 2 vectors: 8 resident CTAs per SM
  h->grid_update = std::max(1, std::min(h->part_cap, std::min(h->num_sms * 8, (n + STEP_THREADS - 1) / STEP_THREADS)));
  CKF(dalloc(h, &h->cd.flags, 4));
  CKF(dalloc(h, &h->cd.sig2, (size_t)m + 1));
  CKF(dalloc(h, &h->cd.pi, (size_t)m + 1));
  CKF(dalloc(h, &h->cd.coef, (size_t)(m + 1) * (MAX_WINDOW + 1)));
  CKF(dalloc(h, &h->cd.R, (size_t)(m + 1) * m));
  CKF(dalloc(h, &h->cd.scal, 8));
  CKF(dalloc(h, &h->cd.counter, 4));
  CKF(dalloc(h, &h->cd.sig2ff, (size_t)m + 1));
  CKF(dalloc(h, &h->cd.piff, (size_t)m + 1));
  CKF(dalloc(h, &h->cd.rff, (size_t)m + 1));
  h->sk_acc_stride = 3 * (int64_t)s + 1;
  {
    long long* acc = nullptr;
    CKF(dalloc(h, &acc, (size_t)(m + 1) * h->sk_acc_stride));
    h->sk_acc = acc;
  }
  CKF(cudaMemsetAsync(h->cd.counter, 0, 4 * sizeof(unsigned), h->st));
  CKF(cudaMemsetAsync(h->cd.R, 0, sizeof(double) * (size_t)(m + 1) * m, h->st));
  CKF(dalloc(h, &h->sd.U, (size_t)s * (m + 1)));
  CKF(dalloc(h, &h->sd.Tw, (size_t)s * (m + 1)));
  CKF(dalloc(h, &h->sd.Tinv, (size_t)m * m));
  CKF(dalloc(h, &h->sd.zg, (size_t)2 * m + 1));
  CKF(dalloc(h, &h->sd.misc, 8));
  CKF(dalloc(h, &h->sd.fcol, (size_t)m));
  if (opt.ortho == KRYLOV_ORTHO_RGS) {
    CKF(dalloc(h, &h->rgs_acc, (size_t)3 * s));
    CKF(cudaMemsetAsync(h->rgs_acc, 0, sizeof(long long) * 3 * (size_t)s, h->st));
  }
  if (f.kind == KRYLOV_F_INVSQRT) {
    double alpha = 0.0;
    CKF(norm_inf(n, h->rp, h->val, h->d_flag, h->h_flags, &alpha, h->st));
    if (ps) {  // ||A||_inf over all ranks' rows
      double* d = nullptr;
      CKF(dalloc(h, &d, 1));
      CKF(cudaMemcpyAsync(d, &alpha, sizeof(double), cudaMemcpyHostToDevice, h->st));
      CKF(cudaStreamSynchronize(h->st));
      if (ps->comm->allreduce_max_f64(ps->comm->ctx, d, 1, h->st) != 0) return fail(KRYLOV_ECUDA);
      CKF(cudaMemcpyAsync(&alpha, d, sizeof(double), cudaMemcpyDeviceToHost, h->st));
      CKF(cudaStreamSynchronize(h->st));
    }
    if (!std::isfinite(alpha)) return fail(KRYLOV_EINVAL);
    if (alpha == 0.0) alpha = 1.0;
    const double u_lo = 0.5 * std::log(alpha * 1e-18) - 38.0;
    const double u_hi = 0.5 * std::log(alpha * 1e4) + 38.0;
    h->q_nodes = (int)std::ceil((u_hi - u_lo) / INVSQRT_H) + 1;
    h->q_u0 = u_lo;
    CKF(dalloc(h, &h->sd.qcarry, (size_t)h->q_nodes));
    CKF(dalloc(h, &h->sd.qpart, (size_t)h->q_nodes * m));
    if (invsqrt_smem(m) == (size_t)256 * sizeof(double))
      CKF(dalloc(h, &h->sd.qwork, (size_t)h->q_nodes * m * m));
  }
  if (f.kind == KRYLOV_F_EXP_NEG) {  // contour-quadrature state of exp(-t z)
    const int nodes = exp_quad_nodes();
    CKF(dalloc(h, &h->sd.qstat, 4));
    CKF(dalloc(h, &h->sd.qcarry, (size_t)2 * nodes));
    CKF(dalloc(h, &h->sd.qpart, (size_t)nodes * m));
    if (exp_quad_smem(m) == (size_t)256 * 2 * sizeof(double))
      CKF(dalloc(h, &h->sd.qwork, (size_t)nodes * m * m * 2));
  }
  CKF(dalloc(h, &h->d_dot, 1));
  if (ps) {
    h->part_mode = 1;
    h->n_halo = (int)ps->n_halo;
    h->n_send = (int)ps->n_send;
    h->row0 = ps->row0;
    h->n_global = ps->n_global;
    h->comm = *ps->comm;
    CKF(dalloc(h, &h->send_idx, (size_t)h->n_send));
    if (h->n_send > 0)
      CKF(cudaMemcpyAsync(h->send_idx, ps->send_idx, sizeof(int) * (size_t)h->n_send, cudaMemcpyHostToDevice,
                          h->st));
    CKF(dalloc(h, &h->sendbuf, (size_t)h->n_send));
    CKF(dalloc(h, &h->recvbuf, (size_t)h->n_halo));
    CKF(dalloc(h, &h->red, (size_t)PART_NQ + 1));
    CKF(dalloc(h, &h->part_acc, (size_t)(m + 1) * 3 * s));
    CKF(dalloc(h, &h->part_E, (size_t)m + 1));
    CKF(cudaMemsetAsync(h->W, 0, (size_t)(m + 1) * h->ldw * sizeof(double), h->st));
    h->part_grid = std::max(1, std::min(h->part_cap, std::min(h->num_sms * 4, (n + STEP_THREADS - 1) / STEP_THREADS)));
    h->part_rows = (n + h->part_grid - 1) / h->part_grid;
    h->part_wb = sketch_word_bits(h->part_rows, 1);
  }
  CKF(cudaStreamSynchronize(h->st));
  {
    const krylov_status cs = choose_product_kernel(h, 0);
    if (cs != KRYLOV_OK) return fail(cs);
  }
#undef CKF
  *out = h;
  return KRYLOV_OK;
}

krylov_status krylov_create(const krylov_csr* A, krylov_func f, int m, int k, int s, uint64_t seed,
                            const krylov_options* opt_in, krylov_handle** out) {
  return create_impl(A, f, m, k, s, seed, opt_in, nullptr, out);
}

krylov_status krylov_create_partition(const krylov_csr* A_local, int64_t n_halo, int64_t row0, int64_t n_global,
                                      const int32_t* send_idx, int64_t n_send, const krylov_comm* comm,
                                      krylov_func f, int m, int k, int s, uint64_t seed,
                                      const krylov_options* opt, krylov_handle** out) {
  if (!comm) return KRYLOV_EINVAL;
  const PartSpec ps{n_halo, row0, n_global, send_idx, n_send, comm};
  return create_impl(A_local, f, m, k, s, seed, opt, &ps, out);
}

krylov_status krylov_apply(krylov_handle* h, const double* b, double* x, double tol, int max_cycles,
                           krylov_stats* st) {
  return apply_impl(h, 0, b, x, tol, max_cycles, st);
}

krylov_status krylov_apply_adjoint(krylov_handle* h, const double* b, double* x, double tol, int max_cycles,
                                   krylov_stats* st) {
  if (h && h->part_mode) return KRYLOV_EUNSUPPORTED;
  return apply_impl(h, 1, b, x, tol, max_cycles, st);
}

krylov_status krylov_apply_batched(krylov_handle* const* hs, int n_inst, int n_rhs, const double* const* B,
                                   double* const* X, const double* t_per_inst, double tol, int max_cycles,
                                   krylov_stats* st) {
  if (!hs || !B || !X || n_inst < 1 || n_rhs < 1 || max_cycles < 1 || !(tol >= 0.0)) return KRYLOV_EINVAL;
  for (int i = 0; i < n_inst; ++i) {
    if (!hs[i] || !B[i] || !X[i]) return KRYLOV_EINVAL;
    if (hs[i]->part_mode) return KRYLOV_EUNSUPPORTED;
    if (t_per_inst && !std::isfinite(t_per_inst[i])) return KRYLOV_EINVAL;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return KRYLOV_EINVAL;  // a handle is not thread-safe
  }
  std::vector<krylov_status> res((size_t)n_inst, KRYLOV_OK);
  for (int i = 0; i < n_inst; ++i) hs[i]->bk_concurrent = std::min(n_inst, 16);
  std::atomic<int> next{0};
  auto worker = [&]() {
    for (int i = next.fetch_add(1); i < n_inst; i = next.fetch_add(1))
      res[(size_t)i] = run_instance(hs[i], n_rhs, B[i], X[i], t_per_inst ? t_per_inst + i : nullptr, tol,
                                    max_cycles, st ? st + (size_t)i * n_rhs : nullptr);
  };
  const int nthreads = std::min(n_inst, 16);
  std::vector<std::thread> pool;
  pool.reserve((size_t)nthreads);
  for (int w = 0; w < nthreads; ++w) pool.emplace_back(worker);
  for (auto& th : pool) th.join();
  krylov_status out = KRYLOV_OK;
  for (int i = 0; i < n_inst; ++i) {
    if (res[(size_t)i] < 0) return res[(size_t)i];
    if (res[(size_t)i] == KRYLOV_NOT_CONVERGED) out = KRYLOV_NOT_CONVERGED;
  }
  return out;
}

krylov_status krylov_apply_host(krylov_handle* h, const double* b_host, double* x_host, double tol,
                                int max_cycles, krylov_stats* st) {
  if (!h || !b_host || !x_host) return KRYLOV_EINVAL;
  if (h->part_mode) return KRYLOV_EUNSUPPORTED;
  if (!h->stage_b) {
    CK(dalloc(h, &h->stage_b, (size_t)h->n));
    CK(dalloc(h, &h->stage_x, (size_t)h->n));
  }
  NvtxRange call_range("krylov_apply_host");
  EventPair evp;
  CK(evp.create());
  cudaEvent_t e0 = evp.a, e1 = evp.b;
  CK(cudaEventRecord(e0, h->st));
  krylov_status r = KRYLOV_ECUDA;
  if (cudaMemcpyAsync(h->stage_b, b_host, sizeof(double) * (size_t)h->n, cudaMemcpyHostToDevice, h->st) ==
      cudaSuccess) {
    r = apply_impl(h, 0, h->stage_b, h->stage_x, tol, max_cycles, st);
    if (r >= 0 && cudaMemcpyAsync(x_host, h->stage_x, sizeof(double) * (size_t)h->n, cudaMemcpyDeviceToHost,
                                  h->st) != cudaSuccess)
      r = KRYLOV_ECUDA;
  }
  cudaEventRecord(e1, h->st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  if (st) st->ms_total = ms;
  return r;
}

krylov_status krylov_set_param(krylov_handle* h, double t) {
  if (!h || !std::isfinite(t)) return KRYLOV_EINVAL;
  h->f.t = t;
  return KRYLOV_OK;
}

krylov_status krylov_spmv(krylov_handle* h, const double* x, double* y, int transpose, const double* dot_with,
                          double* dot_out) {
  if (!h || !x || !y) return KRYLOV_EINVAL;
  if (h->part_mode) return KRYLOV_EUNSUPPORTED;
  if (transpose) {
    krylov_status s = build_transpose(h);
    if (s != KRYLOV_OK) return s;
  }
  launch_spmv_f64(h->n, transpose ? h->rpt : h->rp, transpose ? h->cit : h->ci, transpose ? h->valt : h->val, x, y,
                  h->st);
  CK(cudaGetLastError());
  if (dot_with && dot_out) {
    launch_dot_f64(dot_with, y, h->n, h->part, h->grid, h->d_dot, h->cd.counter, h->st);
    CK(cudaMemcpyAsync(h->h_scal + 8, h->d_dot, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    *dot_out = h->h_scal[8];
  } else {
    CK(cudaStreamSynchronize(h->st));
  }
  return KRYLOV_OK;
}

int64_t krylov_size(const krylov_handle* h) { return h ? h->n : 0; }

krylov_status krylov_sketch_columns(int64_t n, int s, int zeta, uint64_t seed, int64_t col0, int64_t count,
                                    int32_t* rows_out, int8_t* signs_out) {
  if (n < 1 || s < 1 || s > 32768 || zeta < 1 || zeta > std::min(s, MAX_ZETA) || col0 < 0 || count < 0 ||
      col0 + count > n || col0 + count > 0xFFFFFFFFLL || !rows_out || !signs_out)
    return KRYLOV_EINVAL;
  if (count == 0) return KRYLOV_OK;
  int* drows = nullptr;
  signed char* dsigns = nullptr;
  int* derr = nullptr;
  CK(cudaMalloc(&drows, sizeof(int) * (size_t)count * zeta));
  CK(cudaMalloc(&dsigns, (size_t)count * zeta));
  CK(cudaMalloc(&derr, sizeof(int)));
  cudaMemset(derr, 0, sizeof(int));
  launch_sketch_columns(col0, count, s, zeta, seed, drows, dsigns, derr, nullptr);
  int herr = 0;
  cudaError_t e = cudaMemcpy(rows_out, drows, sizeof(int) * (size_t)count * zeta, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(signs_out, dsigns, (size_t)count * zeta, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(drows);
  cudaFree(dsigns);
  cudaFree(derr);
  if (e != cudaSuccess) return cuda_status(e);
  return herr ? KRYLOV_ECUDA : KRYLOV_OK;
}

krylov_status krylov_last_cycle(const krylov_handle* h, double* T, int64_t T_cap, double* X, int64_t X_cap,
                                double* z, int64_t z_cap, int* m_eff) {
  if (!h) return KRYLOV_EINVAL;
  if (h->last_cycle < 1) return KRYLOV_EINVAL;
  const int me = h->last_me, nc = h->last_nc, M = h->m;
  if (m_eff) *m_eff = me;
  if (T) {
    if (T_cap < (int64_t)nc * nc) return KRYLOV_EINVAL;
    std::vector<double> tw((size_t)h->s * nc);
    CK(cudaMemcpy(tw.data(), h->sd.Tw, sizeof(double) * tw.size(), cudaMemcpyDeviceToHost));
    for (int b = 0; b < nc; ++b)
      for (int a = 0; a < nc; ++a) T[(size_t)b * nc + a] = (a <= b) ? tw[(size_t)b * h->s + a] : 0.0;
  }
  if (X) {
    if (X_cap < (int64_t)me * me) return KRYLOV_EINVAL;
    std::vector<double> xb((size_t)M * M);
    CK(cudaMemcpy(xb.data(), h->sd.Xblk + (size_t)(h->last_cycle - 1) * M * M, sizeof(double) * xb.size(),
                  cudaMemcpyDeviceToHost));
    for (int b = 0; b < me; ++b)
      for (int a = 0; a < me; ++a) X[(size_t)b * me + a] = xb[(size_t)b * M + a];
  }
  if (z) {
    if (z_cap < me) return KRYLOV_EINVAL;
    CK(cudaMemcpy(z, h->sd.zg, sizeof(double) * me, cudaMemcpyDeviceToHost));
  }
  return KRYLOV_OK;
}

krylov_status krylov_probe_bounded_wait(uint64_t limit_ns, int* timed_out, double* wait_ns) {
  if (limit_ns < 1 || limit_ns > 10000000000ull || !timed_out || !wait_ns) return KRYLOV_EINVAL;
  unsigned long long* d_out = nullptr;
  CK(cudaMalloc(&d_out, 4 * sizeof(unsigned long long)));
  unsigned long long h_out[4] = {0, 0, 0, 0};
  cudaError_t e = cudaMemset(d_out, 0, 4 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = probe_bounded_wait((unsigned long long)limit_ns, d_out, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(h_out, d_out, sizeof(h_out), cudaMemcpyDeviceToHost);
  cudaFree(d_out);
  if (e != cudaSuccess) return cuda_status(e);
  for (int c = 0; c < 2; ++c) {
    timed_out[c] = (int)h_out[c];
    wait_ns[c] = (double)h_out[2 + c];
  }
  return KRYLOV_OK;
}

}  // extern "C"
