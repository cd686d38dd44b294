// internal.h -- host-side declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace krylov {

// Per-cycle device state written by the step kernels' reducers and read by the
// following kernels (all device memory, owned by the handle).
struct CycleDev {
  int* flags;      // [0] m_eff, [1] breakdown, [2] error bits, [3] spare
  double* sig2;    // (m+1) squared norms of the stored basis vectors
  double* pi;      // (m+1) squared norms of the raw products A w_j
  double* coef;    // (m+1) x (MAX_WINDOW+1): window coefficients then rho
  double* R;       // (m+1) x m column-major, leading dimension m+1
  double* scal;    // [0] eta, [1] 1/eta, [2] ||y||^2, [3] ||x||^2, [4] ||b||^2,
                   // [5] bound on ||w_1||^2 of the next cycle, [6] bound on
                   // ||w_{j+1}|| for the next materialized column (fixed-point sketch scale)
  unsigned* counter;  // arrival counters of the last-block reducers (zeroed)
  // float-float pairs of the float-float step kernels (the next kernel reads these)
  float2* sig2ff;  // (m+1) ||w_j||^2
  float2* piff;    // (m+1) ||p_j||^2
  float2* rff;     // (m+1) R[j+1, j]
};

enum : int { ERR_SKETCH = 1, ERR_NONFINITE = 2, ERR_TIMEOUT = 4 };

struct SmallDev;

// Stored sparse sign embedding (generated once per handle on the device).
struct SketchTable {
  int packed;          // 1: rows8/neg8 (s <= 255, zeta <= 8); 0: rows16/neg32
  uint2* rows8;        // n: 8 row bytes per column (0xFF = unused)
  uint8_t* neg8;       // n: sign bits (1 = -1)
  uint16_t* rows16;    // n * zeta
  uint32_t* neg32;     // n
};

// Where the step kernels take the entries of S from.
enum : int { SK_TAB8 = 0, SK_TAB16 = 1, SK_GEN8 = 2, SK_GEN = 3 };

struct StepLaunch {
  int n;
  const int* row_ptr;
  const int* col;
  const void* val;   // double or float (narrowed)
  int val_f32;       // 1 if val is float
  void* W;           // basis slots, slot stride ldw elements
  int64_t ldw;
  int j;             // column handled by this launch
  int k;             // window
  int mat;           // 1: materialize column j from p_prev; 0: column j already stored
  int spmv;          // 1: form p_j = A w_j and the window dots
  const void* p_prev;
  void* p_out;
  void* sk_part;     // sketch partials of column j: [grid][s] (double or float)
  double* part;      // scalar partials [grid][2 + MAX_WINDOW]
  double* part_w;    // float-float basis: ||w_j||^2 CTA partials, half j & 1 of [2][part_w_stride]
  int part_w_stride;
  void* sk_acc;      // float-float basis: exact sketch of column j at j * sk_acc_stride: [3][s] int64 word
  int64_t sk_acc_stride;  // sums, then E (int64); column j + 1's is zeroed by the kernel of column j
  double thr;        // breakdown threshold (relative)
  int s, zeta;
  uint64_t seed;
  int grid;          // number of CTAs (persistent)
  int rows_per_cta;
  int grid_mat;      // float-float materialize kernel: CTAs and rows per CTA (one CTA
  int rows_mat;      // per SM with the staged row streams; else grid, rows_per_cta)
  int m;             // restart length (leading dimension of R is m+1)
  SketchTable sk_tab;
  int sk_mode;       // SK_* : stored table or regeneration in the kernel
  int sk_copies;     // lane-private copies of each sketch bin in shared memory
  int fx_wb;         // bits per fixed-point word of the sketch bins
  int tma_cap;       // staged nonzeros per 256-row tile (0: no bulk-copy staging)
  const int16_t* dcol;  // [nnz + 8] col - row per nonzero when the bandwidth is below 2^15 (staged
                        // product kernel: 2 bytes per column instead of 4), else null
  // Rows too long for a row per thread (power-law operators, float-float
  // basis): row_ptr/col/val above then describe a copy of the operator with
  // these rows emptied, whose product kernel gives p_i = 0 there (no dot
  // contribution) and leaves the reduction to ff_spmv_long_kernel, which forms
  // the long rows from the full operator with a CTA per row and reduces.
  int n_long;                 // 0: no long rows (everything below is unused)
  int n_big;                  // the first n_big long rows take a CTA each, the others a warp each
  const int* long_rows;       // [n_long] row indices, longest first
  const int* rp_full;         // full operator
  const int* col_full;
  const void* val_full;       // float or float2 like val
  int grid_long;              // CTAs of the long-row kernel
  double* part_long;          // [grid_long][2 + MAX_WINDOW] its scalar partials
  int grid_spmv;     // CTAs of the separate product kernel (float-float basis)
  int rows_spmv;     // rows per CTA of that kernel (a multiple of 256)
  int rgs;           // 1: randomized Gram-Schmidt cycle (the product kernel forms p and ||p||^2 only)
  // segment plan of the operator (float-float basis; seg null: no plan): per
  // 256-row tile the contiguous pieces of w_j that its columns touch and, per
  // nonzero, the 16-bit position of its column among the staged pieces
  const int4* seg;          // [tiles][SEG_MAX]: start, length, offset, unused
  const int* seg_n;         // [tiles] pieces per tile
  const uint16_t* lcol;     // [nnz + 16] tile-local column positions
  int seg_cap;              // max staged entries of w_j per tile (even)
  int lcap;                 // max aligned nonzero span per tile (multiple of 8)
  // sliced layout of the operator (float-float basis; sell_col null: none):
  // 256-row tile g holds entries [sell_off[g], sell_off[g + 1]) of sell_col /
  // sell_val, padded to the tile's longest row, entry q of row r at q * 256 + r
  const int* sell_off;      // [tiles + 1]
  int sell_maxl;            // longest row of any tile (sizes the product kernel's stages)
  const int16_t* sell_col;  // col - row (padding: 0)
  const void* sell_val;     // float or float2 like val (padding: 0)
};

constexpr int SELL_MAXL = 16;  // longest row of a tile in the sliced layout

constexpr int SEG_MAX = 16;        // pieces of w_j per tile
constexpr int SEG_CAP_MAX = 3072;  // staged entries of w_j per tile (24 KB float-float)
constexpr int SEG_GAP = 64;        // columns closer than this join one piece

// Per-right-hand-side strides (in elements) of the small-problem and cycle
// arrays when several independent problems are laid out one after another
// (the block form); all zero for one problem.
struct BatchStride {
  int64_t U, Tw, Tinv, zg, Xblk, gam, misc, G, S0, fcol;  // SmallDev arrays
  int64_t flags, sig2, pi, coef, R, scal;                 // CycleDev arrays
};

// Arguments of the block-form kernels (nb right-hand sides of one matrix,
// vectors row-major n x nb, float-float basis).
struct BlockLaunch {
  int n, nb, m, k, s, zeta, j;
  const int* rp;
  const int* ci;
  const void* val;
  int val_f32;
  void* W;              // (m+1) slots of n x nb: float2 (float-float) or float (basis32)
  int64_t slot;         // n * nb
  const void* p_prev;   // products, same element type as W
  void* p_out;
  int basis32;          // 1: float32 storage of the basis and products (float-float arithmetic)
  double* part;         // per-CTA partials [grid][NQ][64]
  CycleDev cd;          // right-hand side 0's cycle state; others at offsets bs
  BatchStride bs;
  unsigned* counter;
  long long* acc;       // [m+1][3][s][64] exact sketch sums
  int* E;               // [m+1][64] fixed-point exponents of the sketch words
  SketchTable tab;
  int grid, rows_per_cta, fx_wb;   // materialize/sketch kernel (and norms)
  int grid_p, rows_p;              // product and update kernels
  double thr;
};

// Arguments of the randomized Gram-Schmidt cycle kernels (Algorithm 1).
struct RgsArgs {
  int n, m, k, s, zeta;
  int grid, rows_per_cta;   // sketch / materialize kernels
  int sk_mode, copies, fx_wb;
  int basis;                // 0 float64, 3 float-float
  int64_t ldw;
  uint64_t seed;
  SketchTable sk_tab;
  void* W;                  // basis slots
  double* part;             // per-CTA partials
  long long* acc;           // [3][s] exact fixed-point sums over CTAs (zero between uses)
  double* U;                // s x (m+1) sketched basis, column-major (U_j = S w_j)
  double* misc;             // small-problem scalars ([0] beta)
  double thr;               // breakdown threshold relative to ||S A w_j||
};

// basis dtype codes (krylov_basis)
int spmv_ctas_per_sm(int vals_f32, int tma_cap, int seg_cap, int lcap);
int sell_ctas_per_sm(int vals_f32, int maxl);
size_t sell_smem_bytes(int vals_f32, int maxl);  // dynamic shared memory of the float-float sliced product
int step_ctas_per_sm(int basis, int sk_mode, int s, int copies, int vals_f32);
int mat_ctas_per_sm(int s, int copies);
void launch_step(int basis, const StepLaunch& L, const CycleDev& cd, int m, cudaStream_t st);
// float32 / bfloat16 bases with staged row streams (step32_kernels.cu): the
// materialize+sketch kernel and the product kernel of step L.j
size_t s32_mat_smem(int s, int copies, int kw, int vt_bytes);
int s32_ctas_per_sm(int basis, int s, int copies);
int s32_spmv_ctas_per_sm(int tma_cap, int di);
int s32_sell_ctas_per_sm();
void launch_step32(int basis, const StepLaunch& L, const CycleDev& cd, cudaStream_t st);
// float-float product kernel alone (p_j = A w_j, window dots unless L.rgs)
void launch_ff_product(const StepLaunch& L, const CycleDev& cd, cudaStream_t st);
// randomized Gram-Schmidt cycle (rgs_kernels.cu)
void launch_rgs_start(const RgsArgs& a, const CycleDev& cd, int cycle, cudaStream_t st);
void launch_rgs_product_f64(const StepLaunch& L, const CycleDev& cd, cudaStream_t st);
void launch_rgs_orth(const RgsArgs& a, const CycleDev& cd, const void* p, int j, cudaStream_t st);
void launch_rgs_mat(const RgsArgs& a, const CycleDev& cd, const void* p, int j, cudaStream_t st);
void launch_rgs_small(const SmallDev& sd, const CycleDev& cd, int m, int me, int has_next, int cycle, double t,
                      cudaStream_t st);
void launch_norm_b(const double* b, int n, double* part, int grid, const CycleDev& cd, cudaStream_t st);
void launch_start(int basis, const double* b, void* W0, int n, const CycleDev& cd, int grid,
                  cudaStream_t st);
void launch_update(int basis, void* W, int64_t ldw, int n, int m_eff, int has_next,
                   const double* zg, double* x, double* part, int grid, const CycleDev& cd, int m,
                   cudaStream_t st);
void launch_sketch_reduce(const void* sk_part, int ncols, int grid, int s, int zeta, int64_t col_stride,
                          double* U, cudaStream_t st);
void launch_spmv_f64(int n, const int* row_ptr, const int* col, const double* val, const double* x,
                     double* y, cudaStream_t st);
void launch_dot_f64(const double* a, const double* b, int n, double* part, int grid, double* out,
                    unsigned* counter, cudaStream_t st);
void launch_sketch_columns(int64_t col0, int64_t count, int s, int zeta, uint64_t seed, int* rows,
                           signed char* signs, int* err, cudaStream_t st);
// table entry i holds column col0 + i of S (a rank's rows in a partitioned solve)
void launch_sketch_table(int n, int s, int zeta, uint64_t seed, const SketchTable& tab, int* err,
                         cudaStream_t st, int64_t col0 = 0);
int sketch_bin_copies(int basis, int s);
int sketch_word_bits(int rows_per_cta, int copies);

// one CTA runs the bounded mbarrier wait on a completing and a never-completing
// phase; d_out (4 values): gave-up flags, then durations in ns
cudaError_t probe_bounded_wait(unsigned long long limit_ns, unsigned long long* d_out, cudaStream_t st);

// ---- handle creation ------------------------------------------------------
// column indices must lie in [0, ncols) (ncols <= 0: [0, n))
cudaError_t validate_csr(int n, int64_t nnz, const int* rp, const int* ci, int* d_flag, int* h_flag,
                         cudaStream_t st, int ncols = 0);
cudaError_t narrow_values(int64_t nnz, const double* v, float* v32, int* d_flag, int* h_flag,
                          cudaStream_t st);
cudaError_t raise_smem_limit(const void* kern, size_t bytes);
cudaError_t norm_inf(int n, const int* rp, const double* val, int* d_flag, int* h_flag, double* out,
                     cudaStream_t st);
cudaError_t tile_span_max(int n, const int* rp, int* d_flag, int* h_flag, cudaStream_t st);
// max |col - row| over the nonzeros into h_flag[0] (synchronizes st)
cudaError_t csr_bandwidth(int n, const int* rp, const int* ci, int* d_flag, int* h_flag, cudaStream_t st);
// dcol[e] = col[e] - row(e); the caller has checked the bandwidth is below 2^15
cudaError_t csr_delta16(int n, const int* rp, const int* ci, int16_t* dcol, cudaStream_t st);
cudaError_t split_values(int64_t nnz, const double* v, float2* vff, cudaStream_t st);
cudaError_t transpose_csr(int n, int64_t nnz, const int* rp, const int* ci, const double* v, int* rpt,
                          int* cit, double* vt, int* work, cudaStream_t st);
// acc0 / n_acc0: the exact sketch accumulator of column 0 (float-float basis), zeroed here
void launch_cycle_reset(const CycleDev& cd, int m, cudaStream_t st, void* acc0 = nullptr, int n_acc0 = 0);
// U from the exact int64 sketches of the float-float materialize kernels
void launch_sketch_finish(const void* acc, int ncols, int s, int64_t col_stride, int wb, int zeta, double* U,
                          cudaStream_t st);
void launch_gather_column(const double* B, int64_t n, int ncols, int r, double* b, cudaStream_t st);
void launch_zero_columns(double* X, int64_t n, int64_t ld, int ncols, cudaStream_t st);
void launch_scatter_column(const double* x, int64_t n, int ncols, int r, double* X, cudaStream_t st);

// ---- small projected problem (FP64) ---------------------------------------
struct SmallDev {
  double* U;       // s x (m+1) sketched basis (column-major)
  double* Tw;      // s x (m+1) Householder work / T on output (leading dim s)
  double* Tinv;    // m x m
  double* zg;      // [0,m) z, [m,2m) g, [2m] 1/tau
  double* Xblk;    // cycles x (m x m): diagonal blocks X^{(c)}
  double* gam;     // cycles: coupling gamma^{(c)} between block c and c+1
  double* misc;    // [0] beta, [1] rho of the last cycle, [2] ||tX||_1 of the last cycle,
                   // [3] |t gamma| of the last coupling, [4] kappa estimate of T,
                   // [5] last entry of the previous inverse block solve (f = 1/z)
  double* G;       // exp block rows, all scale levels
  double* S0;      // Horner ping-pong buffers (2 x cycles x m x m)
  double* fcol;    // m: first column of the last block row of f(H)
  double* qcarry;  // z^{-1/2}: per quadrature node, last entry of the previous block solve
  double* qpart;   // z^{-1/2}: nodes x m weighted block solutions
  double* qwork;   // z^{-1/2}: nodes x m x m LU work when it does not fit in shared memory
  double* gphi;    // phi_1: per scale level and block row, the m-vector of the augmented
                   // exponential's extra column (levels x cycles x m)
  double* qstat;   // exp by contour quadrature: [0] sigma, [1] largest |entry| of the first
                   // column so far, [2] difference to scaling and squaring, [3] difference
                   // between the two contours (both relative to [1])
};

// z^{-1/2} quadrature nodes keep their m x m LU work in shared memory up to this size.
constexpr size_t INVSQRT_SMEM_MAX = 100 * 1024;
size_t invsqrt_smem(int m);
// exp(-t z) by contour quadrature (small_kernels.cu): complex m x m LU work per
// point in shared memory up to this size, else in sd.qwork (points x m x m complex)
constexpr size_t EXP_QUAD_SMEM_MAX = 200 * 1024;
size_t exp_quad_smem(int m);
int exp_quad_nodes();
void launch_exp_quad_sigma(const SmallDev& sd, int m_eff, double t, const double* fsq, cudaStream_t st);
// block row a of the first column of exp(-t H) into sd.fcol (fsq: the
// scaling-and-squaring block to compare with, or null)
void launch_exp_quad(const SmallDev& sd, const CycleDev& cd, int m, int m_eff, int a, double t, const double* fsq,
                     cudaStream_t st);

__host__ __device__ inline SmallDev offset_sd(SmallDev sd, const BatchStride& b, int r) {
  sd.U += b.U * r;
  sd.Tw += b.Tw * r;
  sd.Tinv += b.Tinv * r;
  sd.zg += b.zg * r;
  sd.Xblk += b.Xblk * r;
  sd.gam += b.gam * r;
  sd.misc += b.misc * r;
  sd.G += b.G * r;
  sd.S0 += b.S0 * r;
  sd.fcol += b.fcol * r;
  return sd;
}
__host__ __device__ inline CycleDev offset_cd(CycleDev cd, const BatchStride& b, int r) {
  cd.flags += b.flags * r;
  cd.sig2 += b.sig2 * r;
  cd.pi += b.pi * r;
  cd.coef += b.coef * r;
  cd.R += b.R * r;
  cd.scal += b.scal * r;
  return cd;
}

// Batched small problem (block form): one problem per cluster (whiten), per
// CTA (z) or per grid z-slice (exp), problems r = 0..nb-1 at offsets r * stride.
// kw: window of the truncated recurrence (band of R_m).
// concurrent: such batched launches running at once on other streams
void launch_whiten_batched(const SmallDev& sd, const CycleDev& cd, const BatchStride& bs, int nb, int concurrent,
                           int s, int m, int ncols, int m_eff, int has_next, int cycle, int kw, double t,
                           cudaStream_t st);
void launch_exp_taylor_batched(const SmallDev& sd, const BatchStride& bs, int nb, int m, int a, int kdeg,
                               double scale, int first, int src, double* dst0, int dst_in_g, cudaStream_t st);
void launch_exp_square_batched(const SmallDev& sd, const BatchStride& bs, int nb, int m, int a, int level,
                               int64_t level_stride, cudaStream_t st);
void launch_z_batched(const SmallDev& sd, const BatchStride& bs, int nb, int m, int m_eff, const double* fcol0,
                      int64_t fcol_stride, cudaStream_t st);

// block form (block_kernels.cu)
size_t bk_mat_smem(int s, int nb);
int bk_ctas_per_sm(int kernel, size_t smem);  // 0: materialize/sketch, 1: product, 2: update
void launch_bk_norm_start(const BlockLaunch& B, const double* b, int64_t ldb, cudaStream_t st);
void launch_bk_step(const BlockLaunch& B, int mat, int spmv, cudaStream_t st);
void launch_bk_sketch_fin(const BlockLaunch& B, const SmallDev& sd, int ncols, cudaStream_t st);
void launch_bk_update(const BlockLaunch& B, const SmallDev& sd, int m_eff, int has_next, double* x, int64_t ldx,
                      const int* active, cudaStream_t st);

// ---- row-partitioned solve (part_kernels.cu) --------------------------------
// One rank's block of n rows; its CSR columns index [0, n + halo): the local
// rows, then the halo entries of the current basis vector.
struct PartLaunch {
  int n;
  const int* rp;
  const int* ci;
  const double* val;
  double* W;            // basis slots (float64), stride ldw >= n + halo
  int64_t ldw;
  double* p;            // product of the current step (n)
  double* part;         // per-CTA partials (grid x NQ)
  double* red;          // all-reduced sums: [0, NQ) product, [NQ] ||w_j||^2
  long long* acc;       // [m+1][3][s] exact sketch word sums (zeroed per cycle)
  int* E;               // [m+1] fixed-point exponent of each column's words
  int grid, rows_per_cta;
};
size_t part_mat_smem(int s);
void launch_part_pack(const double* w, const int* idx, int count, double* out, cudaStream_t st);
void launch_part_unpack(const double* in, int count, double* w_halo, cudaStream_t st);
void launch_part_norm_finish(const CycleDev& cd, cudaStream_t st);
void launch_part_mat(const PartLaunch& P, const StepLaunch& L, const CycleDev& cd, int mat, cudaStream_t st);
void launch_part_product(const PartLaunch& P, const StepLaunch& L, const CycleDev& cd, cudaStream_t st);
void launch_part_reduce_mat(const StepLaunch& L, const CycleDev& cd, const double* red, int mat, cudaStream_t st);
void launch_part_reduce_product(const StepLaunch& L, const CycleDev& cd, const double* red, cudaStream_t st);
void launch_part_sketch_u(const long long* acc, const int* E, int ncols, int s, int zeta, int wb, double* U,
                          cudaStream_t st);

void launch_whiten(const SmallDev& sd, const CycleDev& cd, int s, int m, int ncols, int m_eff,
                   int has_next, int cycle, int kw, double t, cudaStream_t st);
// One Horner step S <- S B kinv + I for block row a (B = scale H).
// gout (phi_1, else null): where the last step stores the Taylor polynomial's
// extra column for block row a, scaled by gscale = 2^-s
void launch_exp_taylor_step(const SmallDev& sd, int m, int a, double kinv, double scale, int first,
                            int last, int src, double* dst, double* gout, double gscale, cudaStream_t st);
// gi/go (phi_1, else null): the phi_1 vectors of block rows 0..a at the input
// level and of block row a at the output level; dbl (cos(t sqrt(z))): the
// double-angle step 2 C^2 - I instead of a square
void launch_exp_square(const SmallDev& sd, int m, int a, int level, int64_t level_stride, const double* gi,
                       double* go, int dbl, cudaStream_t st);
void launch_inv_block(const SmallDev& sd, int m, int m_eff, int a, cudaStream_t st);
void launch_invsqrt_block(const SmallDev& sd, const CycleDev& cd, int m, int m_eff, int a, double u0, double hq,
                          int nodes, cudaStream_t st);
void launch_z(const SmallDev& sd, int m, int m_eff, const double* fcol_src, cudaStream_t st);

}  // namespace krylov
