/*
 * krylov.h -- C ABI of the GB300 randomized restarted Krylov library for f(A) b.
 *
 * Method: Guidotti, Martinsson, Acebron, Monteiro, "Accelerating a restarted
 * Krylov method for matrix functions with randomization" (arXiv 2503.22631).
 * The library approximates f(A) b for a square sparse A (CSR), a vector b and
 * f analytic on the spectrum of A (Sec. 1), by restart cycles of m Arnoldi-like
 * steps (Sec. 4, Algorithm 2).  Each step is one sparse matrix-vector product,
 * an orthogonalization of the new vector against the last k basis vectors, and
 * one sparse-sign sketch of the stored vector (Sec. 2.1, Eq. 3).  Each cycle
 * ends with the sketched small problem in FP64: a thin QR of the sketched
 * basis (basis whitening, App. A, Eq. A.1), f of the block lower-bidiagonal
 * projected matrix (Algorithm 2), and one streaming solution update.
 *
 * Conventions for every call:
 *  - Pointers named "device" are CUDA device pointers on the current device;
 *    pointers named "host" are ordinary host memory.  All vectors are dense,
 *    contiguous float64 of length n unless stated.
 *  - Work is issued on the handle's stream (krylov_options.stream, NULL =
 *    legacy default stream).  Calls return after the result is complete
 *    (the library synchronizes the stream at cycle boundaries).
 *  - No call throws; errors are returned as krylov_status.  Negative codes are
 *    errors (outputs unspecified), positive codes are informational (outputs
 *    hold the last iterate).
 *  - A handle is not thread-safe: one call at a time per handle.
 *  - Every entry point fails with KRYLOV_ECUDA when the CUDA runtime reports an
 *    error, and never falls back to host computation.
 */
#ifndef KRYLOV_H
#define KRYLOV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct krylov_handle krylov_handle; /* opaque, owned by the library */

typedef enum {
  KRYLOV_OK = 0,
  KRYLOV_NOT_CONVERGED = 1,   /* max_cycles reached before ||y|| <= tol ||x||   */
  KRYLOV_BREAKDOWN_EXACT = 2, /* happy breakdown: invariant subspace, x exact   */
  KRYLOV_EINVAL = -1,         /* invalid argument (sizes, CSR structure, ...)   */
  KRYLOV_ENOMEM = -2,         /* device allocation failed                       */
  KRYLOV_ECUDA = -3,          /* CUDA runtime / launch error                    */
  KRYLOV_ENONFINITE = -4,     /* NaN/Inf in b or in the projected problem       */
  KRYLOV_ETIMEOUT = -5,       /* a bounded device wait gave up (result invalid) */
  KRYLOV_EUNSUPPORTED = -6    /* option combination not implemented             */
} krylov_status;

/* f(z); exp(-t z) is Eq. (19)'s heat kernel and the exponential of Sec. 5.1 with
 * the time folded in; phi_1(-t z) = (1 - e^{-t z}) / (t z) is the phi function of
 * Sec. 5 (u(t) = u_0 + t phi_1(-L t) b for the convection-diffusion problem with a
 * constant load); cos(t sqrt(z)) is the membrane example of Sec. 5 (the wave
 * equation u'' = -L u); z^{-1/2} and 1/z are extensions (Stieltjes functions). */
typedef enum {
  KRYLOV_F_EXP_NEG = 0,  /* f(z) = exp(-t z) */
  KRYLOV_F_INVSQRT = 1,  /* f(z) = z^{-1/2}  */
  KRYLOV_F_INV = 2,      /* f(z) = 1/z       */
  KRYLOV_F_PHI1_NEG = 3, /* f(z) = phi_1(-t z) = (1 - e^{-t z}) / (t z); phi_1(0) = 1 */
  KRYLOV_F_COS_SQRT = 4  /* f(z) = cos(t sqrt(z)) (an entire function of z) */
} krylov_fkind;

typedef struct {
  int kind;  /* krylov_fkind */
  double t;  /* t of exp(-t z), phi_1(-t z) and cos(t sqrt(z)); finite (EINVAL
                otherwise); ignored by z^{-1/2} and 1/z */
} krylov_func;

/* CSR matrix, borrowed for the duration of krylov_create (the library copies
 * it); 1 <= n <= 2^31 - 2^20 and 0 <= nnz <= 2^31 - 16, else KRYLOV_EINVAL.
 * row_ptr: n+1 int32, monotone, row_ptr[0] = 0, row_ptr[n] = nnz;
 * col_idx: nnz int32 in [0, n); val: nnz float64.  on_device != 0 means the
 * three arrays are device pointers, else host pointers.  (App. A: CSR.) */
typedef struct {
  int64_t n;
  int64_t nnz;
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const double* val;
  int on_device;
} krylov_csr;

/* Storage and arithmetic of the Krylov basis and the step vectors:
 *   F64   float64 storage, float64 arithmetic (reference precision);
 *   F32   float32 storage and arithmetic (float64 across-CTA sums);
 *   BF16  bfloat16 storage, float32 arithmetic;
 *   DF64  float-float storage (hi + lo float pairs, ~48-bit significand, 8 bytes)
 *         with float-float products, orthogonalization and sketches on the
 *         float32 pipes: FP64-class accuracy without float64 arithmetic in the
 *         streaming kernels. */
typedef enum {
  KRYLOV_BASIS_F64 = 0,
  KRYLOV_BASIS_F32 = 1,
  KRYLOV_BASIS_BF16 = 2,
  KRYLOV_BASIS_DF64 = 3
} krylov_basis;
/* Orthogonalization of a cycle:
 *   TRUNC  classical Gram-Schmidt against the last k stored vectors, then the
 *          sketched basis is whitened (App. A, Eq. A.1) for the restart;
 *   RGS    Algorithm 1: Gram-Schmidt in sketch space against the last k
 *          sketches (all of them when k >= m: the paper's randomized restart),
 *          one basis update per step; float64 and float-float bases only
 *          (KRYLOV_EUNSUPPORTED otherwise). */
typedef enum { KRYLOV_ORTHO_TRUNC = 0, KRYLOV_ORTHO_RGS = 1 } krylov_ortho;

typedef struct {
  int zeta;        /* nonzeros per sketch column (Eq. 3); 1 <= zeta <= min(s, 32). Default 8 */
  int basis_dtype; /* krylov_basis: storage of the Krylov basis and step vectors. Default F64 */
  int ortho;       /* krylov_ortho: TRUNC (default) or RGS */
  int narrow_values_if_exact; /* F64 basis: stream A's values as float32 when every value
                                 round-trips exactly (lossless). Default 1 */
  int use_graph;   /* capture the m steps of a cycle in a CUDA graph. Default 1 */
  int abs_tol;     /* 1: stop when ||y|| <= tol (Algorithm 2 as printed);
                      0: stop when ||y|| <= tol * ||x|| (default) */
  int sketch_regenerate; /* 0 (default): S is generated once at create into a device table
                            (9 bytes per column when s <= 255 and zeta <= 8) that the step
                            kernels read; 1: the step kernels regenerate every column of S
                            with the counter-based generator instead (no table, more
                            arithmetic per step).  Both give bit-identical S. */
  void* stream;    /* cudaStream_t for all work; NULL = legacy default stream */
  int autotune;    /* float-float basis: 1 (default) times the two product kernels on the
                      operator at create (w_j pieces staged in shared memory from a per-tile
                      segment plan, or w_j gathered through L1/L2) and keeps the staged
                      pieces only when they are faster by more than 3 %; 0 uses the staged
                      pieces whenever the operator has a segment plan; 2 always gathers
                      (a fixed kernel choice, e.g. for profiling); other values: EINVAL */
  int block_rhs;   /* batched form: 1 (default) advances up to 64 right-hand sides of a matrix
                      together through the block kernels (float-float or float32 basis, TRUNC,
                      exp, packed sketch table, m <= 64, max_cycles <= 16); 0 solves them one by
                      one */
} krylov_options;

typedef struct {
  int cycles;              /* restart cycles run */
  int breakdown;           /* 1 if the last cycle ended in a happy breakdown */
  int steps;               /* Arnoldi steps (sparse products) run */
  double last_update_norm; /* ||y|| of the last cycle (Sec. 4 error estimate) */
  double x_norm;           /* ||x|| after the last cycle */
  double kappa_T_max;      /* max over cycles of cond_1 estimate of T (whitening) */
  double ms_total;         /* wall time of the call measured with CUDA events */
  double bytes_moved;      /* algorithmic HBM bytes of the call (roofline model) */
  int launches;            /* kernels launched by the call */
  int step_launches;       /* launches of the fused step kernel */
  double ms_steps;         /* device time of the step-kernel phases (CUDA events) */
  double step_bytes;       /* algorithmic HBM bytes of those phases */
  int status;              /* krylov_status of the call (per right-hand side in the batched form) */
  int fquad_cycles;        /* exp(-t z): cycles whose block of f(H) came from the contour quadrature
                              alone (the cycle count beyond which scaling and squaring stops) */
  double ms_small;         /* device time of the small-problem phases (sketch sums, whitening, f of
                              the projected matrix, z) */
} krylov_stats;

/* Fill *opt with the defaults listed above. */
void krylov_options_default(krylov_options* opt);

/* Create a handle: copy A to the device, validate it (EINVAL on a non-monotone
 * row_ptr or a column index out of range), fix the sketch S from (s, zeta,
 * seed) and allocate the cycle workspaces (m+1 basis vectors, two product
 * vectors, the s x (m+1) sketch, the projected-problem history).
 *   f      : the function and its parameter;
 *   m      : restart length (Algorithm 2), 1 <= m <= 256;
 *   k      : orthogonalization window: 1 <= k <= 4 with TRUNC (Sec. 5:
 *            incomplete orthogonalization against the last k vectors),
 *            1 <= k <= m with RGS (k = m: full sketch orthogonalization);
 *   s      : sketch rows d of Eq. (3), m+1 <= s <= 1024;
 *   seed   : keys the counter-based generator of S;
 *   opt    : may be NULL (defaults);
 *   out    : receives the handle (owned by the caller, free with krylov_destroy). */
krylov_status krylov_create(const krylov_csr* A, krylov_func f, int m, int k, int s,
                            uint64_t seed, const krylov_options* opt, krylov_handle** out);

/* Row-partitioned solve (one process per GPU).  A rank owns a contiguous
 * block of rows of A and the same rows of b and x.  Per Arnoldi step the
 * ranks exchange the halo of the current basis vector (the entries of other
 * ranks' rows that their rows reference) and sum k + 2 scalars (||A w_j||^2
 * and the window dots of Algorithm 1's loop body, then ||w_{j+1}||^2); the
 * sketch columns are keyed by global row, so the sketch of a basis vector is
 * the sum over ranks of their rows' sketches (Sec. 2.1, Eq. 3 applied
 * columnwise), summed exactly once per cycle.  The small projected problem is
 * solved redundantly on every rank from identical inputs; the solution update
 * x += W z stays local.  The library calls back into the caller for every
 * exchange (see krylov_comm); the callbacks must be collective: every rank
 * calls them in the same order with the same counts. */
typedef struct {
  void* ctx;  /* passed back unchanged */
  /* in-place sum over all ranks of count float64 values at the DEVICE pointer
   * buf; work already issued on `stream` must complete first, and the sum must
   * be complete (visible on `stream`) when the callback returns.  0 = success. */
  int (*allreduce_sum_f64)(void* ctx, double* buf, int64_t count, void* stream);
  /* same for int64 values (exact integer sums) */
  int (*allreduce_sum_i64)(void* ctx, int64_t* buf, int64_t count, void* stream);
  /* in-place maximum over all ranks of count float64 values (device) */
  int (*allreduce_max_f64)(void* ctx, double* buf, int64_t count, void* stream);
  /* halo exchange: send (device, n_send values, in the order of the send_idx
   * given at create) goes to the neighbours, recv (device, n_halo values, in
   * the order of the halo columns n .. n + n_halo - 1) is filled from them */
  int (*halo_exchange_f64)(void* ctx, const double* send, double* recv, void* stream);
} krylov_comm;

/* Create this rank's handle of a row-partitioned solve.
 *   A_local : the rank's rows (A->n = n_local rows) with columns renumbered:
 *             [0, n_local) are the rank's own rows, [n_local, n_local + n_halo)
 *             the halo columns in the order the exchange delivers them
 *             (borrowed, copied; EINVAL on a column outside that range);
 *   row0    : global index of local row 0 (keys the sketch columns);
 *   n_global: rows of the whole matrix;
 *   send_idx: host, n_send local row indices whose entries the neighbours
 *             need, in the order the exchange sends them;
 *   comm    : collective callbacks (copied; ctx must outlive the handle);
 *   f, m, k, s, seed, opt : as for krylov_create, with the float64 basis and
 *             TRUNC orthogonalization (EUNSUPPORTED otherwise).
 * krylov_apply on such a handle takes the rank's rows of b and x and is
 * collective.  krylov_apply_adjoint, krylov_apply_batched, krylov_spmv and
 * krylov_apply_host return EUNSUPPORTED on it. */
krylov_status krylov_create_partition(const krylov_csr* A_local, int64_t n_halo, int64_t row0, int64_t n_global,
                                      const int32_t* send_idx, int64_t n_send, const krylov_comm* comm,
                                      krylov_func f, int m, int k, int s, uint64_t seed,
                                      const krylov_options* opt, krylov_handle** out);

/* x <- approximation of f(A) b by Algorithm 2 (with the whitened restart of
 * App. A).  b: device, n float64, read only; x: device, n float64, overwritten.
 * tol: stopping tolerance (relative unless opt.abs_tol); tol = 0 runs exactly
 * max_cycles cycles.  st may be NULL.  Returns OK, NOT_CONVERGED or
 * BREAKDOWN_EXACT on success; EINVAL for a NULL h, b or x, max_cycles < 1 or
 * tol < 0 (or NaN); ENONFINITE when b or the projected problem holds NaN/Inf;
 * ETIMEOUT when a bounded device wait gave up. */
krylov_status krylov_apply(krylov_handle* h, const double* b, double* x, double tol,
                           int max_cycles, krylov_stats* st);

/* Same as krylov_apply with b and x in HOST memory; the copies to and from the
 * device are part of the call (and of st->ms_total). */
krylov_status krylov_apply_host(krylov_handle* h, const double* b_host, double* x_host,
                                double tol, int max_cycles, krylov_stats* st);

/* x <- f(A)^T b = f(A^T) b for real A and real-coefficient f: the same method on
 * the transposed CSR, which is built on the device on first use and cached.
 * Arguments as for krylov_apply. */
krylov_status krylov_apply_adjoint(krylov_handle* h, const double* b, double* x, double tol,
                                   int max_cycles, krylov_stats* st);

/* Change the parameter t of f for subsequent calls (e.g. exp(-t z) at a new t).
 * EINVAL for a NULL handle or a non-finite t. */
krylov_status krylov_set_param(krylov_handle* h, double t);

/* y <- A x (transpose = 0) or A^T x (transpose = 1).  x, y: device float64, n.
 * If dot_with is not NULL, also *dot_out (host) <- <dot_with, y>.  Used for the
 * derivative in t of exp(-tA) b (d/dt = -A exp(-tA) b). */
krylov_status krylov_spmv(krylov_handle* h, const double* x, double* y, int transpose,
                          const double* dot_with, double* dot_out);

/* y <- A x and, if dot_with is not NULL, *dot_out <- <dot_with, y>, without
 * allocating anything.  The paper has no counterpart: this is for callers that
 * cannot allocate device memory when they need the product -- numerical code
 * called back from inside a custom device allocator or memory pool (a nested
 * allocation would re-enter it) and real-time loops in which cudaMalloc may
 * block or synchronize the device.  Unlike
 * krylov_spmv it needs no handle: row_ptr (n+1), col_idx, val (nnz, float64),
 * x, y (n) and dot_with, dot_out (n and 1 element) are caller-owned DEVICE
 * pointers (dot_with and dot_out both NULL or both set); stream is a
 * cudaStream_t (NULL = legacy default stream).  The call is asynchronous on
 * that stream; it does not validate the CSR structure (krylov_create does).
 * Scratch: a fixed 16 KiB device array inside the library, shared by all
 * calls on a device and kept until the process exits; the first call on a
 * device looks its address up (make it before any stream capture: a first
 * call on a capturing stream returns KRYLOV_EINVAL), and calls that overlap
 * on the GPU race on it (serialize them).  The grid is capped at 2048 CTAs,
 * rows per CTA grow with n.  Limits: 1 <= n <= 2^31 - 2,
 * 0 <= nnz <= 2^31 - 1, else KRYLOV_EINVAL. */
krylov_status krylov_spmv_dot_noalloc(int64_t n, int64_t nnz, const int32_t* row_ptr,
                                      const int32_t* col_idx, const double* val, const double* x,
                                      double* y, const double* dot_with, double* dot_out,
                                      void* stream);

/* Problem size n of a handle (0 for NULL). */
int64_t krylov_size(const krylov_handle* h);

/* Release the handle and all device memory it owns.  NULL is ignored. */
void krylov_destroy(krylov_handle* h);

/* Batched form: f(A_i) b_{i,r} for n_inst handles (matrices of uneven size) and
 * n_rhs right-hand sides each.  Algorithm 2 runs independently for every
 * (instance, right-hand side); instances run concurrently, each on a stream of
 * its own that is ordered after the handle's stream on entry and before it on
 * return, with one host worker thread per instance (at most 16 at a time).
 *   hs         : n_inst distinct handles (one matrix each);
 *   B[i], X[i] : device float64, row-major n_i x n_rhs (column r is b_{i,r} and
 *                x_{i,r}); X[i] is overwritten;
 *   t_per_inst : NULL, or n_inst finite values of the parameter t of each
 *                handle's f (the handle's t is restored afterwards);
 *   st         : NULL, or n_inst * n_rhs stats, entry i * n_rhs + r, each with its
 *                own status.
 * Every right-hand side is attempted; one that fails (a negative status in its
 * stats, its column of X unspecified) does not stop the others, except for a
 * CUDA or allocation error, which ends its instance.  Returns the first negative
 * status met (instances in order), else KRYLOV_NOT_CONVERGED if any right-hand
 * side did not meet tol, else KRYLOV_OK.
 * EINVAL for null or repeated handles, null B or X, n_inst < 1, n_rhs < 1,
 * max_cycles < 1, tol < 0 or a non-finite t. */
krylov_status krylov_apply_batched(krylov_handle* const* hs, int n_inst, int n_rhs, const double* const* B,
                                   double* const* X, const double* t_per_inst, double tol, int max_cycles,
                                   krylov_stats* st);

/* Static description of a status code ("unknown status" for other values). */
const char* krylov_status_string(krylov_status s);

/* ---- inspection entry points used by the parity tests ------------------ */

/* Sparse sign columns [col0, col0 + count) of S as generated on the device
 * (Sec. 2.1, Eq. 3): rows_out (host, count*zeta int32) and signs_out (host,
 * count*zeta int8, +1/-1), entries of a column in acceptance order.  The same
 * generator feeds every sketch the library computes.  EINVAL unless
 * 1 <= s <= 32768, 1 <= zeta <= min(s, 32), col0 >= 0, count >= 0,
 * col0 + count <= n and both outputs are set; count = 0 writes nothing. */
krylov_status krylov_sketch_columns(int64_t n, int s, int zeta, uint64_t seed, int64_t col0,
                                    int64_t count, int32_t* rows_out, int8_t* signs_out);

/* Matrices of the last cycle run by h (host copies, column-major):
 * T (s_cols x s_cols, s_cols = m_eff + 1 or m_eff after a breakdown),
 * X (m_eff x m_eff, Eq. A.1), z (m_eff coefficients of the update
 * x += W_m z) and m_eff itself.  Any output pointer may be NULL; sizes given
 * in elements must be large enough (EINVAL otherwise). */
krylov_status krylov_last_cycle(const krylov_handle* h, double* T, int64_t T_cap, double* X,
                                int64_t X_cap, double* z, int64_t z_cap, int* m_eff);

/* Self-test of failure detection without a fault.  The staged kernels wait
 * for their bulk copies with a bounded mbarrier wait (1 s per wait); when a
 * wait gives up the kernel sets a timeout flag, drains its own copies (again
 * with a bound) and returns, and the call reports KRYLOV_ETIMEOUT.  This probe runs that wait in
 * one CTA on the current device, on a barrier phase that completes and on one
 * that never does (transaction bytes announced, no copy issued), with the
 * bound limit_ns (1 .. 10^10 ns, else EINVAL):
 *   timed_out : host, 2 ints: 1 where the wait gave up (expected: 0, 1);
 *   wait_ns   : host, 2 doubles: the waits' durations in ns (the second one
 *               at least limit_ns).
 * The device stays usable afterwards. */
krylov_status krylov_probe_bounded_wait(uint64_t limit_ns, int* timed_out, double* wait_ns);

#ifdef __cplusplus
}
#endif
#endif /* KRYLOV_H */
