// kernels.cuh -- device-side building blocks shared by the library's kernels.
//
// Contents
//  * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the sparse sign
//    column generator of Sec. 2.1, Eq. (3): zeta distinct rows per column,
//    uniform, Rademacher signs.  The exact word-to-entry mapping (fixed so the
//    host-side reference implementation can reproduce S bit for bit) is:
//      counter (j, block, 0, 0), key (seed lo, seed hi); each output word is
//      split into two 16-bit chunks, low half first; a chunk c proposes row
//      (c & 0x7FFF) mod s with sign bit c >> 15; the proposal is rejected when
//      (c & 0x7FFF) >= 32768 - (32768 mod s) or when the row was already taken
//      by this column; at most SKETCH_MAX_BLOCKS counter blocks per column.
//  * storage-type conversions for the basis (float64 / float32 / bfloat16).
//  * the deterministic "last block reduces" pattern used by the step kernels.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace krylov {

constexpr int SKETCH_MAX_BLOCKS = 64;
constexpr int MAX_WINDOW = 4;       // k <= 4 (orthogonalization window)
constexpr int STEP_THREADS = 256;   // threads per CTA of the streaming kernels
constexpr int MAX_ZETA = 32;

struct Philox4 {
  uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

// Ten Philox rounds on counter c with key (k0, k1).
__host__ __device__ __forceinline__ Philox4 philox4x32_10(Philox4 c, uint32_t k0, uint32_t k1) {
  const uint32_t MA = 0xD2511F53u, MB = 0xCD9E8D57u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = mulhi32(MA, c.x), lo0 = MA * c.x;
    const uint32_t hi1 = mulhi32(MB, c.z), lo1 = MB * c.z;
    Philox4 o;
    o.x = hi1 ^ c.y ^ k0;
    o.y = lo1;
    o.z = hi0 ^ c.w ^ k1;
    o.w = lo0;
    c = o;
  }
  return c;
}

struct SketchSpec {
  int s;          // rows of S
  int zeta;       // nonzeros per column
  uint32_t lim;   // 32768 - 32768 % s
  uint32_t k0, k1;
  float scale;    // 1/sqrt(zeta)
};

// Generate column j of S.  Calls emit(row, negative) once per accepted entry,
// in acceptance order.  Returns the number of entries produced (== zeta unless
// the block budget ran out, which the caller reports as an error).
template <int ZMAX, typename Emit>
__host__ __device__ __forceinline__ int sketch_column(uint32_t j, const SketchSpec& sp, Emit&& emit) {
  int rows[ZMAX];
  int cnt = 0;
  for (uint32_t blk = 0; blk < (uint32_t)SKETCH_MAX_BLOCKS && cnt < sp.zeta; ++blk) {
    const Philox4 w = philox4x32_10(Philox4{j, blk, 0u, 0u}, sp.k0, sp.k1);
    const uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint32_t ch = (words[q >> 1] >> (16 * (q & 1))) & 0xFFFFu;
      const uint32_t v = ch & 0x7FFFu;
      if (cnt < sp.zeta && v < sp.lim) {
        const int row = (int)(v % (uint32_t)sp.s);
        bool dup = false;
#pragma unroll
        for (int e = 0; e < ZMAX; ++e) dup |= (e < cnt) && (rows[e] == row);
        if (!dup) {
#pragma unroll
          for (int e = 0; e < ZMAX; ++e)
            if (e == cnt) rows[e] = row;
          emit(row, (ch >> 15) != 0u);
          ++cnt;
        }
      }
    }
  }
  return cnt;
}

// ceil(2^32 / s): floor(v / s) = umulhi(v, sketch_inv_s(s)) for v < 2^15, s < 2^15.
__host__ __device__ __forceinline__ uint32_t sketch_inv_s(int s) {
  return (uint32_t)((0x100000000ull + (uint64_t)s - 1) / (uint64_t)s);
}

// Fast path of sketch_column for s <= 255 and zeta <= 8: the accepted rows are
// kept as bytes packed in two words (0xFF marks an empty slot, never a row),
// duplicates are found with SIMD byte compares, and v mod s uses the exact
// multiply-high identity floor(v / s) = umulhi(v, ceil(2^32 / s)) for
// v < 2^15.  Produces the same entries, in the same order, as sketch_column.
// Returns the count; rows in (*p0, *p1) byte e, sign bit e of *neg.
__device__ __forceinline__ int sketch_column_packed(uint32_t j, const SketchSpec& sp, uint32_t inv_s,
                                                     uint32_t* p0, uint32_t* p1, uint32_t* neg) {
  uint32_t r0 = 0xFFFFFFFFu, r1 = 0xFFFFFFFFu, ng = 0u;
  int cnt = 0;
  for (uint32_t blk = 0; blk < (uint32_t)SKETCH_MAX_BLOCKS && cnt < sp.zeta; ++blk) {
    const Philox4 w = philox4x32_10(Philox4{j, blk, 0u, 0u}, sp.k0, sp.k1);
    const uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint32_t ch = (words[q >> 1] >> (16 * (q & 1))) & 0xFFFFu;
      const uint32_t v = ch & 0x7FFFu;
      const uint32_t row = v - (uint32_t)sp.s * __umulhi(v, inv_s);
      const uint32_t rep = row * 0x01010101u;
      const bool dup = (__vcmpeq4(r0, rep) | __vcmpeq4(r1, rep)) != 0u;
      if (cnt < sp.zeta && v < sp.lim && !dup) {
        const uint32_t sh = 8u * (uint32_t)(cnt & 3);
        const uint32_t keep = ~(0xFFu << sh);
        if (cnt < 4) r0 = (r0 & keep) | (row << sh);
        else r1 = (r1 & keep) | (row << sh);
        ng |= (ch >> 15) << cnt;
        ++cnt;
      }
    }
  }
  *p0 = r0;
  *p1 = r1;
  *neg = ng;
  return cnt;
}

// ---- float-float ("df64") arithmetic ---------------------------------------
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  Built from the error-free transformations
// TwoSum (Knuth) and TwoProduct via fused multiply-add (e.g. Dekker 1971;
// Muller et al., Handbook of Floating-Point Arithmetic, ch. 4).
struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, e);
}
// a * b with a float and b float-float
__device__ __forceinline__ ff ff_mul_f(ff b, float a) {
  const float p = __fmul_rn(a, b.hi);
  float e = __fmaf_rn(a, b.hi, -p);
  e = __fmaf_rn(a, b.lo, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
// acc + a * b (a float, b float-float)
__device__ __forceinline__ ff ff_fma_f(float a, ff b, ff acc) { return ff_add(acc, ff_mul_f(b, a)); }
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_from_double(double d) {
  const float h = __double2float_rn(d);
  return {h, __double2float_rn(d - (double)h)};
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// Add v to the pair of shared-memory bins (hi[b], lo[b]): the rounding error
// of the atomic float add on hi is recovered exactly from the returned old
// value (TwoSum) and added to lo together with v.lo, so hi + lo carries the
// float-float sum regardless of the order in which threads arrive.
__device__ __forceinline__ void ff_atomic_add(float* hi, float* lo, ff v) {
  const float old = atomicAdd(hi, v.hi);
  const ff s = two_sum(old, v.hi);
  atomicAdd(lo, __fadd_rn(s.lo, v.lo));
}

// ---- bulk asynchronous copies (TMA, 1-D) and mbarriers ----------------------
// Addresses of bulk copies must be 16-byte aligned and sizes multiples of 16.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// One arrival that also announces `bytes` of transactions for this phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Expect `bytes` more transaction bytes in the current phase, without arriving.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Arrive without expecting transaction bytes.
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar)) : "memory");
}
// Global -> shared bulk copy whose completion is reported to `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// L2 eviction priority for streams that are read once per pass (the CSR
// tiles, the sketch table): evict-first keeps the vectors that later loads
// gather from resident in L2.
#ifndef KRYLOV_L2_HINT
#define KRYLOV_L2_HINT 1
#endif
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
// bulk copy with an L2 cache policy (pol from l2_policy_evict_first)
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                              uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}
// a stream read once per pass: evict-first in L2 (KRYLOV_L2_HINT, on by
// default: 29.3 -> 27.8 ms of step kernels per headline solve, the gathers of
// w_j and the window loads then hit L2)
__device__ __forceinline__ void bulk_g2s_stream(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  if (KRYLOV_L2_HINT) bulk_g2s_hint(dst, src, bytes, bar, l2_policy_evict_first());
  else bulk_g2s(dst, src, bytes, bar);
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for phase `parity` of `bar`: false if it has not completed
// after `limit_ns` nanoseconds (the caller reports a timeout instead of hanging).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

// ---- programmatic dependent launch ------------------------------------------
// A kernel launched with programmatic stream serialization may start while the
// previous kernel in the stream is still running: pdl_wait() blocks until that
// kernel (and so everything before it) has completed and its writes are
// visible; pdl_trigger() lets the next kernel start launching.  Both are no-ops
// for a normal launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---- storage conversions --------------------------------------------------
template <typename T> struct Store;
template <> struct Store<double> {
  __device__ __forceinline__ static double load(const double* p) { return *p; }
  __device__ __forceinline__ static double round_f64(double v) { return v; }
  __device__ __forceinline__ static float round_f32(float v) { return v; }
  __device__ __forceinline__ static void put(double* p, double v) { *p = v; }
};
template <> struct Store<float> {
  __device__ __forceinline__ static float load(const float* p) { return *p; }
  __device__ __forceinline__ static void put(float* p, float v) { *p = v; }
};
template <> struct Store<__nv_bfloat16> {
  __device__ __forceinline__ static float load(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  __device__ __forceinline__ static void put(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};

// Value of a number after a round trip through storage type T.
template <typename T, typename A> __device__ __forceinline__ A stored(A v);
template <> __device__ __forceinline__ double stored<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float stored<float, float>(float v) { return v; }
template <> __device__ __forceinline__ float stored<__nv_bfloat16, float>(float v) {
  return __bfloat162float(__float2bfloat16_rn(v));
}

__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }

template <typename A> __device__ __forceinline__ A warp_sum(A v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum in a fixed order (warp shuffles, then warp 0 over the warp
// partials).  Result valid in thread 0.  `sh` holds >= 32 entries.
// Sum of column q of a count x stride array of per-CTA partials, computed by
// one warp: lane l takes rows l, l+32, ... in order, then a fixed shuffle tree.
// The result (in every lane) does not depend on timing, only on count.
__device__ __forceinline__ double warp_sum_partials(const double* part, int count, int stride, int q) {
  // up to 16 loads per lane in flight at once (one round trip to L2 for up to
  // 512 partials), then added in the order c = lane, lane + 32, ...
  constexpr int B = 16;
  const int lane = (int)(threadIdx.x & 31);
  double t = 0.0;
  for (int c0 = lane; c0 < count; c0 += 32 * B) {
    double v[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int c = c0 + 32 * u;
      v[u] = (c < count) ? __ldcg(part + (size_t)c * stride + q) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < B; ++u) t += v[u];
  }
  return warp_sum(t);
}

template <typename A> __device__ __forceinline__ A block_sum(A v, A* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  A r = 0;
  if (wid == 0) {
    r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : A(0);
    r = warp_sum(r);
  }
  return r;
}

}  // namespace krylov
