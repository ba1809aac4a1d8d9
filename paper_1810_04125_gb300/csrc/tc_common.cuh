// Tensor-core building blocks shared by the mixed-precision kernels
// (tcgen05 MMA issue, TMEM loads, mbarriers, bulk copies, the splitting of
// FP64 values into TF32 / BF16 terms and the float-float accumulation).
//
// Shared-memory layout of a K-major tile with `rows` rows and BK elements of
// e bytes (16-byte chunks of 16/e elements): core matrices of 8 rows x 16 B
// (128 B contiguous); chunk c of row r at (r/8)*1024 + c*128 + (r%8)*16,
// i.e. leading-dimension byte offset 128 (next core matrix along K) and
// stride byte offset 1024 (next group of 8 rows); no swizzle.
#pragma once
#include <stdint.h>

#include "hss_internal.h"

namespace hss {
namespace {

constexpr int BM = 128;            // rows per CTA (TMEM lanes)
constexpr uint32_t TILE_A_BYTES = 16384;   // 128 rows x 128 B of K

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ uint32_t mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok;
}

// Bounded wait for the phase of `parity`; false (and *err set) on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, int code) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0 && gtimer() - t0 > 2000000000ull) {
      atomicCAS(err, 0, code);
      return false;
    }
  }
}

// mbar_wait by a whole warp (all 32 lanes converged): the warp gives up as a
// whole, so warp-collective operations after the wait (tcgen05.ld, __syncwarp)
// never wait for a lane that left.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t* bar, uint32_t parity, int* err, int code) {
  const bool ok = mbar_wait(bar, parity, err, code);
  return __all_sync(0xffffffffu, ok) != 0;
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// shared-memory matrix descriptor: start, LBO, SBO (bytes), SM100 version 1,
// no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor: D = F32, A = B = fmt (TF32 = 2 with kind::tf32,
// BF16 = 1 with kind::f16), both K-major, M = 128, N
__host__ __device__ constexpr uint32_t idesc(uint32_t fmt, uint32_t N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <int PREC>
__device__ __forceinline__ void mma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if (PREC == HSS_PREC_TF32X2) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// ---- splitting of an FP64 value into tensor-core terms
__device__ __forceinline__ float round_tf32(float x) {
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7F800000u) == 0x7F800000u) return x;   // inf / nan kept
  u += 0x00000FFFu + ((u >> 13) & 1u);              // round to nearest even at bit 13
  return __uint_as_float(u & 0xFFFFE000u);
}

__device__ __forceinline__ uint16_t bf16_bits(float x) {
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7F800000u) == 0x7F800000u) return (uint16_t)(u >> 16);
  u += 0x00007FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
__device__ __forceinline__ float bf16_val(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

template <int PREC>
struct Split;

template <>
struct Split<HSS_PREC_TF32X2> {
  static constexpr int T = 2;      // terms
  static constexpr int EV = 4;     // elements per 16-byte chunk
  static constexpr int BK = 32;    // K per stage (128 bytes per row)
  static constexpr int KSTEP = 8;  // K per MMA
  static constexpr uint32_t FMT = 2;
  // v: EV FP64 values -> T chunks of 16 bytes
  __device__ static void split(const double* v, uint4* out) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float f = __double2float_rn(v[e]);
      float hi = round_tf32(f);
      float lo = round_tf32(f - hi);
      h[e] = __float_as_uint(hi);
      l[e] = __float_as_uint(lo);
    }
    out[0] = make_uint4(h[0], h[1], h[2], h[3]);
    out[1] = make_uint4(l[0], l[1], l[2], l[3]);
  }
  __device__ static uint4 pack_r(const double* v) {   // R values are TF32-exact
    return make_uint4(__float_as_uint((float)v[0]), __float_as_uint((float)v[1]),
                      __float_as_uint((float)v[2]), __float_as_uint((float)v[3]));
  }
};

template <>
struct Split<HSS_PREC_BF16X3> {
  static constexpr int T = 3;
  static constexpr int EV = 8;
  static constexpr int BK = 64;
  static constexpr int KSTEP = 16;
  static constexpr uint32_t FMT = 1;
  __device__ static void split(const double* v, uint4* out) {
    uint32_t w[3][4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      uint16_t b[3][2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        float f = __double2float_rn(v[e + q]);
        uint16_t b0 = bf16_bits(f);
        float r1 = f - bf16_val(b0);
        uint16_t b1 = bf16_bits(r1);
        float r2 = r1 - bf16_val(b1);
        uint16_t b2 = bf16_bits(r2);
        b[0][q] = b0; b[1][q] = b1; b[2][q] = b2;
      }
#pragma unroll
      for (int t = 0; t < 3; ++t) w[t][e / 2] = (uint32_t)b[t][0] | ((uint32_t)b[t][1] << 16);
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) out[t] = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
  }
  __device__ static uint4 pack_r(const double* v) {   // R values are BF16-exact
    uint32_t w[4];
#pragma unroll
    for (int e = 0; e < 4; ++e)
      w[e] = (uint32_t)bf16_bits((float)v[2 * e]) | ((uint32_t)bf16_bits((float)v[2 * e + 1]) << 16);
    return make_uint4(w[0], w[1], w[2], w[3]);
  }
};

// first index and one-past-last of the halving-tree leaf containing i
__device__ __forceinline__ void leaf_range(int i, int n, int leaf, int& lo, int& hi) {
  int l = 0, size = n;
  while (size > leaf) {
    int h = size / 2;
    if (i < l + h) size = h;
    else { l += h; size -= h; }
  }
  lo = l;
  hi = l + size;
}


__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// ---------------------------------------------------------------------------
// Accumulation.  The tensor core adds every product into the FP32 TMEM
// accumulator with a rounding whose error is biased, so a long chain of
// MMAs into one accumulator loses accuracy in proportion to its length
// (about 2e-8 per MMA relative to the result).  Each CTA therefore
// accumulates only a short chain (DRAIN k-tiles) into one of two TMEM
// buffers, with the leading split term (HI) and the correction terms (LO) in
// separate accumulators; drain warps move a finished chain into per-thread
// float-float (compensated-sum) accumulators while the tensor core fills the other
// buffer.  TMEM columns: buffer b, accumulator x at (2 b + x) N.
//
// Drain thread layout: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows) and
// column quarter h of the N-column tile (NH = N / 4 columns per thread);
// sixteen drain warps cover the 128 x N tile once.

__device__ __forceinline__ void tmem_ld16_nw(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// (s, e) += x by compensated (Kahan) summation: the pending correction e
// joins the addend, and e keeps what the addition to s lost.  The sum of the
// chains is then exact to about two roundings of its value, whatever their
// number (Kahan's bound), in four additions instead of the seven of an
// error-free TwoSum.
__device__ __forceinline__ void ff_add(float& s, float& e, float x) {
  const float xc = __fadd_rn(x, e);
  const float t = __fadd_rn(s, xc);
  e = __fsub_rn(xc, __fsub_rn(t, s));
  s = t;
}

// Drain one finished chain from TMEM buffer b into (s, e).
template <int NH>
__device__ __forceinline__ void drain_chain(uint32_t tmem, int N, int b, int q, int h, float* s, float* e) {
  const uint32_t lane_off = (uint32_t)(32 * q) << 16;
  const uint32_t hi = tmem + lane_off + (uint32_t)((2 * b) * N + h * NH);
  const uint32_t lo = tmem + lane_off + (uint32_t)((2 * b + 1) * N + h * NH);
#pragma unroll
  for (int c = 0; c < NH; c += 16) {
    float x[16];
    tmem_ld16_nw(hi + c, x);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 16; ++i) ff_add(s[c + i], e[c + i], x[i]);
    tmem_ld16_nw(lo + c, x);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 16; ++i) e[c + i] = __fadd_rn(e[c + i], x[i]);
  }
}

// float -> double by integer operations (exact; the FP64 conversion unit is
// as slow as the FP64 pipe on this part).  Zero and normal floats only: the
// float-float parts of a sample are never subnormal, infinite or NaN unless
// the input is (the samples are checked for NaN/Inf afterwards).
__device__ __forceinline__ double f2d_exact(float x) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t ex = (u >> 23) & 0xFFu;
  if (ex == 0u) return 0.0;
  if (ex == 0xFFu) return (double)x;
  const uint64_t sign = (uint64_t)(u >> 31) << 63;
  const uint64_t e64 = (uint64_t)(ex - 127u + 1023u) << 52;
  const uint64_t man = (uint64_t)(u & 0x7FFFFFu) << 29;
  return __longlong_as_double((long long)(sign | e64 | man));
}

// Write one thread's row of the result (NH columns from col).
template <int NH>
__device__ __forceinline__ void store_row(double* S, long long lds, int n, int ncols, int row, int col,
                                          int atomic, const float* s, const float* e) {
  if (row >= n) return;
  double* out = S + (long long)row * lds + col;
#pragma unroll
  for (int j = 0; j < NH; ++j) {
    if (col + j < ncols) {
      const double v = f2d_exact(s[j]) + f2d_exact(e[j]);
      if (atomic) atomicAdd(out + j, v);
      else out[j] = v;
    }
  }
}

// Issue the MMAs of one k-tile (BK/KSTEP k-steps, T terms) into buffer b.
template <int PREC>
__device__ __forceinline__ void mma_ktile(uint32_t base, uint32_t tmem, int N, int b, bool first,
                                          uint32_t id) {
  using SP = Split<PREC>;
  constexpr int T = SP::T, BK = SP::BK;
  const uint32_t hi = tmem + (uint32_t)((2 * b) * N), lo = tmem + (uint32_t)((2 * b + 1) * N);
#pragma unroll
  for (int ks = 0; ks < BK / SP::KSTEP; ++ks) {
    const uint64_t bd = sdesc(base + T * TILE_A_BYTES + ks * 256u, 128u, 1024u);
    mma<PREC>(hi, sdesc(base + ks * 256u, 128u, 1024u), bd, id, (first && ks == 0) ? 0u : 1u);
#pragma unroll
    for (int t = 1; t < T; ++t)
      mma<PREC>(lo, sdesc(base + t * TILE_A_BYTES + ks * 256u, 128u, 1024u), bd, id,
                (first && ks == 0 && t == 1) ? 0u : 1u);
  }
}

}  // namespace
}  // namespace hss
