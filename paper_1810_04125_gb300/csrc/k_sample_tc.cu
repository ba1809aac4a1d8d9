// Mixed-precision sampling on the tcgen05 tensor cores:
//     S = (A - D^(L)) R        (orientation 0, S^r)
//     S = (A - D^(L))^T R      (orientation 1, S^c)
// i.e. eq. sample_off_diag at the leaf level with the leaf subtraction folded
// into the tile staging, as in the FP64 kernel.
//
// Precision (the two mixed forms):
//   TF32X2: every entry a of A is rounded once to FP32 and split as
//           a ~= a0 + a1 with a0, a1 TF32 values (22 significant bits);
//           R holds TF32 values exactly; two kind::tf32 products.
//   BF16X3: a ~= a0 + a1 + a2 with BF16 terms (24 significant bits); R holds
//           BF16 values exactly; three kind::f16 (bf16) products.
// Every product of terms is exact in FP32 and accumulates in FP32 in TMEM;
// the epilogue adds the FP32 tile into the FP64 output.
//
// CTA: 128 output rows x N sample columns (N <= 128, a multiple of 16),
// K (the summation index) staged BK at a time through an NS-deep ring of
// shared-memory stages.  Warps 0-3 produce (load or generate FP64 entries,
// zero the leaf diagonal block, split, write the canonical K-major layout)
// and later drain TMEM; warp 4 owns the TMEM allocation and one of its
// threads issues the MMAs and the tcgen05.commit arrivals.  Every mbarrier
// wait is bounded (about 2 s of %globaltimer); on expiry the kernel records
// an error code and leaves the pipeline, frees its TMEM and returns.
//
// Shared-memory layout of a K-major tile with `rows` rows and BK elements of
// e bytes (16-byte chunks of 16/e elements): core matrices of 8 rows x 16 B
// (128 B contiguous); chunk c of row r at (r/8)*1024 + c*128 + (r%8)*16,
// i.e. leading-dimension byte offset 128 (next core matrix along K) and
// stride byte offset 1024 (next group of 8 rows); no swizzle.
#include <stdint.h>

#include "hss_internal.h"

namespace hss {
namespace {

constexpr int BM = 128;            // rows per CTA (TMEM lanes)
constexpr int NSTAGE = 3;
constexpr int NPROD = 128;         // producer / epilogue threads (warps 0-3)
constexpr int NTHREADS = NPROD + 32;
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

// 32 TMEM lanes x 16 consecutive 32-bit columns
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
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

struct TcArgs {
  SrcDev src;
  int leaf;
  int trans;
  int ncols;          // sample columns computed (this launch)
  int N;              // columns per CTA tile (multiple of 16, <= 256)
  int tmem_cols;      // power of two >= N
  int ksplit;         // CTAs along K
  const double* R;    // n x ncols col-major (ld ldr)
  long long ldr;
  double* S;          // row-major output, row stride lds
  long long lds;
  int atomic;         // 1: add into S (pre-zeroed); 0: store
  int* err;
};

template <int PREC>
__global__ void __launch_bounds__(NTHREADS, 1) k_sample_tc(TcArgs a) {
  using SP = Split<PREC>;
  constexpr int T = SP::T, EV = SP::EV, BK = SP::BK, KC = BK / EV;   // KC = 8 chunks
  extern __shared__ __align__(1024) uint8_t smem[];
  const int n = a.src.n;
  const int N = a.N;
  const uint32_t tileB = (uint32_t)N * 128u;
  const uint32_t stage_bytes = T * TILE_A_BYTES + tileB;
  uint8_t* stages = smem;
  uint64_t* full = (uint64_t*)(smem + NSTAGE * stage_bytes);
  uint64_t* empty = full + NSTAGE;
  uint64_t* done = empty + NSTAGE;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  int* lrow_lo = (int*)(tmem_slot + 4);
  int* lrow_hi = lrow_lo + BM;

  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int row0 = blockIdx.x * BM;
  const int col0 = blockIdx.y * N;
  const int nk_total = (n + BK - 1) / BK;
  const int kt0 = (int)((long long)nk_total * blockIdx.z / a.ksplit);
  const int kt1 = (int)((long long)nk_total * (blockIdx.z + 1) / a.ksplit);
  const int nk = kt1 - kt0;

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) { mbar_init(&full[s], NPROD); mbar_init(&empty[s], 1); }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < BM) {
    int r = row0 + tid, lo = 0x7fffffff, hi = 0x7fffffff;
    if (r < n) leaf_range(r, n, a.leaf, lo, hi);
    lrow_lo[tid] = lo;
    lrow_hi[tid] = hi;
  }
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"((uint32_t)a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  if (warp < 4) {
    // ------------------------------------------------------------ producers
    for (int it = 0; it < nk && ok; ++it) {
      const int s = it % NSTAGE;
      const uint32_t ph = (uint32_t)(it / NSTAGE) & 1u;
      if (!mbar_wait(&empty[s], ph ^ 1u, a.err, 2)) { ok = false; break; }
      uint8_t* st = stages + s * stage_bytes;
      const int k0 = (kt0 + it) * BK;
      // A tile: 128 rows x KC chunks; unit u -> (row, chunk)
      for (int u = tid; u < BM * KC; u += NPROD) {
        int r, c;
        if (!a.trans) { r = u % BM; c = u / BM; }                       // consecutive rows
        else { r = (u / (8 * KC)) * 8 + (u % 8); c = (u / 8) % KC; }    // consecutive K
        const int gr = row0 + r;
        const int lo = lrow_lo[r], hi = lrow_hi[r];
        double v[EV];
#pragma unroll
        for (int e = 0; e < EV; ++e) {
          const int gk = k0 + c * EV + e;
          double x = 0.0;
          if (gr < n && gk < n && (gk < lo || gk >= hi))
            x = a.trans ? entry(a.src, gk, gr) : entry(a.src, gr, gk);
          v[e] = x;
        }
        uint4 chunk[T];
        SP::split(v, chunk);
        const uint32_t off = (uint32_t)(r / 8) * 1024u + (uint32_t)c * 128u + (uint32_t)(r % 8) * 16u;
#pragma unroll
        for (int t = 0; t < T; ++t) *(uint4*)(st + t * TILE_A_BYTES + off) = chunk[t];
      }
      // B tile: N rows (sample columns) x KC chunks, R K-contiguous
      uint8_t* sb = st + T * TILE_A_BYTES;
      for (int u = tid; u < N * KC; u += NPROD) {
        const int r = (u / (8 * KC)) * 8 + (u % 8), c = (u / 8) % KC;
        const int gc = col0 + r;
        double v[EV];
#pragma unroll
        for (int e = 0; e < EV; ++e) {
          const int gk = k0 + c * EV + e;
          v[e] = (gc < a.ncols && gk < n) ? a.R[(long long)gk + (long long)gc * a.ldr] : 0.0;
        }
        const uint32_t off = (uint32_t)(r / 8) * 1024u + (uint32_t)c * 128u + (uint32_t)(r % 8) * 16u;
        *(uint4*)(sb + off) = SP::pack_r(v);
      }
      fence_async_smem();
      mbar_arrive(&full[s]);
    }
  } else if (lane == 0) {
    // ------------------------------------------------------------- MMA issuer
    const uint32_t id = idesc(SP::FMT, (uint32_t)N);
    uint32_t acc = 0;
    for (int it = 0; it < nk; ++it) {
      const int s = it % NSTAGE;
      const uint32_t ph = (uint32_t)(it / NSTAGE) & 1u;
      if (!mbar_wait(&full[s], ph, a.err, 3)) { ok = false; break; }
      tc_fence_after();
      const uint32_t base = smem_u32(stages + s * stage_bytes);
#pragma unroll
      for (int ks = 0; ks < BK / SP::KSTEP; ++ks) {
        const uint64_t bd = sdesc(base + T * TILE_A_BYTES + ks * 256u, 128u, 1024u);
#pragma unroll
        for (int t = 0; t < T; ++t) {
          const uint64_t ad = sdesc(base + t * TILE_A_BYTES + ks * 256u, 128u, 1024u);
          mma<PREC>(tmem, ad, bd, id, acc);
          acc = 1;
        }
      }
      mma_commit(&empty[s]);
    }
    mma_commit(done);   // arrives once every issued MMA has completed
  }

  // ----------------------------------------------------------------- epilogue
  if (warp < 4) {
    bool have = mbar_wait(done, 0u, a.err, 4) && ok && nk > 0;
    have = __all_sync(0xffffffffu, have);   // tcgen05.ld is warp-collective
    tc_fence_after();
    if (have) {
      const int r = row0 + warp * 32 + lane;
      for (int c0 = 0; c0 < N; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (r < n) {
          double* out = a.S + (long long)r * a.lds + col0 + c0;
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            if (col0 + c0 + e < a.ncols) {
              if (a.atomic) atomicAdd(out + e, (double)v[e]);
              else out[e] = (double)v[e];
            }
          }
        }
      }
    }
  } else {
    // warp 4's other lanes wait for the issuer's last commit before freeing TMEM
    mbar_wait(done, 0u, a.err, 5);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 4) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)a.tmem_cols)
                 : "memory");
  }
}

template <int PREC>
size_t smem_bytes(int N) {
  constexpr int T = Split<PREC>::T;
  return (size_t)NSTAGE * (T * TILE_A_BYTES + (size_t)N * 128) + 8 * (2 * NSTAGE + 1) + 16 +
         2 * BM * sizeof(int) + 1024;
}

template <int PREC>
cudaError_t launch_t(const TcArgs& a0, int grid_x, int grid_y, cudaStream_t st) {
  TcArgs a = a0;
  size_t sm = smem_bytes<PREC>(a.N);
  cudaError_t e = cudaFuncSetAttribute(k_sample_tc<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  k_sample_tc<PREC><<<dim3(grid_x, grid_y, a.ksplit), NTHREADS, sm, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Packed path (a dense A is re-read on every pass): the operands are split
// once into canonical K-major tiles in global memory,
//   A, orientation o: tile (rb, kt) = T consecutive 16 KB term tiles at
//       ((o * nrb + rb) * nkt + kt) * T * 16 KB        (leaf diagonal zeroed)
//   R: tile (ct, kt) of N rows x BK at (ct * nkt + kt) * N * 128 bytes,
// and the main loop moves whole tiles with cp.async.bulk issued by one
// thread, completing on the stage mbarrier (expect_tx); one thread issues the
// MMAs; no per-element work is left in the loop.

template <int PREC>
__global__ void __launch_bounds__(256) k_pack_a(SrcDev src, int leaf, int nrb, int nkt, uint8_t* out) {
  using SP = Split<PREC>;
  constexpr int T = SP::T, EV = SP::EV, BK = SP::BK, KC = BK / EV;
  __shared__ int rlo[BM], rhi[BM];
  const int n = src.n;
  const long long tile = blockIdx.x;
  const long long per_o = (long long)nrb * nkt;
  const int o = (int)(tile / per_o);
  const long long rem = tile % per_o;
  const int rb = (int)(rem / nkt), kt = (int)(rem % nkt);
  const int row0 = rb * BM, k0 = kt * BK;
  if (threadIdx.x < BM) {
    int r = row0 + threadIdx.x, lo = 0x7fffffff, hi = 0x7fffffff;
    if (r < n) leaf_range(r, n, leaf, lo, hi);
    rlo[threadIdx.x] = lo;
    rhi[threadIdx.x] = hi;
  }
  __syncthreads();
  uint8_t* dst = out + (size_t)tile * T * TILE_A_BYTES;
  for (int u = threadIdx.x; u < BM * KC; u += blockDim.x) {
    int r, c;
    if (!o) { r = u % BM; c = u / BM; }
    else { r = (u / (8 * KC)) * 8 + (u % 8); c = (u / 8) % KC; }
    const int gr = row0 + r, lo = rlo[r], hi = rhi[r];
    double v[EV];
#pragma unroll
    for (int e = 0; e < EV; ++e) {
      const int gk = k0 + c * EV + e;
      double x = 0.0;
      if (gr < n && gk < n && (gk < lo || gk >= hi)) x = o ? entry(src, gk, gr) : entry(src, gr, gk);
      v[e] = x;
    }
    uint4 chunk[T];
    SP::split(v, chunk);
    const uint32_t off = (uint32_t)(r / 8) * 1024u + (uint32_t)c * 128u + (uint32_t)(r % 8) * 16u;
#pragma unroll
    for (int t = 0; t < T; ++t) *(uint4*)(dst + t * TILE_A_BYTES + off) = chunk[t];
  }
}

template <int PREC>
__global__ void __launch_bounds__(256) k_pack_r(const double* R, long long ldr, int n, int ncols, int N,
                                                int nkt, uint8_t* out) {
  using SP = Split<PREC>;
  constexpr int EV = SP::EV, BK = SP::BK, KC = BK / EV;
  const int tile = blockIdx.x, ct = tile / nkt, kt = tile % nkt;
  uint8_t* dst = out + (size_t)tile * N * 128;
  for (int u = threadIdx.x; u < N * KC; u += blockDim.x) {
    const int r = (u / (8 * KC)) * 8 + (u % 8), c = (u / 8) % KC;
    const int gc = ct * N + r;
    double v[EV];
#pragma unroll
    for (int e = 0; e < EV; ++e) {
      const int gk = kt * BK + c * EV + e;
      v[e] = (gc < ncols && gk < n) ? R[(long long)gk + (long long)gc * ldr] : 0.0;
    }
    const uint32_t off = (uint32_t)(r / 8) * 1024u + (uint32_t)c * 128u + (uint32_t)(r % 8) * 16u;
    *(uint4*)(dst + off) = SP::pack_r(v);
  }
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

struct TcPackedArgs {
  const uint8_t* A;
  const uint8_t* Rp;
  int n, nrb, nkt, N, ncols, tmem_cols, ksplit, trans;
  double* S;
  long long lds;
  int atomic;
  int* err;
};

template <int PREC>
constexpr int packed_stages() { return PREC == HSS_PREC_TF32X2 ? 4 : 3; }

template <int PREC>
__global__ void __launch_bounds__(128, 1) k_sample_tc_packed(TcPackedArgs a) {
  using SP = Split<PREC>;
  constexpr int T = SP::T, BK = SP::BK, NS = packed_stages<PREC>();
  extern __shared__ __align__(1024) uint8_t smem[];
  const int N = a.N;
  const uint32_t tileB = (uint32_t)N * 128u;
  const uint32_t stage_bytes = T * TILE_A_BYTES + tileB;
  uint64_t* full = (uint64_t*)(smem + NS * stage_bytes);
  uint64_t* empty = full + NS;
  uint64_t* done = empty + NS;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int rb = blockIdx.x, ct = blockIdx.y;
  const int kt0 = (int)((long long)a.nkt * blockIdx.z / a.ksplit);
  const int kt1 = (int)((long long)a.nkt * (blockIdx.z + 1) / a.ksplit);
  const int nk = kt1 - kt0;
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"((uint32_t)a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint8_t* gA = a.A + ((size_t)(a.trans * a.nrb + rb) * a.nkt + kt0) * (T * TILE_A_BYTES);
  const uint8_t* gB = a.Rp + ((size_t)ct * a.nkt + kt0) * tileB;
  bool ok = true;
  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------- bulk-copy producer
    for (int it = 0; it < nk; ++it) {
      const int s = it % NS;
      const uint32_t ph = (uint32_t)(it / NS) & 1u;
      if (!mbar_wait(&empty[s], ph ^ 1u, a.err, 12)) { ok = false; break; }
      uint8_t* st = smem + s * stage_bytes;
      mbar_expect_tx(&full[s], stage_bytes);
#pragma unroll
      for (int t = 0; t < T; ++t)
        bulk_g2s(st + t * TILE_A_BYTES, gA + (size_t)it * (T * TILE_A_BYTES) + t * TILE_A_BYTES,
                 TILE_A_BYTES, &full[s]);
      bulk_g2s(st + T * TILE_A_BYTES, gB + (size_t)it * tileB, tileB, &full[s]);
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------- MMA issuer
    const uint32_t id = idesc(SP::FMT, (uint32_t)N);
    uint32_t acc = 0;
    for (int it = 0; it < nk; ++it) {
      const int s = it % NS;
      const uint32_t ph = (uint32_t)(it / NS) & 1u;
      if (!mbar_wait(&full[s], ph, a.err, 13)) { ok = false; break; }
      tc_fence_after();
      const uint32_t base = smem_u32(smem + s * stage_bytes);
#pragma unroll
      for (int ks = 0; ks < BK / SP::KSTEP; ++ks) {
        const uint64_t bd = sdesc(base + T * TILE_A_BYTES + ks * 256u, 128u, 1024u);
#pragma unroll
        for (int t = 0; t < T; ++t) {
          const uint64_t ad = sdesc(base + t * TILE_A_BYTES + ks * 256u, 128u, 1024u);
          mma<PREC>(tmem, ad, bd, id, acc);
          acc = 1;
        }
      }
      mma_commit(&empty[s]);
    }
    mma_commit(done);
  }
  __syncwarp();
  // ----------------------------------------------------------------- epilogue
  bool have = mbar_wait(done, 0u, a.err, 14) && nk > 0;
  have = __all_sync(0xffffffffu, have && ok);
  tc_fence_after();
  if (have) {
    const int r = rb * BM + warp * 32 + lane;
    const int col0 = ct * N;
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (r < a.n) {
        double* out = a.S + (long long)r * a.lds + col0 + c0;
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          if (col0 + c0 + e < a.ncols) {
            if (a.atomic) atomicAdd(out + e, (double)v[e]);
            else out[e] = (double)v[e];
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)a.tmem_cols)
                 : "memory");
  }
}

int tile_n(int ncols) {
  int N = ((ncols + 15) / 16) * 16;
  return N > 128 ? 128 : N;
}

template <int PREC>
cudaError_t launch_packed_t(const TcPackedArgs& a, int gx, int gy, cudaStream_t st) {
  constexpr int T = Split<PREC>::T, NS = packed_stages<PREC>();
  const size_t sm = (size_t)NS * (T * TILE_A_BYTES + (size_t)a.N * 128) + 8 * (2 * NS + 1) + 16 + 1024;
  cudaError_t e = cudaFuncSetAttribute(k_sample_tc_packed<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  k_sample_tc_packed<PREC><<<dim3(gx, gy, a.ksplit), 128, sm, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

size_t packed_a_bytes(int n, int precision) {
  const int T = precision == HSS_PREC_TF32X2 ? 2 : 3, bk = precision == HSS_PREC_TF32X2 ? 32 : 64;
  const size_t nrb = (n + BM - 1) / BM, nkt = (n + bk - 1) / bk;
  return 2 * nrb * nkt * T * (size_t)TILE_A_BYTES;
}

size_t packed_r_bytes(int n, int ncols, int precision) {
  const int bk = precision == HSS_PREC_TF32X2 ? 32 : 64;
  const int N = tile_n(ncols);
  const size_t nct = (ncols + N - 1) / N, nkt = (n + bk - 1) / bk;
  return nct * nkt * (size_t)N * 128;
}

cudaError_t launch_pack_a(const SrcDev& src, int leaf, int precision, void* out, cudaStream_t st) {
  const int n = src.n;
  const int bk = precision == HSS_PREC_TF32X2 ? 32 : 64;
  const int nrb = (n + BM - 1) / BM, nkt = (n + bk - 1) / bk;
  const long long tiles = 2LL * nrb * nkt;
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (precision == HSS_PREC_TF32X2)
    k_pack_a<HSS_PREC_TF32X2><<<(unsigned)tiles, 256, 0, st>>>(src, leaf, nrb, nkt, (uint8_t*)out);
  else
    k_pack_a<HSS_PREC_BF16X3><<<(unsigned)tiles, 256, 0, st>>>(src, leaf, nrb, nkt, (uint8_t*)out);
  return cudaGetLastError();
}

cudaError_t launch_pack_r(const double* R, long long ldr, int n, int ncols, int precision, void* out,
                          cudaStream_t st) {
  if (n <= 0 || ncols <= 0) return cudaSuccess;
  const int bk = precision == HSS_PREC_TF32X2 ? 32 : 64;
  const int N = tile_n(ncols), nct = (ncols + N - 1) / N, nkt = (n + bk - 1) / bk;
  if (precision == HSS_PREC_TF32X2)
    k_pack_r<HSS_PREC_TF32X2><<<nct * nkt, 256, 0, st>>>(R, ldr, n, ncols, N, nkt, (uint8_t*)out);
  else
    k_pack_r<HSS_PREC_BF16X3><<<nct * nkt, 256, 0, st>>>(R, ldr, n, ncols, N, nkt, (uint8_t*)out);
  return cudaGetLastError();
}

int sample_tc_packed_ksplit(int n, int ncols, int precision) {
  const int bk = precision == HSS_PREC_TF32X2 ? 32 : 64;
  const int N = tile_n(ncols);
  const int gx = (n + BM - 1) / BM, gy = (ncols + N - 1) / N, nkt = (n + bk - 1) / bk;
  int ks = (4 * 152 + gx * gy - 1) / (gx * gy);
  if (ks > nkt) ks = nkt;
  return ks < 1 ? 1 : ks;
}

cudaError_t launch_sample_tc_packed(const void* A, const void* Rp, int n, int ncols, int precision,
                                    int trans, double* S, long long lds, int* err, cudaStream_t st) {
  if (n <= 0 || ncols <= 0) return cudaSuccess;
  TcPackedArgs a;
  const int bk = precision == HSS_PREC_TF32X2 ? 32 : 64;
  a.A = (const uint8_t*)A;
  a.Rp = (const uint8_t*)Rp;
  a.n = n;
  a.nrb = (n + BM - 1) / BM;
  a.nkt = (n + bk - 1) / bk;
  a.N = tile_n(ncols);
  a.ncols = ncols;
  int tc = 32;
  while (tc < a.N) tc *= 2;
  a.tmem_cols = tc;
  a.ksplit = sample_tc_packed_ksplit(n, ncols, precision);
  a.trans = trans;
  a.S = S;
  a.lds = lds;
  a.atomic = a.ksplit > 1 ? 1 : 0;
  a.err = err;
  const int gy = (ncols + a.N - 1) / a.N;
  if (precision == HSS_PREC_TF32X2) return launch_packed_t<HSS_PREC_TF32X2>(a, a.nrb, gy, st);
  if (precision == HSS_PREC_BF16X3) return launch_packed_t<HSS_PREC_BF16X3>(a, a.nrb, gy, st);
  return cudaErrorInvalidValue;
}

// S (+)= (A - D^(L))^{[T]} R in a mixed precision; S must be zeroed by the
// caller when the K range is split across CTAs (ksplit > 1 adds atomically).
cudaError_t launch_sample_tc(const SrcDev& src, int leaf, int precision, int trans, int ncols,
                             const double* R, long long ldr, double* S, long long lds, int* err,
                             int* used_atomic, cudaStream_t st) {
  const int n = src.n;
  if (n <= 0 || ncols <= 0) return cudaSuccess;
  TcArgs a;
  a.src = src;
  a.leaf = leaf;
  a.trans = trans;
  a.ncols = ncols;
  int N = ((ncols + 15) / 16) * 16;
  if (N > 128) N = 128;                        // several column tiles of 128
  a.N = N;
  int tc = 32;
  while (tc < N) tc *= 2;
  a.tmem_cols = tc;
  const int gx = (n + BM - 1) / BM, gy = (ncols + N - 1) / N;
  const int bk = precision == HSS_PREC_TF32X2 ? Split<HSS_PREC_TF32X2>::BK : Split<HSS_PREC_BF16X3>::BK;
  const int nk = (n + bk - 1) / bk;
  int ks = (2 * 152 + gx * gy - 1) / (gx * gy);
  if (ks > nk) ks = nk;
  if (ks < 1) ks = 1;
  a.ksplit = ks;
  a.R = R;
  a.ldr = ldr;
  a.S = S;
  a.lds = lds;
  a.atomic = ks > 1 ? 1 : 0;
  a.err = err;
  *used_atomic = a.atomic;
  if (precision == HSS_PREC_TF32X2) return launch_t<HSS_PREC_TF32X2>(a, gx, gy, st);
  if (precision == HSS_PREC_BF16X3) return launch_t<HSS_PREC_BF16X3>(a, gx, gy, st);
  return cudaErrorInvalidValue;
}

int sample_tc_ksplit(int n, int ncols, int precision) {
  int N = ((ncols + 15) / 16) * 16;
  if (N > 128) N = 128;
  const int gx = (n + BM - 1) / BM, gy = (ncols + N - 1) / N;
  const int bk = precision == HSS_PREC_TF32X2 ? 32 : 64;
  const int nk = (n + bk - 1) / bk;
  int ks = (2 * 152 + gx * gy - 1) / (gx * gy);
  if (ks > nk) ks = nk;
  return ks < 1 ? 1 : ks;
}

}  // namespace hss
