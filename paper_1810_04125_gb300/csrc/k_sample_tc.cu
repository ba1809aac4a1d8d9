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
// Every product of terms is exact in FP32; partial sums are kept short in
// TMEM and carried in float-float registers (see "Accumulation" below).
//
// Two kernels share the tile format: the packed kernel streams a dense A that
// was split once into canonical tiles (cp.async.bulk into an mbarrier ring);
// the generating kernel computes the entries (Toeplitz table lookups, point
// kernels) in its producer warps.  In both, one thread issues tcgen05.mma, the
// R tile arrives pre-packed by bulk copy, and every mbarrier wait is bounded
// (about 2 s of %globaltimer): on expiry the kernel records an error code,
// leaves its loops, frees its TMEM and returns.
//
// The shared-memory tile layout and the accumulation scheme are described in
// tc_common.cuh.
#include <stdint.h>

#include <algorithm>

#include "tc_common.cuh"

namespace hss {
namespace {

constexpr int NSTAGE = 3;                  // stages of the generating kernel

// Entry A(i, j) for the generating producers.  The Laplace kernel
// 1 / (4 pi |x_i - x_j|) avoids the FP64 square root and division (long
// sequences on the FP64 pipe, which bounds this kernel): |x_i - x_j|^-1 from
// the FP32 reciprocal square root of r^2, refined by one Newton-Raphson step
// for x^(-1/2), y1 = y0 (3 - r^2 y0^2) / 2, in FP64 — relative error about
// 1.5 e0^2 for an initial error e0 ~ 1e-7, far below the split that follows.
// r^2 outside the FP32 normal range, the diagonal and the other kinds take
// the plain definition.
__device__ __forceinline__ double entry_gen(const SrcDev& s, int i, int j) {
  if (s.kind != HSS_SRC_LAPLACE || i == j) return entry(s, i, j);
  double r2 = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double t = s.a[i + c * s.ld] - s.a[j + c * s.ld];
    r2 = __fma_rn(t, t, r2);
  }
  const float r2f = __double2float_rn(r2);
  if (!(r2f >= 1.1754943508222875e-38f) || !(r2f <= 1e38f)) return entry(s, i, j);
  const double y0 = (double)rsqrtf(r2f);
  const double y1 = y0 * __fma_rn(-0.5 * r2 * y0, y0, 1.5);
  return y1 * (1.0 / (4.0 * 3.141592653589793));
}

// ---------------------------------------------------------------------------
// Generating kernel (entries computed by the producer warps).
// Warps 0-7: generate the A tile of each stage, drain chains, write the
// result; warp 8: TMEM allocation and (lane 0) the MMA issue.  The R tile of
// each stage comes pre-packed and is moved by warp 0 lane 0 with one bulk
// copy (expect_tx on the stage barrier, which also counts the 256
// producer arrivals).
struct TcArgs {
  SrcDev src;
  int leaf;
  int trans;
  int ncols;          // sample columns of this launch
  int N;              // columns per CTA tile (32, 64 or 128)
  int tmem_cols;      // power of two >= 4 N
  int ksplit;         // CTAs along K
  int nkt;            // k-tiles of K
  int drain;          // k-tiles per accumulation chain
  const uint8_t* Rp;  // packed R tiles (ct, kt), N x BK each
  double* S;          // row-major output, row stride lds
  long long lds;
  int atomic;         // 1: add into S (pre-zeroed); 0: store
  int* err;
  const void* toep;   // Toeplitz source: its diagonals split into the T terms
                      // (entry of A_ij at (i - j) + n - 1: TF32 x 2 both terms
                      // in one 8-byte word, BF16 x 3 term-major), or NULL
};

constexpr int GEN_WARPS = 16;
// k-tiles per accumulation chain (generated entries): TF32 x 2 carries its
// chains four k-tiles long (its samples serve tolerances >= 1e-4; measured
// error of the samples below 5e-7), BF16 x 3 two (tolerances down to 1e-6)
__host__ __device__ constexpr int drain_gen(int precision) { return precision == HSS_PREC_TF32X2 ? 4 : 2; }
constexpr int TW = 80;   // window entries per term and producer warp (>= 8 + BK - 1)

// The diagonals c_t of a Toeplitz matrix (A_ij = c_{i-j}: the first column
// for i >= j, the first row for i < j), t = -(n-1) .. n-1, split into the T
// terms of the mixed form exactly as the producers split an entry: the
// generating kernel then assembles a tile from a window of consecutive
// diagonals instead of evaluating and splitting every entry.  TF32 x 2: the
// two terms of a diagonal side by side (one 8-byte word); BF16 x 3: term
// after term (2n - 1 entries each).
template <int PREC>
__global__ void k_toeplitz_terms(const double* col, const double* row, int n, void* out) {
  using SP = Split<PREC>;
  constexpr int T = SP::T, EV = SP::EV;
  const long long len = 2LL * n - 1;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < len; q += (long long)gridDim.x * blockDim.x) {
    const long long t = q - (n - 1);
    double v[EV];
    const double x = t >= 0 ? col[t] : row[-t];
#pragma unroll
    for (int e = 0; e < EV; ++e) v[e] = x;
    uint4 ch[T];
    SP::split(v, ch);
    if constexpr (PREC == HSS_PREC_TF32X2) {
      ((uint2*)out)[q] = make_uint2(ch[0].x, ch[1].x);
    } else {
#pragma unroll
      for (int k = 0; k < T; ++k) ((uint16_t*)out)[k * len + q] = (uint16_t)(ch[k].x & 0xFFFFu);
    }
  }
}
constexpr int GEN_THREADS = GEN_WARPS * 32 + 32;

template <int PREC, int NH, int TRANS>
__global__ void __maxnreg__(96) k_sample_tc_gen(TcArgs a) {
  using SP = Split<PREC>;
  constexpr int T = SP::T, EV = SP::EV, BK = SP::BK, KC = BK / EV;
  constexpr int DR = drain_gen(PREC);
  constexpr int NP = GEN_WARPS * 32;
  extern __shared__ __align__(1024) uint8_t smem[];
  const int n = a.src.n, N = a.N;
  const uint32_t tileB = (uint32_t)N * 128u;
  const uint32_t stage_bytes = T * TILE_A_BYTES + tileB;
  uint64_t* full = (uint64_t*)(smem + NSTAGE * stage_bytes);
  uint64_t* empty = full + NSTAGE;
  uint64_t* tfull = empty + NSTAGE;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = (uint32_t*)(tempty + 2);
  int* lrow_lo = (int*)(tmem_slot + 4);
  int* lrow_hi = lrow_lo + BM;
  // per producer warp: T window rows of TW diagonals (Toeplitz path)
  uint32_t* win32 = (uint32_t*)(lrow_hi + BM) + (size_t)(threadIdx.x / 32) * T * TW;
  uint16_t* win16 = (uint16_t*)win32;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int rb = blockIdx.x, ct = blockIdx.y;
  const int row0 = rb * BM, col0 = ct * N;
  const int kt0 = (int)((long long)a.nkt * blockIdx.z / a.ksplit);
  const int kt1 = (int)((long long)a.nkt * (blockIdx.z + 1) / a.ksplit);
  const int nk = kt1 - kt0;
  const int nchain = (nk + DR - 1) / DR;
  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) { mbar_init(&full[s], NP + 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], GEN_WARPS); }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < BM) {
    int r = row0 + tid, lo = 0x7fffffff, hi = 0x7fffffff;
    if (r < n) leaf_range(r, n, a.leaf, lo, hi);
    lrow_lo[tid] = lo;
    lrow_hi[tid] = hi;
  }
  if (warp == GEN_WARPS) {
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
  const uint8_t* gB = a.Rp + ((size_t)ct * a.nkt + kt0) * tileB;

  if (warp < GEN_WARPS) {
    const int q = warp % 4, h = warp / 4;
    // this warp's rows (Toeplitz path): all below n, and the union of their
    // leaf blocks [wlo, whi)
    int wlo = 0x7fffffff, whi = -1;
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) {
      wlo = min(wlo, lrow_lo[8 * warp + rr]);
      whi = max(whi, lrow_hi[8 * warp + rr]);
    }
    const bool rows_ok = row0 + 8 * warp + 8 <= n;
    float s[NH], e[NH];
#pragma unroll
    for (int j = 0; j < NH; ++j) { s[j] = 0.f; e[j] = 0.f; }
    bool ok = true;
    int drained = 0;   // chains drained so far
    // the Toeplitz diagonal terms: entry t of term k at tterm[k][t], |t| < n
    const uint2* tterm64 = a.toep ? (const uint2*)a.toep + (n - 1) : nullptr;
    const uint16_t* tterm16 = a.toep ? (const uint16_t*)a.toep + (n - 1) : nullptr;
    uint2* win64 = (uint2*)win32;
    const long long tlen = 2LL * n - 1;
    int st = 0;
    uint32_t ph = 0u;
    for (int it = 0; it < nk && ok; ++it) {
      if (it > 0 && ++st == NSTAGE) { st = 0; ph ^= 1u; }
      if (!mbar_wait_warp(&empty[st], ph ^ 1u, a.err, 2)) { ok = false; break; }
      uint8_t* sp = smem + st * stage_bytes;
      if (tid == 0) {
        mbar_expect_tx(&full[st], tileB);
        bulk_g2s(sp + T * TILE_A_BYTES, gB + (size_t)it * tileB, tileB, &full[st]);
      }
      const int k0 = (kt0 + it) * BK;
      if (a.toep) {
        // Toeplitz: this warp's 8 rows of the tile from a window of 8 + BK - 1
        // consecutive diagonals (orientation 0: A(r, k) = c_{r - k}; 1:
        // A(k, r) = c_{k - r}), masked only where the rows reach past n or a
        // row's leaf block meets the tile's columns
        const int rw = 8 * warp;
        const int tb = TRANS ? k0 - row0 - rw - 7 : row0 - k0 + rw - (BK - 1);
        __syncwarp();
#pragma unroll
        for (int qq0 = 0; qq0 < 8 + BK - 1; qq0 += 32) {
          const int qq = qq0 + lane;
          if (qq < 8 + BK - 1) {
            const int t = tb + qq;
            const bool in = t > -n && t < n;
            if constexpr (PREC == HSS_PREC_TF32X2) {
              win64[qq] = in ? tterm64[t] : make_uint2(0u, 0u);
            } else {
#pragma unroll
              for (int k = 0; k < T; ++k) win16[k * TW + qq] = in ? tterm16[k * tlen + t] : (uint16_t)0;
            }
          }
        }
        __syncwarp();
        const bool clean = rows_ok && k0 + BK <= n && (k0 + BK <= wlo || k0 >= whi);
#pragma unroll
        for (int i2 = 0; i2 < 2; ++i2) {
          const int idx = lane + 32 * i2, rl = idx % 8, c = idx / 8, r = rw + rl;
          // window position of the chunk's first entry; the next entries
          // step by +1 (orientation 1) or -1 (orientation 0)
          const int q0 = TRANS ? c * EV - rl + 7 : rl - c * EV + (BK - 1);
          constexpr int dq = TRANS ? 1 : -1;
          uint4 chunk[T];
          if (PREC == HSS_PREC_TF32X2 && clean) {
            uint2 w[4];
#pragma unroll
            for (int e2 = 0; e2 < 4; ++e2) w[e2] = win64[q0 + dq * e2];
            chunk[0] = make_uint4(w[0].x, w[1].x, w[2].x, w[3].x);
            chunk[T - 1] = make_uint4(w[0].y, w[1].y, w[2].y, w[3].y);
          } else if (PREC == HSS_PREC_TF32X2) {
            const int gr = row0 + r, lo = lrow_lo[r], hi = lrow_hi[r];
            uint2 w[4];
#pragma unroll
            for (int e2 = 0; e2 < 4; ++e2) {
              const int gk = k0 + c * EV + e2;
              const bool keep = gr < n && gk < n && (gk < lo || gk >= hi);
              w[e2] = keep ? win64[q0 + dq * e2] : make_uint2(0u, 0u);
            }
            chunk[0] = make_uint4(w[0].x, w[1].x, w[2].x, w[3].x);
            chunk[T - 1] = make_uint4(w[0].y, w[1].y, w[2].y, w[3].y);
          } else if (clean) {
#pragma unroll
            for (int k = 0; k < T; ++k) {
              uint32_t wv[4];
#pragma unroll
              for (int e2 = 0; e2 < 4; ++e2)
                wv[e2] = (uint32_t)win16[k * TW + q0 + dq * (2 * e2)] |
                         ((uint32_t)win16[k * TW + q0 + dq * (2 * e2 + 1)] << 16);
              chunk[k] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
            }
          } else {
            const int gr = row0 + r, lo = lrow_lo[r], hi = lrow_hi[r];
#pragma unroll
            for (int k = 0; k < T; ++k) {
              uint32_t wv[4];
#pragma unroll
              for (int e2 = 0; e2 < 4; ++e2) {
                uint32_t pair = 0u;
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                  const int x = 2 * e2 + hh;
                  const int gk = k0 + c * EV + x;
                  const bool keep = gr < n && gk < n && (gk < lo || gk >= hi);
                  pair |= (keep ? (uint32_t)win16[k * TW + q0 + dq * x] : 0u) << (16 * hh);
                }
                wv[e2] = pair;
              }
              chunk[k] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
            }
          }
          const uint32_t off = (uint32_t)(r / 8) * 1024u + (uint32_t)c * 128u + (uint32_t)(r % 8) * 16u;
#pragma unroll
          for (int t = 0; t < T; ++t) *(uint4*)(sp + t * TILE_A_BYTES + off) = chunk[t];
        }
      } else {
        for (int u = tid; u < BM * KC; u += NP) {
          int r, c;
          if (!TRANS) { r = u % BM; c = u / BM; }
          else { r = (u / (8 * KC)) * 8 + (u % 8); c = (u / 8) % KC; }
          const int gr = row0 + r, lo = lrow_lo[r], hi = lrow_hi[r];
          double v[EV];
#pragma unroll
          for (int x = 0; x < EV; ++x) {
            const int gk = k0 + c * EV + x;
            double val = 0.0;
            if (gr < n && gk < n && (gk < lo || gk >= hi))
              val = TRANS ? entry_gen(a.src, gk, gr) : entry_gen(a.src, gr, gk);
            v[x] = val;
          }
          uint4 chunk[T];
          SP::split(v, chunk);
          const uint32_t off = (uint32_t)(r / 8) * 1024u + (uint32_t)c * 128u + (uint32_t)(r % 8) * 16u;
#pragma unroll
          for (int t = 0; t < T; ++t) *(uint4*)(sp + t * TILE_A_BYTES + off) = chunk[t];
        }
      }
      fence_async_smem();
      mbar_arrive(&full[st]);
      // after the last tile of chain c, drain chain c-1
      const int c = it / DR;
      if ((it % DR == DR - 1 || it == nk - 1) && c >= 1) {
        const int cd = c - 1, b = cd & 1;
        if (!mbar_wait_warp(&tfull[b], (uint32_t)(cd >> 1) & 1u, a.err, 6)) { ok = false; break; }
        tc_fence_after();
        drain_chain<NH>(tmem, N, b, q, h, s, e);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[b]);
        drained = c;
      }
    }
    // drain what is left (the last chain)
    for (int cd = drained; ok && cd < nchain; ++cd) {
      const int b = cd & 1;
      if (!mbar_wait_warp(&tfull[b], (uint32_t)(cd >> 1) & 1u, a.err, 7)) { ok = false; break; }
      tc_fence_after();
      drain_chain<NH>(tmem, N, b, q, h, s, e);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[b]);
    }
    if (ok) store_row<NH>(a.S, a.lds, n, a.ncols, row0 + 32 * q + lane, col0 + h * NH, a.atomic, s, e);
  } else if (lane == 0) {
    // ------------------------------------------------------------- MMA issuer
    const uint32_t id = idesc(SP::FMT, (uint32_t)N);
    int st = 0;
    uint32_t ph = 0u;
    for (int it = 0; it < nk; ++it) {
      if (it > 0 && ++st == NSTAGE) { st = 0; ph ^= 1u; }
      const int c = it / DR, b = c & 1;
      const bool first = (it % DR) == 0;
      if (first && !mbar_wait(&tempty[b], ((uint32_t)(c >> 1) & 1u) ^ 1u, a.err, 8)) break;
      if (!mbar_wait(&full[st], ph, a.err, 3)) break;
      tc_fence_after();
      mma_ktile<PREC>(smem_u32(smem + st * stage_bytes), tmem, N, b, first, id);
      mma_commit(&empty[st]);
      if (it % DR == DR - 1 || it == nk - 1) mma_commit(&tfull[b]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == GEN_WARPS) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)a.tmem_cols)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// Packed path (a dense A is re-read on every pass): the operands are split
// once into canonical K-major tiles in global memory,
//   A, orientation o: tile (rb, kt) = T consecutive 16 KB term tiles at
//       ((o * nrb + rb) * nkt + kt) * T * 16 KB        (leaf diagonal zeroed)
//   R: tile (ct, kt) of N rows x BK at (ct * nkt + kt) * N * 128 bytes,
// and the main loop moves whole tiles with cp.async.bulk issued by one
// thread, completing on the stage mbarrier (expect_tx).  Warp 0 lane 0
// copies, warp 1 owns TMEM and (lane 0) issues the MMAs, warps 2-9 drain
// chains and write the result.

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
    for (int x = 0; x < EV; ++x) {
      const int gk = k0 + c * EV + x;
      double val = 0.0;
      if (gr < n && gk < n && (gk < lo || gk >= hi)) val = o ? entry_gen(src, gk, gr) : entry_gen(src, gr, gk);
      v[x] = val;
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
    for (int x = 0; x < EV; ++x) {
      const int gk = kt * BK + c * EV + x;
      v[x] = (gc < ncols && gk < n) ? R[(long long)gk + (long long)gc * ldr] : 0.0;
    }
    const uint32_t off = (uint32_t)(r / 8) * 1024u + (uint32_t)c * 128u + (uint32_t)(r % 8) * 16u;
    *(uint4*)(dst + off) = SP::pack_r(v);
  }
}

struct TcPackedArgs {
  const uint8_t* A;
  const uint8_t* Rp;
  int n, nrb, nkt, N, ncols, tmem_cols, ksplit, trans, drain;
  double* S;
  long long lds;
  int atomic;
  int* err;
};

template <int PREC>
constexpr int packed_stages() { return PREC == HSS_PREC_TF32X2 ? 4 : 3; }

constexpr int PK_THREADS = 18 * 32;   // copy warp, MMA warp, 16 drain warps

template <int PREC, int NH>
__global__ void __maxnreg__(96) k_sample_tc_packed(TcPackedArgs a) {
  using SP = Split<PREC>;
  constexpr int T = SP::T, NS = packed_stages<PREC>();
  extern __shared__ __align__(1024) uint8_t smem[];
  const int N = a.N;
  const uint32_t tileB = (uint32_t)N * 128u;
  const uint32_t stage_bytes = T * TILE_A_BYTES + tileB;
  uint64_t* full = (uint64_t*)(smem + NS * stage_bytes);
  uint64_t* empty = full + NS;
  uint64_t* tfull = empty + NS;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = (uint32_t*)(tempty + 2);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  // column tiles vary fastest across the grid: the CTAs that stream one
  // row block of A for different column tiles run together and share it
  // through L2, so A crosses HBM once per pass
  const int rb = blockIdx.y, ct = blockIdx.x;
  const int kt0 = (int)((long long)a.nkt * blockIdx.z / a.ksplit);
  const int kt1 = (int)((long long)a.nkt * (blockIdx.z + 1) / a.ksplit);
  const int nk = kt1 - kt0, DR = a.drain;
  const int nchain = (nk + DR - 1) / DR;
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], 16); }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
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
  if (warp == 0) {
    if (lane == 0) {
      for (int it = 0; it < nk; ++it) {
        const int s = it % NS;
        const uint32_t ph = (uint32_t)(it / NS) & 1u;
        if (!mbar_wait(&empty[s], ph ^ 1u, a.err, 12)) break;
        uint8_t* st = smem + s * stage_bytes;
        mbar_expect_tx(&full[s], stage_bytes);
#pragma unroll
        for (int t = 0; t < T; ++t)
          bulk_g2s(st + t * TILE_A_BYTES, gA + (size_t)it * (T * TILE_A_BYTES) + t * TILE_A_BYTES,
                   TILE_A_BYTES, &full[s]);
        bulk_g2s(st + T * TILE_A_BYTES, gB + (size_t)it * tileB, tileB, &full[s]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t id = idesc(SP::FMT, (uint32_t)N);
      for (int it = 0; it < nk; ++it) {
        const int s = it % NS;
        const uint32_t ph = (uint32_t)(it / NS) & 1u;
        const int c = it / DR, b = c & 1;
        const bool first = (it % DR) == 0;
        if (first && !mbar_wait(&tempty[b], ((uint32_t)(c >> 1) & 1u) ^ 1u, a.err, 15)) break;
        if (!mbar_wait(&full[s], ph, a.err, 13)) break;
        tc_fence_after();
        mma_ktile<PREC>(smem_u32(smem + s * stage_bytes), tmem, N, b, first, id);
        mma_commit(&empty[s]);
        if (it % DR == DR - 1 || it == nk - 1) mma_commit(&tfull[b]);
      }
    }
  } else {
    // --------------------------------------------------------- drain warps
    const int q = warp % 4, h = (warp - 2) / 4;
    float s[NH], e[NH];
#pragma unroll
    for (int j = 0; j < NH; ++j) { s[j] = 0.f; e[j] = 0.f; }
    bool ok = true;
    for (int cd = 0; cd < nchain; ++cd) {
      const int b = cd & 1;
      if (!mbar_wait_warp(&tfull[b], (uint32_t)(cd >> 1) & 1u, a.err, 14)) { ok = false; break; }
      tc_fence_after();
      drain_chain<NH>(tmem, N, b, q, h, s, e);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[b]);
    }
    if (ok && nk > 0)
      store_row<NH>(a.S, a.lds, a.n, a.ncols, rb * BM + 32 * q + lane, ct * N + h * NH, a.atomic, s, e);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)a.tmem_cols)
                 : "memory");
  }
}

int tile_n(int ncols) { return ncols <= 64 ? 64 : 128; }

int tmem_cols_for(int N) {
  int tc = 32;
  while (tc < 4 * N) tc *= 2;
  return tc;
}

constexpr int DRAIN_PACKED = 2;   // k-tiles per accumulation chain (dense, packed)

template <int PREC>
cudaError_t launch_packed_t(const TcPackedArgs& a, int gx, int gy, cudaStream_t st) {
  constexpr int T = Split<PREC>::T, NS = packed_stages<PREC>();
  const size_t sm = (size_t)NS * (T * TILE_A_BYTES + (size_t)a.N * 128) + 8 * (2 * NS + 4) + 16 + 1024;
  dim3 grid(gy, gx, a.ksplit);   // x: column tiles, y: row blocks
#define HSS_LAUNCH_PK(NHV)                                                                          \
  do {                                                                                              \
    cudaError_t e = cudaFuncSetAttribute(k_sample_tc_packed<PREC, NHV>,                             \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);     \
    if (e != cudaSuccess) return e;                                                                 \
    k_sample_tc_packed<PREC, NHV><<<grid, PK_THREADS, sm, st>>>(a);                                 \
  } while (0)
  if (a.N == 64) HSS_LAUNCH_PK(16);
  else HSS_LAUNCH_PK(32);
#undef HSS_LAUNCH_PK
  return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_gen_t(const TcArgs& a, int gx, int gy, cudaStream_t st) {
  constexpr int T = Split<PREC>::T;
  const size_t sm = (size_t)NSTAGE * (T * TILE_A_BYTES + (size_t)a.N * 128) + 8 * (2 * NSTAGE + 4) + 16 +
                    2 * BM * sizeof(int) + (size_t)GEN_WARPS * T * TW * sizeof(uint32_t) + 1024;
  dim3 grid(gx, gy, a.ksplit);
#define HSS_LAUNCH_GEN(NHV, TR)                                                                     \
  do {                                                                                              \
    cudaError_t e = cudaFuncSetAttribute(k_sample_tc_gen<PREC, NHV, TR>,                            \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);     \
    if (e != cudaSuccess) return e;                                                                 \
    k_sample_tc_gen<PREC, NHV, TR><<<grid, GEN_THREADS, sm, st>>>(a);                               \
  } while (0)
  if (a.N == 64) {
    if (a.trans) HSS_LAUNCH_GEN(16, 1);
    else HSS_LAUNCH_GEN(16, 0);
  } else {
    if (a.trans) HSS_LAUNCH_GEN(32, 1);
    else HSS_LAUNCH_GEN(32, 0);
  }
#undef HSS_LAUNCH_GEN
  return cudaGetLastError();
}

int bk_of(int precision) { return precision == HSS_PREC_TF32X2 ? 32 : 64; }

// K split across CTAs: enough CTAs for `waves` waves, but at least 64 k-tiles
// per CTA so that the epilogue (one pass over the 128 x N tile) stays small
// against the main loop.
int ksplit_for(int gx, int gy, int nkt, int waves) {
  int ks = (waves * 152 + gx * gy - 1) / (gx * gy);
  const int cap = nkt / 64;
  if (ks > cap) ks = cap;
  return ks < 1 ? 1 : ks;
}

}  // namespace

size_t toeplitz_terms_bytes(int n, int precision) {
  return (size_t)(2LL * n - 1) * (precision == HSS_PREC_TF32X2 ? 2 * 4 : 3 * 2);
}

cudaError_t launch_toeplitz_terms(const SrcDev& src, int precision, void* out, cudaStream_t st) {
  if (src.kind != HSS_SRC_TOEPLITZ || src.n <= 0) return cudaErrorInvalidValue;
  const long long len = 2LL * src.n - 1;
  const unsigned grid = (unsigned)std::min<long long>((len + 255) / 256, 152LL * 16);
  if (precision == HSS_PREC_TF32X2) k_toeplitz_terms<HSS_PREC_TF32X2><<<grid, 256, 0, st>>>(src.a, src.b, src.n, out);
  else if (precision == HSS_PREC_BF16X3) k_toeplitz_terms<HSS_PREC_BF16X3><<<grid, 256, 0, st>>>(src.a, src.b, src.n, out);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

size_t packed_a_bytes(int n, int precision) {
  const int T = precision == HSS_PREC_TF32X2 ? 2 : 3, bk = bk_of(precision);
  const size_t nrb = (n + BM - 1) / BM, nkt = (n + bk - 1) / bk;
  return 2 * nrb * nkt * T * (size_t)TILE_A_BYTES;
}

size_t packed_r_bytes(int n, int ncols, int precision) {
  const int bk = bk_of(precision);
  const int N = tile_n(ncols);
  const size_t nct = (ncols + N - 1) / N, nkt = (n + bk - 1) / bk;
  return nct * nkt * (size_t)N * 128;
}

cudaError_t launch_pack_a(const SrcDev& src, int leaf, int precision, void* out, cudaStream_t st) {
  if (src.kind < HSS_SRC_DENSE || src.kind > HSS_SRC_LAPLACE) return cudaErrorInvalidValue;   // no entries on the device
  const int n = src.n;
  const int bk = bk_of(precision);
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
  const int bk = bk_of(precision);
  const int N = tile_n(ncols), nct = (ncols + N - 1) / N, nkt = (n + bk - 1) / bk;
  if (precision == HSS_PREC_TF32X2)
    k_pack_r<HSS_PREC_TF32X2><<<nct * nkt, 256, 0, st>>>(R, ldr, n, ncols, N, nkt, (uint8_t*)out);
  else
    k_pack_r<HSS_PREC_BF16X3><<<nct * nkt, 256, 0, st>>>(R, ldr, n, ncols, N, nkt, (uint8_t*)out);
  return cudaGetLastError();
}

int sample_tc_packed_ksplit(int n, int ncols, int precision) {
  const int N = tile_n(ncols);
  const int gx = (n + BM - 1) / BM, gy = (ncols + N - 1) / N, nkt = (n + bk_of(precision) - 1) / bk_of(precision);
  return ksplit_for(gx, gy, nkt, tuning_get().sample_waves_packed);
}

int sample_tc_ksplit(int n, int ncols, int precision) {
  const int N = tile_n(ncols);
  const int gx = (n + BM - 1) / BM, gy = (ncols + N - 1) / N, nkt = (n + bk_of(precision) - 1) / bk_of(precision);
  return ksplit_for(gx, gy, nkt, tuning_get().sample_waves_generated);
}

cudaError_t launch_sample_tc_packed(const void* A, const void* Rp, int n, int ncols, int precision,
                                    int trans, double* S, long long lds, int* err, cudaStream_t st) {
  if (n <= 0 || ncols <= 0) return cudaSuccess;
  TcPackedArgs a;
  a.A = (const uint8_t*)A;
  a.Rp = (const uint8_t*)Rp;
  a.n = n;
  a.nrb = (n + BM - 1) / BM;
  a.nkt = (n + bk_of(precision) - 1) / bk_of(precision);
  a.N = tile_n(ncols);
  a.ncols = ncols;
  a.tmem_cols = tmem_cols_for(a.N);
  a.ksplit = sample_tc_packed_ksplit(n, ncols, precision);
  a.trans = trans;
  a.drain = DRAIN_PACKED;
  a.S = S;
  a.lds = lds;
  a.atomic = a.ksplit > 1 ? 1 : 0;
  a.err = err;
  const int gy = (ncols + a.N - 1) / a.N;
  if (precision == HSS_PREC_TF32X2) return launch_packed_t<HSS_PREC_TF32X2>(a, a.nrb, gy, st);
  if (precision == HSS_PREC_BF16X3) return launch_packed_t<HSS_PREC_BF16X3>(a, a.nrb, gy, st);
  return cudaErrorInvalidValue;
}

// S (+)= (A - D^(L))^{[T]} R with entries generated by the producer warps;
// Rp holds R packed by launch_pack_r; S must be zeroed by the caller when the
// K range is split across CTAs (*used_atomic).
cudaError_t launch_sample_tc(const SrcDev& src, int leaf, int precision, int trans, int ncols,
                             const void* Rp, double* S, long long lds, int* err, int* used_atomic,
                             const void* toep, cudaStream_t st) {
  if (src.kind < HSS_SRC_DENSE || src.kind > HSS_SRC_LAPLACE) return cudaErrorInvalidValue;   // no entries on the device
  const int n = src.n;
  if (n <= 0 || ncols <= 0) return cudaSuccess;
  TcArgs a;
  a.src = src;
  a.leaf = leaf;
  a.trans = trans;
  a.ncols = ncols;
  a.N = tile_n(ncols);
  a.tmem_cols = tmem_cols_for(a.N);
  a.nkt = (n + bk_of(precision) - 1) / bk_of(precision);
  const int gx = (n + BM - 1) / BM, gy = (ncols + a.N - 1) / a.N;
  a.ksplit = sample_tc_ksplit(n, ncols, precision);
  a.drain = drain_gen(precision);
  a.Rp = (const uint8_t*)Rp;
  a.S = S;
  a.lds = lds;
  a.atomic = a.ksplit > 1 ? 1 : 0;
  a.err = err;
  a.toep = src.kind == HSS_SRC_TOEPLITZ ? toep : nullptr;
  *used_atomic = a.atomic;
  if (precision == HSS_PREC_TF32X2) return launch_gen_t<HSS_PREC_TF32X2>(a, gx, gy, st);
  if (precision == HSS_PREC_BF16X3) return launch_gen_t<HSS_PREC_BF16X3>(a, gx, gy, st);
  return cudaErrorInvalidValue;
}

}  // namespace hss
