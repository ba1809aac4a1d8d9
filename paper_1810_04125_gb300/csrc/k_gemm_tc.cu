// Batched tile products on the tcgen05 tensor cores for the products that
// only form samples, used by the mixed-precision forms:
//  - the upward merge of Algorithm 2 (ComputeLocalSamples, non-leaf),
//      tau.S^r = [nu1.S^r(nu1.J^r,:) - B12 nu2.R^r ; nu2.S^r(nu2.J^r,:) - B21 nu1.R^r]
//    and the same for S^c with the transposed generators;
//  - ReduceLocalSamples, tau.R^r = x(J) + X x(J complement) (eq. ID).
// Each job computes C(rows_c(i), j) = alpha sum_l A(i,l) B(l,j) + beta C0(i,j)
// + gamma C(rows_c(i), j) (the FP64 tile kernel's contract), with A and B
// FP64 operands read through strided / row-gather views.
//
// Arithmetic: both operands are split while they are staged into three TF32
// terms, x = x0 + x1 + x2 + r with |r| < 2^-32 |x| (the leading three 11-bit
// fields of the FP64 significand, cut by integer operations), and the six
// term products with ta + tb <= 2 are issued: x0 y0 into the HI accumulator,
// the other five into LO.  The terms left out are below 2^-32 |A||B|, so the
// error is that of the FP32 accumulation in TMEM, kept small as in the
// sampling kernels: every k-tile (four MMAs into HI) is one chain, drained
// into float-float registers while the tensor core fills the other buffer.
// Both mixed forms (TF32X2, BF16X3 sampling) use this kernel: its error
// stays below that of their samples, whose leaf rows it combines.
//
// Warps 0-15 stage the operand tiles of each k-tile (128 rows of A, N rows of
// B^T, K-major canonical layout of tc_common.cuh), drain the chains and write
// the result; warp 16 owns TMEM and its lane 0 issues the MMAs.  Every wait
// is bounded (about 2 s); on expiry the kernel records an error code, frees
// its TMEM and returns.
#include <stdint.h>

#include "tc_common.cuh"

namespace hss {
namespace {

constexpr int GT_WARPS = 16;
constexpr int GT_THREADS = GT_WARPS * 32 + 32;
constexpr int GT_T = 3;          // TF32 terms per operand
constexpr int GT_BK = 32;        // K per k-tile (128 bytes of TF32 per row)
constexpr int GT_KC = GT_BK / 4; // 16-byte chunks per row
constexpr int GT_NPAIR = 6;      // (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)

template <int N>
constexpr int gt_stages() { return N == 128 ? 2 : 3; }

__device__ __forceinline__ int pair_a(int p) { return p < 1 ? 0 : (p < 3 ? p - 1 : p - 3); }
__device__ __forceinline__ int pair_b(int p) { return p < 1 ? 0 : (p < 3 ? 2 - p : 5 - p); }

// x = x0 + x1 + x2 + r, |r| < 2^-32 |x|: the leading three 11-bit fields of
// the FP64 significand, each as a TF32 value (bit patterns in t).  Integer
// operations only.  Terms below the FP32 normal range are dropped; zero and
// FP64 subnormals give zeros; Inf/NaN give an Inf/NaN leading term.
__device__ __forceinline__ void split3_tf32(double x, uint32_t* t) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
  const int E = (int)((u >> 52) & 0x7FFull);
  t[0] = t[1] = t[2] = 0u;
  if (E == 0) return;
  if (E == 0x7FF) {
    t[0] = sign | 0x7F800000u | (((u & 0xFFFFFFFFFFFFFull) != 0ull) ? 0x00400000u : 0u);
    return;
  }
  const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int e = E - 1023;
#pragma unroll
  for (int q = 0; q < GT_T; ++q) {
    const uint32_t c = (uint32_t)(m >> (42 - 11 * q)) & 0x7FFu;
    if (c == 0u) continue;
    const int lz = __clz(c) - 21;
    const int fe = e - 11 * q - lz;
    if (fe < -126) continue;
    if (fe > 127) { t[q] = sign | 0x7F800000u; continue; }
    t[q] = sign | ((uint32_t)(fe + 127) << 23) | (((c << lz) & 0x3FFu) << 13);
  }
}

__device__ __forceinline__ const double* op_row(const Opnd& o, int i) {
  int r = o.rows ? o.rows[i] : i;
  const double* b = o.p;
  if (r >= o.split) { b = o.p2; r -= o.split; }
  return b + (long long)r * o.rs;
}

// Stage one operand tile: `rows` tile rows (the output rows for A, the
// output columns for B) x GT_BK elements of K, split into GT_T terms.
// elem(t, l0, v) writes the four FP64 values of tile row t at k indices
// l0..l0+3 (0 outside the job).  rows_fast: consecutive lanes take
// consecutive tile rows (unit stride along the rows in global memory), else
// consecutive 16-byte chunks along K.
template <class F, int NP = GT_WARPS * 32>
__device__ __forceinline__ void stage_tile(uint8_t* dst, uint32_t term_bytes, int rows, bool rows_fast,
                                           int tid, F elem) {
  for (int u = tid; u < rows * GT_KC; u += NP) {
    int r, c;
    if (rows_fast) { r = u % rows; c = u / rows; }
    else { r = (u / (8 * GT_KC)) * 8 + (u % 8); c = (u / 8) % GT_KC; }
    double v[4];
    elem(r, c * 4, v);
    uint32_t w[4][GT_T];
#pragma unroll
    for (int x = 0; x < 4; ++x) split3_tf32(v[x], w[x]);
    const uint32_t off = (uint32_t)(r / 8) * 1024u + (uint32_t)c * 128u + (uint32_t)(r % 8) * 16u;
#pragma unroll
    for (int t = 0; t < GT_T; ++t)
      *(uint4*)(dst + t * term_bytes + off) = make_uint4(w[0][t], w[1][t], w[2][t], w[3][t]);
  }
}

__device__ __forceinline__ void mma_pairs(uint32_t base, uint32_t tileB, uint32_t tmem, int N, int b,
                                          uint32_t id) {
  const uint32_t hi = tmem + (uint32_t)((2 * b) * N), lo = tmem + (uint32_t)((2 * b + 1) * N);
  const uint32_t bbase = base + GT_T * TILE_A_BYTES;
#pragma unroll
  for (int ks = 0; ks < GT_BK / 8; ++ks) {
#pragma unroll
    for (int p = 0; p < GT_NPAIR; ++p) {
      const uint64_t ad = sdesc(base + pair_a(p) * TILE_A_BYTES + ks * 256u, 128u, 1024u);
      const uint64_t bd = sdesc(bbase + pair_b(p) * tileB + ks * 256u, 128u, 1024u);
      const uint32_t acc = (ks == 0 && p <= 1) ? 0u : 1u;   // each k-tile starts a chain
      mma<HSS_PREC_TF32X2>(p == 0 ? hi : lo, ad, bd, id, acc);
    }
  }
}

template <int N>
__global__ void __maxnreg__(96) k_gemm_tc(const GemmJob* __restrict__ jobs,
                                           const GemmTile* __restrict__ tiles, int tmem_cols, int* err) {
  constexpr int NH = N / 4, NS = gt_stages<N>();
  constexpr int NPROD = GT_WARPS * 32;
  constexpr uint32_t tileB = (uint32_t)N * 128u;
  constexpr uint32_t stage_bytes = GT_T * (TILE_A_BYTES + tileB);
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ GemmJob sj;
  uint64_t* full = (uint64_t*)(smem + NS * stage_bytes);
  uint64_t* empty = full + NS;
  uint64_t* tfull = empty + NS;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = (uint32_t*)(tempty + 2);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const GemmTile tl = tiles[blockIdx.x];
  if (tid == 0) {
    sj = jobs[tl.job];
    for (int s = 0; s < NS; ++s) { mbar_init(&full[s], NPROD); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], GT_WARPS); }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == GT_WARPS) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"((uint32_t)tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int M = sj.M, Nj = sj.N, K = sj.K;
  const int i0 = tl.ti * BM, j0 = tl.tj * N;
  const int nk = (K + GT_BK - 1) / GT_BK;   // one chain per k-tile

  if (warp < GT_WARPS) {
    const int q = warp % 4, h = warp / 4;
    float s[NH], e[NH];
#pragma unroll
    for (int j = 0; j < NH; ++j) { s[j] = 0.f; e[j] = 0.f; }
    // A rows contiguous in memory -> lanes along rows; B is staged as B^T
    // (tile rows = output columns): contiguous along its columns -> lanes
    // along rows
    const bool a_rows_fast = sj.A.rs == 1 && !sj.A.rows;
    const bool b_rows_fast = sj.B.cs == 1;
    bool ok = true;
    for (int it = 0; it < nk && ok; ++it) {
      const int st = it % NS;
      const uint32_t ph = (uint32_t)(it / NS) & 1u;
      if (!mbar_wait_warp(&empty[st], ph ^ 1u, err, 21)) { ok = false; break; }
      uint8_t* sp = smem + st * stage_bytes;
      const int k0 = it * GT_BK;
      stage_tile(sp, TILE_A_BYTES, BM, a_rows_fast, tid, [&](int r, int kc, double* v) {
        const int i = i0 + r;
        const double* row = i < M ? op_row(sj.A, i) : nullptr;
        const long long cs = sj.A.cs;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const int l = k0 + kc + x;
          v[x] = (row && l < K) ? row[(long long)l * cs] : 0.0;
        }
      });
      stage_tile(sp + GT_T * TILE_A_BYTES, tileB, N, b_rows_fast, tid, [&](int r, int kc, double* v) {
        const int j = j0 + r;
        const long long cs = sj.B.cs;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const int l = k0 + kc + x;
          v[x] = (j < Nj && l < K) ? op_row(sj.B, l)[(long long)j * cs] : 0.0;
        }
      });
      fence_async_smem();
      mbar_arrive(&full[st]);
      // drain the chain of the previous k-tile
      if (it >= 1) {
        const int cd = it - 1, b = cd & 1;
        if (!mbar_wait_warp(&tfull[b], (uint32_t)(cd >> 1) & 1u, err, 22)) { ok = false; break; }
        tc_fence_after();
        drain_chain<NH>(tmem, N, b, q, h, s, e);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[b]);
      }
    }
    if (ok && nk >= 1) {
      const int cd = nk - 1, b = cd & 1;
      if (!mbar_wait_warp(&tfull[b], (uint32_t)(cd >> 1) & 1u, err, 23)) ok = false;
      else {
        tc_fence_after();
        drain_chain<NH>(tmem, N, b, q, h, s, e);
        tc_fence_before();
      }
    }
    // epilogue: C(rows_c(i), j) = alpha acc + beta C0(i, j) + gamma C(...)
    const int i = i0 + 32 * q + lane;
    if (ok && i < M) {
      int r = sj.c_rows ? sj.c_rows[i] : i;
      double* base = sj.C;
      if (r >= sj.c_split) { base = sj.C2; r -= sj.c_split; }
      double* out = base + (long long)r * sj.c_rs;
      const double* c0 = sj.beta != 0.0 ? op_row(sj.C0, i) : nullptr;
      const double alpha = sj.alpha, beta = sj.beta, gamma = sj.gamma;
      const long long ccs = sj.c_cs, c0cs = sj.C0.cs;
      const int jb = j0 + h * NH;
#pragma unroll
      for (int x = 0; x < NH; ++x) {
        const int j = jb + x;
        if (j < Nj) {
          double v = alpha * (f2d_exact(s[x]) + f2d_exact(e[x]));
          if (c0) v += beta * c0[(long long)j * c0cs];
          double* dst = out + (long long)j * ccs;
          if (gamma != 0.0) v += gamma * *dst;
          *dst = v;
        }
      }
    }
  } else if (lane == 0) {
    const uint32_t id = idesc(2u, (uint32_t)N);
    for (int it = 0; it < nk; ++it) {
      const int st = it % NS;
      const uint32_t ph = (uint32_t)(it / NS) & 1u;
      const int b = it & 1;
      if (!mbar_wait(&tempty[b], ((uint32_t)(it >> 1) & 1u) ^ 1u, err, 24)) break;
      if (!mbar_wait(&full[st], ph, err, 25)) break;
      tc_fence_after();
      mma_pairs(smem_u32(smem + st * stage_bytes), tileB, tmem, N, b, id);
      mma_commit(&empty[st]);
      mma_commit(&tfull[b]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == GT_WARPS) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)tmem_cols)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// Packed operands.  k_gemm_tc splits every operand element again for every
// output tile that reads it (A once per column tile, B once per row tile);
// here each element is split once into its three terms, in the canonical
// layout of stage_tile, and the product kernel only moves whole tiles.
template <int N>
__global__ void __launch_bounds__(256) k_gemm_pack(const GemmJob* __restrict__ jobs,
                                                   const PackUnit* __restrict__ units) {
  constexpr uint32_t tileB = (uint32_t)N * 128u;
  const PackUnit u = units[blockIdx.x];
  const GemmJob& j = jobs[u.job];
  const int k0 = u.kt * GT_BK, K = j.K;
  if (u.which == 0) {
    uint8_t* dst = j.pa + ((size_t)u.tile * j.nkt + u.kt) * (GT_T * (size_t)TILE_A_BYTES);
    const int i0 = u.tile * BM, M = j.M;
    const bool rows_fast = j.A.rs == 1 && !j.A.rows;
    const long long cs = j.A.cs;
    auto elem = [&](int r, int kc, double* v) {
      const int i = i0 + r;
      const double* row = i < M ? op_row(j.A, i) : nullptr;
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        const int l = k0 + kc + x;
        v[x] = (row && l < K) ? row[(long long)l * cs] : 0.0;
      }
    };
    stage_tile<decltype(elem), 256>(dst, TILE_A_BYTES, BM, rows_fast, threadIdx.x, elem);
  } else {
    uint8_t* dst = j.pb + ((size_t)u.tile * j.nkt + u.kt) * (GT_T * (size_t)tileB);
    const int j0 = u.tile * N, Nj = j.N;
    const bool rows_fast = j.B.cs == 1;
    const long long cs = j.B.cs;
    auto elem = [&](int r, int kc, double* v) {
      const int c = j0 + r;
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        const int l = k0 + kc + x;
        v[x] = (c < Nj && l < K) ? op_row(j.B, l)[(long long)c * cs] : 0.0;
      }
    };
    stage_tile<decltype(elem), 256>(dst, tileB, N, rows_fast, threadIdx.x, elem);
  }
}

constexpr int GP_THREADS = (2 + GT_WARPS) * 32;   // copy warp, MMA warp, 16 drain warps

template <int N>
__global__ void __maxnreg__(96) k_gemm_tc_pk(const GemmJob* __restrict__ jobs,
                                              const GemmTile* __restrict__ tiles, int tmem_cols, int* err) {
  constexpr int NH = N / 4, NS = gt_stages<N>();
  constexpr uint32_t tileB = (uint32_t)N * 128u;
  constexpr uint32_t a_bytes = GT_T * TILE_A_BYTES, b_bytes = GT_T * tileB;
  constexpr uint32_t stage_bytes = a_bytes + b_bytes;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ GemmJob sj;
  uint64_t* full = (uint64_t*)(smem + NS * stage_bytes);
  uint64_t* empty = full + NS;
  uint64_t* tfull = empty + NS;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = (uint32_t*)(tempty + 2);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const GemmTile tl = tiles[blockIdx.x];
  if (tid == 0) {
    sj = jobs[tl.job];
    for (int s = 0; s < NS; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], GT_WARPS); }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"((uint32_t)tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int M = sj.M, Nj = sj.N, K = sj.K;
  const int i0 = tl.ti * BM, j0 = tl.tj * N;
  const int nk = (K + GT_BK - 1) / GT_BK;   // one chain per k-tile
  if (warp == 0) {
    if (lane == 0) {
      const uint8_t* gA = sj.pa + (size_t)tl.ti * sj.nkt * a_bytes;
      const uint8_t* gB = sj.pb + (size_t)tl.tj * sj.nkt * b_bytes;
      int st = 0;
      uint32_t ph = 0u;
      for (int it = 0; it < nk; ++it) {
        if (it > 0 && ++st == NS) { st = 0; ph ^= 1u; }
        if (!mbar_wait(&empty[st], ph ^ 1u, err, 26)) break;
        uint8_t* sp = smem + st * stage_bytes;
        mbar_expect_tx(&full[st], stage_bytes);
        bulk_g2s(sp, gA + (size_t)it * a_bytes, a_bytes, &full[st]);
        bulk_g2s(sp + a_bytes, gB + (size_t)it * b_bytes, b_bytes, &full[st]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t id = idesc(2u, (uint32_t)N);
      int st = 0;
      uint32_t ph = 0u;
      for (int it = 0; it < nk; ++it) {
        if (it > 0 && ++st == NS) { st = 0; ph ^= 1u; }
        const int b = it & 1;
        if (!mbar_wait(&tempty[b], ((uint32_t)(it >> 1) & 1u) ^ 1u, err, 27)) break;
        if (!mbar_wait(&full[st], ph, err, 28)) break;
        tc_fence_after();
        mma_pairs(smem_u32(smem + st * stage_bytes), tileB, tmem, N, b, id);
        mma_commit(&empty[st]);
        mma_commit(&tfull[b]);
      }
    }
  } else {
    // drain warps 2 .. 17: TMEM lane quarter warp % 4, column quarter h
    const int q = warp % 4, h = (warp - 2) / 4;
    float s[NH], e[NH];
#pragma unroll
    for (int x = 0; x < NH; ++x) { s[x] = 0.f; e[x] = 0.f; }
    bool ok = true;
    for (int cd = 0; cd < nk; ++cd) {
      const int b = cd & 1;
      if (!mbar_wait_warp(&tfull[b], (uint32_t)(cd >> 1) & 1u, err, 29)) { ok = false; break; }
      tc_fence_after();
      drain_chain<NH>(tmem, N, b, q, h, s, e);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[b]);
    }
    // epilogue: C(rows_c(i), j) = alpha acc + beta C0(i, j) + gamma C(...)
    const int i = i0 + 32 * q + lane;
    if (ok && i < M) {
      int r = sj.c_rows ? sj.c_rows[i] : i;
      double* base = sj.C;
      if (r >= sj.c_split) { base = sj.C2; r -= sj.c_split; }
      double* out = base + (long long)r * sj.c_rs;
      const double* c0 = sj.beta != 0.0 ? op_row(sj.C0, i) : nullptr;
      const double alpha = sj.alpha, beta = sj.beta, gamma = sj.gamma;
      const long long ccs = sj.c_cs, c0cs = sj.C0.cs;
      const int jb = j0 + h * NH;
#pragma unroll
      for (int x = 0; x < NH; ++x) {
        const int jj = jb + x;
        if (jj < Nj) {
          double v = alpha * (f2d_exact(s[x]) + f2d_exact(e[x]));
          if (c0) v += beta * c0[(long long)jj * c0cs];
          double* dst = out + (long long)jj * ccs;
          if (gamma != 0.0) v += gamma * *dst;
          *dst = v;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)tmem_cols)
                 : "memory");
  }
}

template <int N>
cudaError_t launch_t(const GemmJob* jobs, const GemmTile* tiles, int ntiles, int* err, cudaStream_t st) {
  constexpr int NS = gt_stages<N>();
  const size_t sm = (size_t)NS * GT_T * (TILE_A_BYTES + (size_t)N * 128) + 8 * (2 * NS + 4) + 16 + 1024;
  int tc = 32;
  while (tc < 4 * N) tc *= 2;
  cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_gemm_tc<N><<<ntiles, GT_THREADS, sm, st>>>(jobs, tiles, tc, err);
  return cudaGetLastError();
}

}  // namespace

// 64 columns per tile: the 16 drain warps then hold 16 float-float columns
// each, which fits the 96 registers a thread can have at 544 threads per CTA
// (a 128-column tile would spill).
int gemm_tc_tile_n(int) { return 64; }

cudaError_t launch_gemm_tc(const GemmJob* jobs_dev, const GemmTile* tiles_dev, int ntiles, int tile_n,
                           int* err, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  if (tile_n == 64) return launch_t<64>(jobs_dev, tiles_dev, ntiles, err, st);
  return cudaErrorInvalidValue;
}

size_t gemm_tc_tile_bytes(int which, int tile_n) {
  return which == 0 ? (size_t)GT_T * TILE_A_BYTES : (size_t)GT_T * tile_n * 128;
}

cudaError_t launch_gemm_tc_pack(const GemmJob* jobs_dev, const PackUnit* units_dev, int nunits, int tile_n,
                                cudaStream_t st) {
  if (nunits <= 0) return cudaSuccess;
  if (tile_n != 64) return cudaErrorInvalidValue;
  k_gemm_pack<64><<<nunits, 256, 0, st>>>(jobs_dev, units_dev);
  return cudaGetLastError();
}

cudaError_t launch_gemm_tc_packed(const GemmJob* jobs_dev, const GemmTile* tiles_dev, int ntiles, int tile_n,
                                  int* err, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  if (tile_n != 64) return cudaErrorInvalidValue;
  constexpr int N = 64, NS = gt_stages<64>();
  const size_t sm = (size_t)NS * GT_T * (TILE_A_BYTES + (size_t)N * 128) + 8 * (2 * NS + 4) + 16 + 1024;
  int tc = 32;
  while (tc < 4 * N) tc *= 2;
  cudaError_t e = cudaFuncSetAttribute(k_gemm_tc_pk<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_gemm_tc_pk<N><<<ntiles, GP_THREADS, sm, st>>>(jobs_dev, tiles_dev, tc, err);
  return cudaGetLastError();
}

}  // namespace hss
