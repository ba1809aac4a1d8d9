// FP64 sampling with the leaf diagonal blocks removed (eq. sample_off_diag at
// the leaf level):  Sr = (A - D^(L)) R  and  Sc = (A - D^(L))^T R.
//
// The leaf subtraction S(I_tau,:) - D_tau R(I_tau,:) of Algorithm 2 is folded
// into the product: entries whose row and column fall in the same leaf are
// replaced by zero while the tile of A is staged, and tiles lying entirely
// inside one leaf block are skipped.  The result is the same matrix as the
// paper's two-step form without the cancellation between A R and D R.
//
// Plain FP64 CUDA-core GEMM: 64 x 64 output tile per CTA, 256 threads with a
// 4 x 4 register tile each, K staged 16 at a time in shared memory.  The
// entries are loaded (dense A) or generated (Toeplitz, Gaussian, Laplace)
// by the staging loop.
#include "hss_internal.h"

namespace hss {
namespace {

constexpr int BM = 64, BN = 64, BK = 16;

template <bool TRANS>
__global__ void __launch_bounds__(256) k_sample_fp64(SrcDev src, int ncols, const double* __restrict__ R,
                                                     long long ldr, double* __restrict__ S, long long lds) {
  __shared__ double As[BK][BM + 2];
  __shared__ double Rs[BK][BN + 2];
  const int n = src.n;
  const int i0 = blockIdx.x * BM, c0 = blockIdx.y * BN;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int ilast = min(i0 + BM, n) - 1;
  const int lid_lo = src.leaf_id[i0], lid_hi = src.leaf_id[ilast];
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

  for (int k0 = 0; k0 < n; k0 += BK) {
    const int klast = min(k0 + BK, n) - 1;
    const int kid_lo = src.leaf_id[k0], kid_hi = src.leaf_id[klast];
    if (lid_lo == lid_hi && kid_lo == kid_hi && lid_lo == kid_lo) continue;  // inside one leaf
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int il, kk;
      if (!TRANS) { il = tid % BM; kk = tid / BM + 4 * q; }
      else { kk = tid % BK; il = tid / BK + 16 * q; }
      int i = i0 + il, k = k0 + kk;
      double v = 0.0;
      if (i < n && k < n && src.leaf_id[i] != src.leaf_id[k])
        v = TRANS ? entry(src, k, i) : entry(src, i, k);
      As[kk][il] = v;
      int cc = tid / BK + 16 * q, kr = tid % BK;
      int c = c0 + cc, kg = k0 + kr;
      Rs[kr][cc] = (c < ncols && kg < n) ? R[(long long)kg + (long long)c * ldr] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) { a[t] = As[kk][ty * 4 + t]; b[t] = Rs[kk][tx * 4 + t]; }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = __fma_rn(a[x], b[y], acc[x][y]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    int i = i0 + ty * 4 + x;
    if (i >= n) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      int c = c0 + tx * 4 + y;
      if (c < ncols) S[(long long)i * lds + c] = acc[x][y];
    }
  }
}

}  // namespace

cudaError_t launch_sample_fp64(const SrcDev& src, int ncols, const double* R, long long ldr,
                               double* Sr, double* Sc, long long lds, cudaStream_t st) {
  if (src.kind < HSS_SRC_DENSE || src.kind > HSS_SRC_LAPLACE) return cudaErrorInvalidValue;   // no entries on the device
  if (src.n <= 0 || ncols <= 0) return cudaSuccess;
  dim3 grid((src.n + BM - 1) / BM, (ncols + BN - 1) / BN);
  if (Sr) k_sample_fp64<false><<<grid, 256, 0, st>>>(src, ncols, R, ldr, Sr, lds);
  if (Sc) k_sample_fp64<true><<<grid, 256, 0, st>>>(src, ncols, R, ldr, Sc, lds);
  return cudaGetLastError();
}

}  // namespace hss
