// Batched strided FP64 tile products for the small dense steps of the
// method, all nodes of a tree level in one launch:
//  - the upward merge of Algorithm 2 (ComputeLocalSamples, non-leaf):
//      tau.S^r = [nu1.S^r(nu1.J^r,:) - B12 nu2.R^r ; nu2.S^r(nu2.J^r,:) - B21 nu1.R^r]
//    (row gather of the child sample, product with the B generator);
//  - ReduceLocalSamples: tau.R^r = V^T x = x(J^c) + Xc x(J^c complement)
//    (eq. ID: V = Pi [I; Xc^T]);
//  - the iterated block Gram-Schmidt products Q^T S and S - Q T of
//    Algorithm 5;
//  - the sweeps of the HSS product.
// Each CTA computes one 64 x 64 tile of one job (tile list built on the
// host); operands are read through row-gather / two-block views.
#include "hss_internal.h"

namespace hss {
namespace {

constexpr int TM = 64, TN = 64, TK = 16;

__device__ __forceinline__ double ld_op(const Opnd& o, int i, int l) {
  int r = o.rows ? o.rows[i] : i;
  const double* b = o.p;
  if (r >= o.split) { b = o.p2; r -= o.split; }
  return b[(long long)r * o.rs + (long long)l * o.cs];
}

__global__ void __launch_bounds__(256) k_gemm(const GemmJob* __restrict__ jobs,
                                              const GemmTile* __restrict__ tiles) {
  __shared__ double As[TK][TM + 2];
  __shared__ double Bs[TK][TN + 2];
  const GemmTile tl = tiles[blockIdx.x];
  const GemmJob jb = jobs[tl.job];
  const int i0 = tl.ti * TM, j0 = tl.tj * TN;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  const int kb = tl.k0, ke = tl.k1;
  const bool split = kb > 0 || ke < jb.K;
  for (int l0 = kb; l0 < ke; l0 += TK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int il = tid % TM, kk = tid / TM + 4 * q;
      int i = i0 + il, l = l0 + kk;
      As[kk][il] = (i < jb.M && l < ke) ? ld_op(jb.A, i, l) : 0.0;
      int jl = tid % TN;
      int j = j0 + jl;
      Bs[kk][jl] = (j < jb.N && l < ke) ? ld_op(jb.B, l, j) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) { a[t] = As[kk][ty * 4 + t]; b[t] = Bs[kk][tx * 4 + t]; }
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
    if (i >= jb.M) continue;
    int r = jb.c_rows ? jb.c_rows[i] : i;
    double* base = jb.C;
    if (r >= jb.c_split) { base = jb.C2; r -= jb.c_split; }
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      int j = j0 + tx * 4 + y;
      if (j >= jb.N) continue;
      double* dst = base + (long long)r * jb.c_rs + (long long)j * jb.c_cs;
      if (split) {
        atomicAdd(dst, jb.alpha * acc[x][y]);
        continue;
      }
      double v = jb.alpha * acc[x][y];
      if (jb.beta != 0.0) v += jb.beta * ld_op(jb.C0, i, j);
      if (jb.gamma != 0.0) v += jb.gamma * *dst;
      *dst = v;
    }
  }
}

}  // namespace

cudaError_t launch_gemm(const GemmJob* jobs_dev, const GemmTile* tiles_dev, int ntiles,
                        cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  k_gemm<<<ntiles, 256, 0, st>>>(jobs_dev, tiles_dev);
  return cudaGetLastError();
}

}  // namespace hss
