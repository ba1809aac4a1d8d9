// Incrementing stopping test on one block (Algorithm 5, eq.
// stopping_criteria), one CTA per node side.  The block has already been
// projected, Sh = (I - Q Q^T)^2 S_k, by the batched tile products; this
// kernel evaluates
//   |Sh|_F / |S_k|_F < eps_r   or   |Sh|_F / sqrt(b) < eps_a,
// then (if neither holds) the Householder QR Sh = Q_k R_k and
//   min |diag R_k| < eps_a   or   min |diag R_k| < eps_r rho,
// with rho = |(R_1)_11| of the side's first block.  When every test fails,
// Q_k is formed explicitly (backward accumulation of the reflectors) and
// appended to the side's basis Q; a basis that reaches m columns spans the
// whole sample space and is sufficient.
#include "hss_internal.h"

namespace hss {
namespace {

constexpr int NT = 256, NW = NT / 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x / 32] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < NW; ++w) t += sh[w];
  return t;
}

__global__ void __launch_bounds__(NT) k_inc_qr(const IncJob* __restrict__ jobs) {
  const IncJob jb = jobs[blockIdx.x];
  const int m = jb.m, b = jb.b, tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  __shared__ double sh[NW];
  double* __restrict__ A = jb.Sh;   // m x b col-major, ld m

  double s = 0.0;
  for (long long e = tid; e < (long long)m * b; e += NT) {
    long long i = e / b;
    int c = (int)(e % b);
    double v = jb.S[i * jb.lds + jb.c0 + c];
    s = __fma_rn(v, v, s);
  }
  const double nS = sqrt(block_sum(s, sh));
  s = 0.0;
  for (long long e = tid; e < (long long)m * b; e += NT) s = __fma_rn(A[e], A[e], s);
  const double nSh = sqrt(block_sum(s, sh));
  if (tid == 0) { jb.res[0] = nS; jb.res[1] = nSh; jb.res[2] = -1.0; jb.res[3] = -1.0; }
  if (b == 0 || nS == 0.0 || nSh < jb.er * nS || nSh / sqrt((double)b) < jb.ea) {
    if (tid == 0) { jb.flag[0] = 1; jb.flag[1] = jb.q; }
    return;
  }
  // Householder QR of Sh, recording |R_jj|
  const int p = min(m, b);
  double mn = 1.0 / 0.0, r11 = 0.0;
  for (int j = 0; j < p; ++j) {
    double* cj = A + (long long)j * m;
    s = 0.0;
    for (int r = j + tid; r < m; r += NT) s = __fma_rn(cj[r], cj[r], s);
    s = block_sum(s, sh);
    const double alpha = sqrt(s);
    const double x0 = cj[j];
    __syncthreads();
    double beta, tau;
    if (alpha == 0.0) { beta = 0.0; tau = 0.0; }
    else {
      beta = x0 >= 0.0 ? -alpha : alpha;
      tau = (beta - x0) / beta;
      const double scal = 1.0 / (x0 - beta);
      for (int r = j + 1 + tid; r < m; r += NT) cj[r] *= scal;
    }
    if (tid == 0) { cj[j] = beta; jb.tau[j] = tau; }
    mn = fmin(mn, alpha);
    if (j == 0) r11 = alpha;
    __syncthreads();
    if (tau != 0.0) {
      for (int c = j + 1 + warp; c < b; c += NW) {
        double* col = A + (long long)c * m;
        double w = 0.0;
        for (int r = j + 1 + lane; r < m; r += 32) w = __fma_rn(cj[r], col[r], w);
        w = warp_sum(w) + col[j];
        const double tw = tau * w;
        for (int r = j + 1 + lane; r < m; r += 32) col[r] = __fma_rn(-tw, cj[r], col[r]);
        __syncwarp();
        if (lane == 0) col[j] -= tw;
      }
    }
    __syncthreads();
  }
  const double rho = jb.rho < 0.0 ? r11 : jb.rho;
  if (tid == 0) { jb.res[2] = mn; jb.res[3] = r11; }
  if (mn < jb.ea || mn < jb.er * rho) {
    if (tid == 0) { jb.flag[0] = 1; jb.flag[1] = jb.q; }
    return;
  }
  // Q_k = H_0 ... H_{p-1} [I; 0], first beff columns, into workspace T
  const int beff = min(b, m - jb.q);
  double* E = jb.T;   // m x beff col-major
  for (long long e = tid; e < (long long)m * beff; e += NT) {
    long long i = e % m;
    long long c = e / m;
    E[e] = (i == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = min(p, beff) - 1; j >= 0; --j) {
    const double tau = jb.tau[j];
    const double* v = A + (long long)j * m;
    if (tau != 0.0) {
      for (int c = j + warp; c < beff; c += NW) {
        double* col = E + (long long)c * m;
        double w = col[j];
        double part = 0.0;
        for (int r = j + 1 + lane; r < m; r += 32) part = __fma_rn(v[r], col[r], part);
        w += warp_sum(part);
        const double tw = tau * w;
        for (int r = j + 1 + lane; r < m; r += 32) col[r] = __fma_rn(-tw, v[r], col[r]);
        __syncwarp();
        if (lane == 0) col[j] -= tw;
      }
    }
    __syncthreads();
  }
  for (long long e = tid; e < (long long)m * beff; e += NT) {
    long long i = e / beff;
    int c = (int)(e % beff);
    jb.Q[i * jb.lds + jb.q + c] = E[i + (long long)c * m];
  }
  if (tid == 0) {
    jb.flag[1] = jb.q + beff;
    jb.flag[0] = (jb.q + beff >= m) ? 1 : 0;
  }
}

}  // namespace

cudaError_t launch_inc_qr(const IncJob* jobs_dev, int njobs, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  k_inc_qr<<<njobs, NT, 0, st>>>(jobs_dev);
  return cudaGetLastError();
}

}  // namespace hss
