// Batched interpolative decomposition by QR with column pivoting (eq. ID):
// for every job, W = S^T (d x m, the sample's rows as columns) is factored
// as W Pi = Q [R1 R2], truncated at the first pivot that fails the rank
// rule, and X = R1^{-1} R2 (= E^T) is formed in place by back substitution.
//
// Rank rules (tolerances already divided by level(tau)):
//   rule 0 (plain):  stop at pivot j when |R_jj| <= eps_a or
//                    |R_jj| <= eps_r |R_11|;
//   rule 1 (HMT):    both tolerances divided by
//                    f(k) = 1 + 4 sqrt(d) / (d - k - 1) * sqrt(min(m_h, n_h)),
//                    k = j + 1, with f = infinity when d - k - 1 <= 0
//                    (eq. RRQRHMTstop, section 2.4.1); accepted when the
//                    stop came at k <= d - p, or when every row was selected.
//
// One CTA of 8 warps per job, working in global memory (the sample copy
// stays L2 resident).  Pivot = largest down-dated column norm (lowest index
// on ties) with the norm recomputed when cancellation has eaten half of the
// digits; the stop test uses the exact norm of the pivot column.
#include "hss_internal.h"

namespace hss {
namespace {

constexpr int NT = 256, NW = NT / 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void argmax_pair(double& v, int& i, double v2, int i2) {
  if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
}

__global__ void __launch_bounds__(NT) k_qrcp(const QrcpJob* __restrict__ jobs) {
  const QrcpJob jb = jobs[blockIdx.x];
  const int m = jb.m, d = jb.d, tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const long long ldw = jb.ldw;
  double* __restrict__ W = jb.W;
  double* __restrict__ nrm = jb.nrm;
  double* __restrict__ orig = jb.nrm + m;
  int* __restrict__ piv = jb.piv;
  __shared__ double sv[NW];
  __shared__ int si[NW];
  __shared__ double s_alpha, s_r11;
  __shared__ int s_p, s_stop;

  // W = S^T and the initial column norms
  for (int c = warp; c < m; c += NW) {
    const double* src = jb.S + (long long)c * jb.lds;
    double* dst = W + (long long)c * ldw;
    double s = 0.0;
    for (int r = lane; r < d; r += 32) {
      double v = src[r];
      dst[r] = v;
      s = __fma_rn(v, v, s);
    }
    s = warp_sum(s);
    if (lane == 0) { nrm[c] = sqrt(s); orig[c] = nrm[c]; piv[c] = c; }
  }
  __syncthreads();

  const int kmax = min(d, m);
  int k = kmax, stopped = 0;
  const double tol3z = 1.4901161193847656e-08;  // sqrt(2^-52)
  for (int j = 0; j < kmax; ++j) {
    // pivot: largest current norm among columns j..m-1
    double bv = -1.0;
    int bi = 0x7fffffff;
    for (int c = j + tid; c < m; c += NT) argmax_pair(bv, bi, nrm[c], c);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
      int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
      argmax_pair(bv, bi, v2, i2);
    }
    if (lane == 0) { sv[warp] = bv; si[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double v = sv[0];
      int i = si[0];
      for (int w = 1; w < NW; ++w) argmax_pair(v, i, sv[w], si[w]);
      s_p = i;
    }
    __syncthreads();
    const int p = s_p;
    if (p != j) {
      for (int r = tid; r < d; r += NT) {
        double t = W[r + j * ldw];
        W[r + j * ldw] = W[r + p * ldw];
        W[r + p * ldw] = t;
      }
      if (tid == 0) {
        double t = nrm[j]; nrm[j] = nrm[p]; nrm[p] = t;
        t = orig[j]; orig[j] = orig[p]; orig[p] = t;
        int ti = piv[j]; piv[j] = piv[p]; piv[p] = ti;
      }
    }
    __syncthreads();
    // exact norm of the pivot column below the diagonal
    double s = 0.0;
    for (int r = j + tid; r < d; r += NT) {
      double v = W[r + j * ldw];
      s = __fma_rn(v, v, s);
    }
    s = warp_sum(s);
    if (lane == 0) sv[warp] = s;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < NW; ++w) t += sv[w];
      double alpha = sqrt(t);
      if (j == 0) s_r11 = alpha;
      double r11 = s_r11, thr_a = jb.ea, thr_r = jb.er * r11;
      if (jb.rule == 1) {
        double den = (double)(d - (j + 1) - 1);
        if (den <= 0.0) { thr_a = 0.0; thr_r = 0.0; }
        else {
          double f = 1.0 + 4.0 * sqrt((double)d) / den * sqrt((double)min(jb.mh, jb.nh));
          thr_a /= f;
          thr_r /= f;
        }
      }
      s_stop = (alpha <= thr_a || alpha <= thr_r) ? 1 : 0;
      s_alpha = alpha;
    }
    __syncthreads();
    if (s_stop) { k = j; stopped = 1; break; }
    // Householder reflector H = I - tau v v^T with v_j = 1, R_jj = beta
    const double alpha = s_alpha, x0 = W[j + j * ldw];
    const double beta = x0 >= 0.0 ? -alpha : alpha;
    const double tau = (beta - x0) / beta;
    const double scal = 1.0 / (x0 - beta);
    __syncthreads();
    for (int r = j + 1 + tid; r < d; r += NT) W[r + j * ldw] *= scal;
    if (tid == 0) W[j + j * ldw] = beta;
    __syncthreads();
    // apply to the trailing columns and down-date their norms
    for (int c = j + 1 + warp; c < m; c += NW) {
      double* col = W + (long long)c * ldw;
      double* vj = W + (long long)j * ldw;
      double wdot = 0.0;
      for (int r = j + 1 + lane; r < d; r += 32) wdot = __fma_rn(vj[r], col[r], wdot);
      wdot = warp_sum(wdot);
      const double top = col[j];
      wdot += top;
      const double tw = tau * wdot;
      for (int r = j + 1 + lane; r < d; r += 32) col[r] = __fma_rn(-tw, vj[r], col[r]);
      const double rjc = top - tw;
      int recompute = 0;
      __syncwarp();
      if (lane == 0) {
        col[j] = rjc;
        double nc = nrm[c];
        if (nc != 0.0) {
          double t = fabs(rjc) / nc;
          t = fmax(0.0, (1.0 + t) * (1.0 - t));
          double ratio = nc / orig[c];
          if (t * ratio * ratio <= tol3z) recompute = 1;
          else nrm[c] = nc * sqrt(t);
        }
      }
      recompute = __shfl_sync(0xffffffffu, recompute, 0);
      if (recompute) {
        __syncwarp();
        double s2 = 0.0;
        for (int r = j + 1 + lane; r < d; r += 32) s2 = __fma_rn(col[r], col[r], s2);
        s2 = warp_sum(s2);
        if (lane == 0) { nrm[c] = sqrt(s2); orig[c] = nrm[c]; }
      }
    }
    __syncthreads();
  }

  int accepted = 1;
  if (jb.rule == 1) accepted = stopped ? (k <= d - jb.p) : (k == m);
  if (jb.do_id && accepted && k > 0 && k < m) {
    // X = R1^{-1} R2 in place: one warp per right-hand side column
    for (int c = k + warp; c < m; c += NW) {
      double* col = W + (long long)c * ldw;
      for (int i = k - 1; i >= 0; --i) {
        __syncwarp();
        double xi = col[i] / W[i + (long long)i * ldw];
        __syncwarp();
        if (lane == 0) col[i] = xi;
        for (int r = lane; r < i; r += 32) col[r] = __fma_rn(-W[r + (long long)i * ldw], xi, col[r]);
      }
    }
  }
  if (tid == 0) { jb.out[0] = k; jb.out[1] = stopped; jb.out[2] = accepted; }
}

}  // namespace

cudaError_t launch_qrcp(const QrcpJob* jobs_dev, int njobs, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  k_qrcp<<<njobs, NT, 0, st>>>(jobs_dev);
  return cudaGetLastError();
}

}  // namespace hss
