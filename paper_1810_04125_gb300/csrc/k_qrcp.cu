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

// ---------------------------------------------------------------------------
// The same factorisation spread over a group of P CTAs per job, for tree
// levels with fewer node sides than SMs (one cooperative launch for the
// level).  Column slot c belongs to CTA rank c mod P.  Per pivot step:
//   every CTA: largest norm among its own slots >= j      -> group barrier
//   owner of slot j: global pivot, swap into slot j, exact pivot norm, the
//   stop decision and the reflector                        -> group barrier
//   every CTA: apply the reflector to its own slots > j and down-date their
//   norms.
// Data written by one CTA and read by another goes through L2 (ld/st .cg);
// the barrier is a monotonic counter per job with a bounded wait (about 2 s
// of %globaltimer, or as soon as another CTA has recorded an error).
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ bool group_barrier(unsigned* bar, unsigned P, unsigned& epoch, int* err, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    epoch += 1;
    const unsigned target = epoch * P;
    __threadfence();
    atomicAdd(bar, 1u);
    int ok = 1;
    const uint64_t t0 = gtimer();
    for (unsigned it = 1; ld_acquire(bar) < target; ++it) {
      if ((it & 63u) == 0) {
        if (*(volatile int*)err) { ok = 0; break; }
        if (gtimer() - t0 > 2000000000ull) { atomicCAS(err, 0, 6); ok = 0; break; }
      }
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

__global__ void __launch_bounds__(NT) k_qrcp_group(const QrcpJob* __restrict__ jobs,
                                                   const int2* __restrict__ map, int* err) {
  const int2 me = map[blockIdx.x];
  const QrcpJob jb = jobs[me.x];
  const int rank = me.y, P = jb.P;
  const int m = jb.m, d = jb.d, tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const long long ldw = jb.ldw;
  double* W = jb.W;
  double* nrm = jb.nrm;
  double* orig = jb.nrm + m;
  int* piv = jb.piv;
  __shared__ double sv[NW];
  __shared__ int si[NW];
  __shared__ int s_ok, s_p, s_stop;
  __shared__ double s_alpha;
  unsigned epoch = 0;

  // this CTA's slots: c = rank + P t
  for (int c = rank + P * warp; c < m; c += P * NW) {
    const double* src = jb.S + (long long)c * jb.lds;
    double* dst = W + (long long)c * ldw;
    double s = 0.0;
    for (int r = lane; r < d; r += 32) {
      double v = src[r];
      __stcg(dst + r, v);
      s = __fma_rn(v, v, s);
    }
    s = warp_sum(s);
    if (lane == 0) { __stcg(nrm + c, sqrt(s)); __stcg(orig + c, sqrt(s)); __stcg(piv + c, c); }
  }
  if (!group_barrier(jb.bar, P, epoch, err, &s_ok)) return;

  const int kmax = min(d, m);
  int k = kmax, stopped = 0;
  const double tol3z = 1.4901161193847656e-08;
  for (int j = 0; j < kmax; ++j) {
    // local argmax over own slots >= j
    double bv = -1.0;
    int bi = 0x7fffffff;
    int t0 = (j > rank) ? (j - rank + P - 1) / P : 0;
    for (int t = t0 + tid;; t += NT) {
      const int c = rank + P * t;
      if (c >= m) break;
      argmax_pair(bv, bi, __ldcg(nrm + c), c);
    }
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
      __stcg(jb.redv + rank, v);
      __stcg(jb.redi + rank, i);
    }
    if (!group_barrier(jb.bar, P, epoch, err, &s_ok)) return;

    if (j % P == rank) {
      // owner of slot j: pivot, swap, reflector, stop decision
      if (tid == 0) {
        double v = __ldcg(jb.redv);
        int i = __ldcg(jb.redi);
        for (int q = 1; q < P; ++q) argmax_pair(v, i, __ldcg(jb.redv + q), __ldcg(jb.redi + q));
        s_p = i;
      }
      __syncthreads();
      const int p = s_p;
      if (p != j) {
        for (int r = tid; r < d; r += NT) {
          double a = __ldcg(W + r + j * ldw), b = __ldcg(W + r + p * ldw);
          __stcg(W + r + j * ldw, b);
          __stcg(W + r + p * ldw, a);
        }
        if (tid == 0) {
          double t = __ldcg(nrm + j); __stcg(nrm + j, __ldcg(nrm + p)); __stcg(nrm + p, t);
          t = __ldcg(orig + j); __stcg(orig + j, __ldcg(orig + p)); __stcg(orig + p, t);
          int ti = __ldcg(piv + j); __stcg(piv + j, __ldcg(piv + p)); __stcg(piv + p, ti);
        }
      }
      __syncthreads();
      double s = 0.0;
      for (int r = j + tid; r < d; r += NT) {
        double v = __ldcg(W + r + j * ldw);
        s = __fma_rn(v, v, s);
      }
      s = warp_sum(s);
      if (lane == 0) sv[warp] = s;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < NW; ++w) t += sv[w];
        const double alpha = sqrt(t);
        if (j == 0) __stcg(jb.bcd + 3, alpha);
        const double r11 = (j == 0) ? alpha : __ldcg(jb.bcd + 3);
        double thr_a = jb.ea, thr_r = jb.er * r11;
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
      if (!s_stop) {
        const double alpha = s_alpha, x0 = __ldcg(W + j + j * ldw);
        const double beta = x0 >= 0.0 ? -alpha : alpha;
        const double tau = (beta - x0) / beta;
        const double scal = 1.0 / (x0 - beta);
        for (int r = j + 1 + tid; r < d; r += NT) __stcg(W + r + j * ldw, __ldcg(W + r + j * ldw) * scal);
        if (tid == 0) { __stcg(W + j + j * ldw, beta); __stcg(jb.bcd, tau); }
      }
      if (tid == 0) __stcg(jb.bci, s_stop);
    }
    if (!group_barrier(jb.bar, P, epoch, err, &s_ok)) return;
    if (tid == 0) s_stop = __ldcg(jb.bci);
    __syncthreads();
    if (s_stop) { k = j; stopped = 1; break; }
    const double tau = __ldcg(jb.bcd);
    const double* vj = W + (long long)j * ldw;
    // reflector on own slots > j, norm down-dating
    int tw0 = (j + 1 > rank) ? (j + 1 - rank + P - 1) / P : 0;
    for (int t = tw0 + warp;; t += NW) {
      const int c = rank + P * t;
      if (c >= m) break;
      double* col = W + (long long)c * ldw;
      double wdot = 0.0;
      for (int r = j + 1 + lane; r < d; r += 32) wdot = __fma_rn(__ldcg(vj + r), __ldcg(col + r), wdot);
      wdot = warp_sum(wdot);
      const double top = __ldcg(col + j);
      wdot += top;
      const double tw = tau * wdot;
      for (int r = j + 1 + lane; r < d; r += 32) __stcg(col + r, __fma_rn(-tw, __ldcg(vj + r), __ldcg(col + r)));
      const double rjc = top - tw;
      int recompute = 0;
      __syncwarp();
      if (lane == 0) {
        __stcg(col + j, rjc);
        double nc = __ldcg(nrm + c);
        if (nc != 0.0) {
          double t2 = fabs(rjc) / nc;
          t2 = fmax(0.0, (1.0 + t2) * (1.0 - t2));
          double ratio = nc / __ldcg(orig + c);
          if (t2 * ratio * ratio <= tol3z) recompute = 1;
          else __stcg(nrm + c, nc * sqrt(t2));
        }
      }
      recompute = __shfl_sync(0xffffffffu, recompute, 0);
      if (recompute) {
        __syncwarp();
        double s2 = 0.0;
        for (int r = j + 1 + lane; r < d; r += 32) {
          double v = __ldcg(col + r);
          s2 = __fma_rn(v, v, s2);
        }
        s2 = warp_sum(s2);
        if (lane == 0) { __stcg(nrm + c, sqrt(s2)); __stcg(orig + c, sqrt(s2)); }
      }
    }
    __syncthreads();   // the next pivot search reads norms down-dated by other warps
  }

  int accepted = 1;
  if (jb.rule == 1) accepted = stopped ? (k <= d - jb.p) : (k == m);
  if (jb.do_id && accepted && k > 0 && k < m) {
    // X = R1^{-1} R2 on own slots >= k (R1 was completed before the last barrier)
    int tk = (k > rank) ? (k - rank + P - 1) / P : 0;
    for (int t = tk + warp;; t += NW) {
      const int c = rank + P * t;
      if (c >= m) break;
      double* col = W + (long long)c * ldw;
      for (int i = k - 1; i >= 0; --i) {
        __syncwarp();
        double xi = __ldcg(col + i) / __ldcg(W + i + (long long)i * ldw);
        __syncwarp();
        if (lane == 0) __stcg(col + i, xi);
        for (int r = lane; r < i; r += 32)
          __stcg(col + r, __fma_rn(-__ldcg(W + r + (long long)i * ldw), xi, __ldcg(col + r)));
      }
    }
  }
  if (rank == 0 && tid == 0) { jb.out[0] = k; jb.out[1] = stopped; jb.out[2] = accepted; }
}

}  // namespace

cudaError_t launch_qrcp(const QrcpJob* jobs_dev, int njobs, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  k_qrcp<<<njobs, NT, 0, st>>>(jobs_dev);
  return cudaGetLastError();
}

int qrcp_group_capacity() {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_qrcp_group, NT, 0) != cudaSuccess) return 0;
  return sms * (per < 2 ? per : 2);
}

cudaError_t launch_qrcp_group(const QrcpJob* jobs_dev, const int2* map_dev, int nctas, int* err,
                              cudaStream_t st) {
  if (nctas <= 0) return cudaSuccess;
  void* args[] = {(void*)&jobs_dev, (void*)&map_dev, (void*)&err};
  return cudaLaunchCooperativeKernel((const void*)k_qrcp_group, dim3(nctas), dim3(NT), args, 0, st);
}

}  // namespace hss
