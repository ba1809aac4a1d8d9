// Batched interpolative decomposition by QR with column pivoting (eq. ID):
// for every job, W = S^T (d x m, the sample's rows as columns) is factored
// as W Pi = Q [R1 R2], truncated at the first pivot that fails the rank
// rule, and X = R1^{-1} R2 (= E^T) is formed by back substitution.
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
// One kernel serves two launch shapes: one CTA per job (many node sides on a
// level), or a group of P CTAs per job in one cooperative launch (upper
// levels with fewer node sides than SMs).  Column c of W is owned by CTA
// rank c mod P and never moves: a pivot column is "retired" (its norm set to
// -1) instead of being swapped, every CTA reads it where it lives and builds
// the same Householder reflector in shared memory, so a pivot step needs a
// single group barrier (after the partial argmaxes are published).  Row j
// of W then holds row j of R for every column; R1(i, i') = W(i, piv[i']) for
// i < i', R1(i, i) = diag[i]; the surviving columns keep R2 in place.
//
// Pivot = largest down-dated column norm (lowest index on ties), recomputed
// when cancellation has eaten half of the digits; the stop test uses the
// exact norm of the pivot column.  The group barrier is a monotonic counter
// per job with a bounded wait (about 2 s of %globaltimer, or as soon as
// another CTA has recorded an error); data written by one CTA and read by
// another goes through L2 (ld/st .cg).
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

// Group barrier of the P CTAs of a job (a plain __syncthreads when P == 1).
__device__ bool group_barrier(unsigned* bar, int P, unsigned& epoch, int* err, int* s_ok) {
  __syncthreads();
  if (P == 1) return true;
  if (threadIdx.x == 0) {
    epoch += 1;
    const unsigned target = epoch * (unsigned)P;
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

// block-wide sum; every thread gets the same value (fixed order)
__device__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x / 32] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < NW; ++w) t += sh[w];
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(NT) k_qrcp(const QrcpJob* __restrict__ jobs,
                                             const int2* __restrict__ map, int* err,
                                             size_t smem_bytes) {
  extern __shared__ double vs[];   // reflector of the current step (d), then W if it fits
  const int2 me = map ? map[blockIdx.x] : make_int2(blockIdx.x, 0);
  const QrcpJob jb = jobs[me.x];
  const int rank = me.y, P = map ? jb.P : 1;
  const int m = jb.m, d = jb.d, tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  // A job worked on by one CTA whose W fits in the dynamic shared memory of
  // the launch keeps W there (written back at the end); all other jobs work
  // on W in global memory (L2).
  const bool own = (P == 1);
  const bool in_smem = own && (size_t)(m + 1) * d * sizeof(double) <= smem_bytes;
  const long long ldw = in_smem ? d : jb.ldw;
  double* W = in_smem ? vs + d : jb.W;
  double* nrm = jb.nrm;          // own columns only; -1 once retired
  double* orig = jb.nrm + m;
  double* diag = jb.diag;
  __shared__ double sh[NW];
  __shared__ int si[NW];
  __shared__ int s_ok;
  unsigned epoch = 0;

  // W = S^T for the own columns, initial norms
  for (int c = rank + P * warp; c < m; c += P * NW) {
    const double* src = jb.S + (long long)c * jb.lds;
    double* dst = W + (long long)c * ldw;
    double s = 0.0;
    for (int r = lane; r < d; r += 32) {
      double v = src[r];
      dst[r] = v;
      s = __fma_rn(v, v, s);
    }
    s = warp_sum(s);
    if (lane == 0) { nrm[c] = s; orig[c] = s; }   // squared norms
  }
  __syncthreads();

  const int kmax = min(d, m);
  int k = kmax, stopped = 0;
  __shared__ double s_tau, s_scal, s_r11;
  __shared__ int s_stop;
  const double tol3z = 1.4901161193847656e-08;   // sqrt(2^-52)
  for (int j = 0; j < kmax; ++j) {
    // largest (squared) norm among the own live columns
    double bv = -1.0;
    int bi = 0x7fffffff;
    for (int c = rank + P * tid; c < m; c += P * NT) argmax_pair(bv, bi, nrm[c], c);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
      int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
      argmax_pair(bv, bi, v2, i2);
    }
    if (lane == 0) { sh[warp] = bv; si[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double v = sh[0];
      int i = si[0];
      for (int w = 1; w < NW; ++w) argmax_pair(v, i, sh[w], si[w]);
      if (P > 1) { __stcg(jb.redv + rank, v); __stcg(jb.redi + rank, i); }
      else { sh[0] = v; si[0] = i; }
    }
    if (!group_barrier(jb.bar, P, epoch, err, &s_ok)) return;
    // every CTA: the pivot, the exact pivot norm and the reflector
    if (P > 1 && warp == 0) {
      // the P partial maxima, read by the 32 lanes at once (the order of
      // the reduction does not matter: ties go to the lowest index)
      double v = -2.0;
      int i = 0x7fffffff;
      for (int q = lane; q < P; q += 32) argmax_pair(v, i, __ldcg(jb.redv + q), __ldcg(jb.redi + q));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        double v2 = __shfl_xor_sync(0xffffffffu, v, o);
        int i2 = __shfl_xor_sync(0xffffffffu, i, o);
        argmax_pair(v, i, v2, i2);
      }
      if (lane == 0) si[0] = i;
    }
    __syncthreads();
    const int p = si[0];
    const double* pc = W + (long long)p * ldw;
    double s = 0.0;
    for (int r = j + tid; r < d; r += NT) {
      const double v = own ? pc[r] : __ldcg(pc + r);
      vs[r] = v;
      s = __fma_rn(v, v, s);
    }
    const double ss = block_sum(s, sh);
    // the step's scalars once (thread 0), broadcast through shared memory:
    // on this part a replicated FP64 sqrt or divide costs more than a column
    if (tid == 0) {
      const double alpha = sqrt(ss);
      if (j == 0) s_r11 = alpha;
      double thr_a = jb.ea, thr_r = jb.er * s_r11;
      if (jb.rule == 1) {
        const double den = (double)(d - (j + 1) - 1);
        if (den <= 0.0) { thr_a = 0.0; thr_r = 0.0; }
        else {
          const double f = 1.0 + 4.0 * sqrt((double)d) / den * sqrt((double)min(jb.mh, jb.nh));
          thr_a /= f;
          thr_r /= f;
        }
      }
      s_stop = (alpha <= thr_a || alpha <= thr_r) ? 1 : 0;
      if (!s_stop) {
        const double x0 = vs[j];
        const double beta = x0 >= 0.0 ? -alpha : alpha;
        s_tau = (beta - x0) / beta;
        s_scal = 1.0 / (x0 - beta);
        if (p % P == rank) {
          nrm[p] = -1.0;               // retired
          __stcg(diag + j, beta);
          __stcg(jb.piv + j, p);
        }
      }
    }
    __syncthreads();
    if (s_stop) { k = j; stopped = 1; break; }
    const double tau = s_tau, scal = s_scal;
    for (int r = j + 1 + tid; r < d; r += NT) vs[r] *= scal;
    if (tid == 0) vs[j] = 1.0;
    __syncthreads();
    // reflector on the own live columns, two per warp at a time (eight
    // independent load streams per lane), then norm down-dating
    for (int c1 = rank + P * warp; c1 < m; c1 += 2 * P * NW) {
      const int c2 = c1 + P * NW;
      const bool l1 = nrm[c1] >= 0.0, l2 = c2 < m && nrm[c2] >= 0.0;
      if (!l1 && !l2) continue;
      const int ca = l1 ? c1 : c2;
      const int cb = (l1 && l2) ? c2 : ca;   // cb == ca: a single column
      double* colA = W + (long long)ca * ldw;
      double* colB = W + (long long)cb * ldw;
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0, b0 = 0.0, b1 = 0.0, b2 = 0.0, b3 = 0.0;
      int r = j + 1 + lane;
      for (; r + 96 < d; r += 128) {
        const double v0 = vs[r], v1 = vs[r + 32], v2 = vs[r + 64], v3 = vs[r + 96];
        a0 = __fma_rn(v0, colA[r], a0);
        a1 = __fma_rn(v1, colA[r + 32], a1);
        a2 = __fma_rn(v2, colA[r + 64], a2);
        a3 = __fma_rn(v3, colA[r + 96], a3);
        b0 = __fma_rn(v0, colB[r], b0);
        b1 = __fma_rn(v1, colB[r + 32], b1);
        b2 = __fma_rn(v2, colB[r + 64], b2);
        b3 = __fma_rn(v3, colB[r + 96], b3);
      }
      for (; r < d; r += 32) {
        const double v0 = vs[r];
        a0 = __fma_rn(v0, colA[r], a0);
        b0 = __fma_rn(v0, colB[r], b0);
      }
      const double topA = colA[j], topB = colB[j];
      const double twA = tau * (warp_sum((a0 + a1) + (a2 + a3)) + topA);
      const double twB = tau * (warp_sum((b0 + b1) + (b2 + b3)) + topB);
      const bool two = cb != ca;
      for (int r2 = j + 1 + lane; r2 < d; r2 += 32) {
        const double v = vs[r2];
        colA[r2] = __fma_rn(-twA, v, colA[r2]);
        if (two) colB[r2] = __fma_rn(-twB, v, colB[r2]);
      }
      __syncwarp();
      for (int q = 0; q < (two ? 2 : 1); ++q) {
        const int c = q ? cb : ca;
        double* col = q ? colB : colA;
        const double rjc = (q ? topB - twB : topA - twA);
        int recompute = 0;
        if (lane == 0) {
          col[j] = rjc;
          // squared-norm down-date; a result that lost most of its digits
          // to cancellation (below tol3z of the norm^2 at its last exact
          // computation) is recomputed from the column
          const double v = __fma_rn(-rjc, rjc, nrm[c]);
          if (v <= tol3z * orig[c]) recompute = 1;
          else nrm[c] = v;
        }
        recompute = __shfl_sync(0xffffffffu, recompute, 0);
        if (recompute) {
          __syncwarp();
          double s2 = 0.0;
          for (int r2 = j + 1 + lane; r2 < d; r2 += 32) s2 = __fma_rn(col[r2], col[r2], s2);
          s2 = warp_sum(s2);
          if (lane == 0) { nrm[c] = s2; orig[c] = s2; }
        }
      }
    }
    __syncthreads();
  }
  // every R entry and pivot of the group visible before the solve
  if (!group_barrier(jb.bar, P, epoch, err, &s_ok)) return;

  int accepted = 1;
  if (jb.rule == 1) accepted = stopped ? (k <= d - jb.p) : (k == m);
  // surviving columns after the k pivots, in column order (rank 0)
  if (rank == 0) {
    int base = k;
    for (int c0 = 0; c0 < m; c0 += NT) {
      const int c = c0 + tid;
      int live = 0;
      if (c < m) {
        const double nc = (c % P == 0) ? nrm[c] : __ldcg(nrm + c);
        live = nc >= 0.0;
        // columns that were never pivoted (a stop leaves its pivot live)
        if (live && stopped) live = 1;
      }
      // block exclusive scan of `live`
      const unsigned bal = __ballot_sync(0xffffffffu, live);
      const int wpre = __popc(bal & ((1u << lane) - 1u));
      if (lane == 0) si[warp] = __popc(bal);
      __syncthreads();
      int off = base;
      for (int w = 0; w < warp; ++w) off += si[w];
      int tot = 0;
      for (int w = 0; w < NW; ++w) tot += si[w];
      if (live) __stcg(jb.piv + off + wpre, c);
      __syncthreads();
      base += tot;
    }
  }
  if (jb.do_id && accepted && k > 0 && k < m) {
    // X = R1^{-1} R2 in place on the own surviving columns
    for (int c = rank + P * warp; c < m; c += P * NW) {
      if (nrm[c] < 0.0) continue;
      double* col = W + (long long)c * ldw;
      for (int i = k - 1; i >= 0; --i) {
        __syncwarp();
        const double xi = col[i] / __ldcg(diag + i);
        __syncwarp();
        if (lane == 0) col[i] = xi;
        const double* ri = W + (long long)__ldcg(jb.piv + i) * ldw;
        for (int r = lane; r < i; r += 32)
          col[r] = __fma_rn(-(own ? ri[r] : __ldcg(ri + r)), xi, col[r]);
      }
    }
    if (in_smem) {
      // X back to the global workspace: W(0:k, c) of the surviving columns
      __syncthreads();
      for (int c = warp; c < m; c += NW) {
        if (nrm[c] < 0.0) continue;
        for (int r = lane; r < k; r += 32) jb.W[r + (long long)c * jb.ldw] = W[r + (long long)c * ldw];
      }
    }
  }
  if (rank == 0 && tid == 0) { jb.out[0] = k; jb.out[1] = stopped; jb.out[2] = accepted; }
}

}  // namespace

int qrcp_group_capacity() {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaFuncSetAttribute(k_qrcp, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_qrcp, NT, 64 * 1024) != cudaSuccess) return 0;
  return sms * (per < 2 ? per : 2);
}

// map == nullptr: one CTA per job (ordinary launch); otherwise map[cta] =
// (job, rank) and the launch is cooperative.  d_max: largest d of the jobs;
// smem_w: dynamic shared memory to request so that single-CTA jobs with
// (m + 1) d doubles up to that size keep W in shared memory (0: none).
cudaError_t launch_qrcp(const QrcpJob* jobs_dev, const int2* map_dev, int nctas, int d_max, size_t smem_w,
                        int* err, cudaStream_t st) {
  if (nctas <= 0) return cudaSuccess;
  size_t sm = sizeof(double) * (size_t)(d_max > 0 ? d_max : 1);
  if (!map_dev && smem_w > sm) sm = smem_w;
  cudaError_t e = cudaFuncSetAttribute(k_qrcp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sm > 64 * 1024 ? sm : 64 * 1024));
  if (e != cudaSuccess) return e;
  if (!map_dev) {
    k_qrcp<<<nctas, NT, sm, st>>>(jobs_dev, nullptr, err, sm);
    return cudaGetLastError();
  }
  void* args[] = {(void*)&jobs_dev, (void*)&map_dev, (void*)&err, (void*)&sm};
  return cudaLaunchCooperativeKernel((const void*)k_qrcp, dim3(nctas), dim3(NT), args, sm, st);
}

}  // namespace hss
