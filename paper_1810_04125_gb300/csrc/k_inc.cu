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
//
// With the HMT criterion (Lemma 4.1, eq. HMT_IQQH) the only test is
//   alpha sqrt(2/pi) max_i |Sh(:, i)|_2 <= eps_a
// (hmt_c = alpha sqrt(2/pi)); on failure the block's Q_k joins Q as above,
// with no test on diag R_k.
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

__device__ double block_max(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x / 32] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < NW; ++w) t = fmax(t, sh[w]);
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
  if (jb.hmt) {
    // the largest squared column norm of Sh, a warp per column
    double cm = 0.0;
    for (int c = warp; c < b; c += NW) {
      const double* col = A + (long long)c * m;
      double w = 0.0;
      for (int r = lane; r < m; r += 32) w = __fma_rn(col[r], col[r], w);
      cm = fmax(cm, warp_sum(w));
    }
    const double est = jb.hmt_c * sqrt(block_max(cm, sh));
    if (tid == 0) jb.res[2] = est;
    if (b == 0 || est <= jb.ea) {
      if (tid == 0) { jb.flag[0] = 1; jb.flag[1] = jb.q; }
      return;
    }
  } else if (b == 0 || nS == 0.0 || nSh < jb.er * nS || nSh / sqrt((double)b) < jb.ea) {
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
  if (tid == 0) { if (!jb.hmt) jb.res[2] = mn; jb.res[3] = r11; }
  if (!jb.hmt && (mn < jb.ea || mn < jb.er * rho)) {
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

// ---------------------------------------------------------------------------
// Group form: the m rows of a side are split over P CTAs (contiguous row
// blocks kept in shared memory), so that the Householder QR of a tall block
// and the formation of Q_k use P SMs.  Every column step needs two group
// reductions (the norm of the pivot column with its top entry, then the
// dots with the trailing columns); the P partial sums are added in rank
// order by every CTA, so all CTAs hold identical scalars.  Same tests, same
// outputs as k_inc_qr.
constexpr int GR_BUDGET = 6144;   // doubles of V (and of E) per CTA: rows x b
constexpr int GR_BMAX = 1024;     // widest block of the group form (tau table)

__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acq(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// bounded group barrier (wait_ns of %globaltimer, about 2 s by default, or
// as soon as another CTA recorded an error); false when it gave up
__device__ bool gbar(unsigned* bar, int P, unsigned& epoch, int* err, int* s_ok, unsigned long long wait_ns) {
  __syncthreads();
  if (P == 1) return true;
  if (threadIdx.x == 0) {
    epoch += 1;
    const unsigned target = epoch * (unsigned)P;
    __threadfence();
    atomicAdd(bar, 1u);
    int ok = 1;
    const uint64_t t0 = gtime();
    for (unsigned it = 1; ld_acq(bar) < target; ++it) {
      if ((it & 63u) == 0 || it == 1) {   // the first spin too: a short limit is seen at once
        if (*(volatile int*)err) { ok = 0; break; }
        if (gtime() - t0 > wait_ns) { atomicCAS(err, 0, 7); ok = 0; break; }
      }
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

__device__ double bsum(double v, double* sh) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x / 32] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < NW; ++w) t += sh[w];
  return t;
}

__global__ void __launch_bounds__(NT, 2) k_inc_group(const IncJob* __restrict__ jobs, const int2* __restrict__ map,
                                                  int* err) {
  extern __shared__ double gsm[];
  const int2 me = map[blockIdx.x];
  const IncJob jb = jobs[me.x];
  const int rank = me.y, P = jb.P;
  const int m = jb.m, b = jb.b, tid = threadIdx.x;
  const int RB = (m + P - 1) / P, r0 = min(m, rank * RB), nr = min(m, r0 + RB) - r0;
  double* V = gsm;                        // nr x b, column-major, ld RB
  double* E = gsm + (size_t)RB * max(b, 1);   // nr x beff
  __shared__ double sh[NW];
  __shared__ double s_sc[4];   // alpha, beta, tau, scal of the current column
  __shared__ double s_taus[GR_BMAX];
  __shared__ int s_ok;
  unsigned epoch = 0;
  const int stride = b + 2;
  auto slot = [&](int parity, int q) { return jb.part + ((size_t)parity * P + q) * stride; };
  int parity = 0;

  for (int e = tid; e < nr * b; e += NT) {
    const int i = e % nr, c = e / nr;
    V[i + (size_t)c * RB] = jb.Sh[(r0 + i) + (size_t)c * m];
  }
  // norms of S_k and of the projected block
  double s1 = 0.0, s2 = 0.0;
  for (int e = tid; e < nr * b; e += NT) {
    const int i = e % nr, c = e / nr;
    const double a = jb.S[(long long)(r0 + i) * jb.lds + jb.c0 + c];
    s1 = __fma_rn(a, a, s1);
    const double h = V[i + (size_t)c * RB];
    s2 = __fma_rn(h, h, s2);
  }
  s1 = bsum(s1, sh);
  s2 = bsum(s2, sh);
  if (tid == 0) { __stcg(slot(parity, rank), s1); __stcg(slot(parity, rank) + 1, s2); }
  if (jb.hmt) {   // partial squared column norms of the projected block
    for (int c = tid / 32; c < b; c += NW) {
      double w = 0.0;
      for (int i = tid % 32; i < nr; i += 32) { const double h = V[i + (size_t)c * RB]; w = __fma_rn(h, h, w); }
      w = warp_sum(w);
      if ((tid & 31) == 0) __stcg(slot(parity, rank) + 2 + c, w);
    }
  }
  if (!gbar(jb.bar, P, epoch, err, &s_ok, jb.wait_ns)) return;
  double nS = 0.0, nSh = 0.0;
  for (int q = 0; q < P; ++q) { nS += __ldcg(slot(parity, q)); nSh += __ldcg(slot(parity, q) + 1); }
  double est = 0.0;
  if (jb.hmt) {   // column totals in rank order, then the largest
    double cm = 0.0;
    for (int c = tid; c < b; c += NT) {
      double w = 0.0;
      for (int q = 0; q < P; ++q) w += __ldcg(slot(parity, q) + 2 + c);
      cm = fmax(cm, w);
    }
    est = jb.hmt_c * sqrt(block_max(cm, sh));
  }
  parity ^= 1;
  nS = sqrt(nS);
  nSh = sqrt(nSh);
  const bool lead = rank == 0 && tid == 0;
  if (lead) { jb.res[0] = nS; jb.res[1] = nSh; jb.res[2] = jb.hmt ? est : -1.0; jb.res[3] = -1.0; }
  if (jb.hmt ? (b == 0 || est <= jb.ea)
             : (b == 0 || nS == 0.0 || nSh < jb.er * nS || nSh / sqrt((double)b) < jb.ea)) {
    if (lead) { jb.flag[0] = 1; jb.flag[1] = jb.q; }
    return;
  }
  // Householder QR of the block, rows split over the group
  const int p = min(m, b);
  double mn = 1.0 / 0.0, r11 = 0.0;
  for (int j = 0; j < p; ++j) {
    double s = 0.0;
    for (int i = tid; i < nr; i += NT)
      if (r0 + i >= j) { const double a = V[i + (size_t)j * RB]; s = __fma_rn(a, a, s); }
    s = bsum(s, sh);
    if (tid == 0) {
      __stcg(slot(parity, rank), s);
      __stcg(slot(parity, rank) + 1, (j >= r0 && j < r0 + nr) ? V[(j - r0) + (size_t)j * RB] : 0.0);
    }
    if (!gbar(jb.bar, P, epoch, err, &s_ok, jb.wait_ns)) return;
    if (tid == 0) {
      double ss = 0.0, x0 = 0.0;
      for (int q = 0; q < P; ++q) { ss += __ldcg(slot(parity, q)); x0 += __ldcg(slot(parity, q) + 1); }
      const double alpha = sqrt(ss);
      double beta = 0.0, tau = 0.0, scal = 0.0;
      if (alpha != 0.0) {
        beta = x0 >= 0.0 ? -alpha : alpha;
        tau = (beta - x0) / beta;
        scal = 1.0 / (x0 - beta);
      }
      s_sc[0] = alpha; s_sc[1] = beta; s_sc[2] = tau; s_sc[3] = scal;
      s_taus[j] = tau;
    }
    parity ^= 1;
    __syncthreads();
    const double alpha = s_sc[0], beta = s_sc[1], tau = s_sc[2], scal = s_sc[3];
    mn = fmin(mn, alpha);
    if (j == 0) r11 = alpha;
    if (lead) jb.tau[j] = tau;
    if (tau != 0.0) {
      for (int i = tid; i < nr; i += NT)
        if (r0 + i > j) V[i + (size_t)j * RB] *= scal;
    }
    __syncthreads();
    if (j >= r0 && j < r0 + nr && tid == 0) V[(j - r0) + (size_t)j * RB] = beta;
    if (tau != 0.0 && j + 1 < b) {
      // dots of v_j (v_j(j) = 1) with the trailing columns, over rows >= j
      const int nc = b - j - 1;
      for (int c = tid / 32; c < nc; c += NW) {   // a warp per column
        double w = 0.0;
        for (int i = tid % 32; i < nr; i += 32) {
          const int r = r0 + i;
          if (r >= j) w = __fma_rn(r == j ? 1.0 : V[i + (size_t)j * RB], V[i + (size_t)(j + 1 + c) * RB], w);
        }
        w = warp_sum(w);
        if ((tid & 31) == 0) __stcg(slot(parity, rank) + c, w);
      }
      if (!gbar(jb.bar, P, epoch, err, &s_ok, jb.wait_ns)) return;
      for (int c = tid; c < nc; c += NT) {
        double w = 0.0;
        for (int q = 0; q < P; ++q) w += __ldcg(slot(parity, q) + c);
        gsm[(size_t)RB * max(b, 1) * 2 + c] = tau * w;   // tw(c), after E
      }
      parity ^= 1;
      __syncthreads();
      const double* tw = gsm + (size_t)RB * max(b, 1) * 2;
      for (int e = tid; e < nr * nc; e += NT) {
        const int i = e % nr, c = e / nr, r = r0 + i;
        if (r >= j) {
          const double v = r == j ? 1.0 : V[i + (size_t)j * RB];
          double& x = V[i + (size_t)(j + 1 + c) * RB];
          x = __fma_rn(-tw[c], v, x);
        }
      }
      __syncthreads();
    }
  }
  const double rho = jb.rho < 0.0 ? r11 : jb.rho;
  if (lead) { if (!jb.hmt) jb.res[2] = mn; jb.res[3] = r11; }
  if (!jb.hmt && (mn < jb.ea || mn < jb.er * rho)) {
    if (lead) { jb.flag[0] = 1; jb.flag[1] = jb.q; }
    return;
  }
  // Q_k = H_0 ... H_{p-1} [I; 0], first beff columns
  const int beff = min(b, m - jb.q);
  for (int e = tid; e < nr * beff; e += NT) {
    const int i = e % nr, c = e / nr;
    E[i + (size_t)c * RB] = (r0 + i == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = min(p, beff) - 1; j >= 0; --j) {
    const double tau = s_taus[j];
    if (tau == 0.0) continue;
    const int nc = beff - j;
    for (int c = tid / 32; c < nc; c += NW) {   // a warp per column
      double w = 0.0;
      for (int i = tid % 32; i < nr; i += 32) {
        const int r = r0 + i;
        if (r >= j) w = __fma_rn(r == j ? 1.0 : V[i + (size_t)j * RB], E[i + (size_t)(j + c) * RB], w);
      }
      w = warp_sum(w);
      if ((tid & 31) == 0) __stcg(slot(parity, rank) + c, w);
    }
    if (!gbar(jb.bar, P, epoch, err, &s_ok, jb.wait_ns)) return;
    for (int c = tid; c < nc; c += NT) {
      double w = 0.0;
      for (int q = 0; q < P; ++q) w += __ldcg(slot(parity, q) + c);
      gsm[(size_t)RB * max(b, 1) * 2 + c] = tau * w;
    }
    parity ^= 1;
    __syncthreads();
    const double* tw = gsm + (size_t)RB * max(b, 1) * 2;
    for (int e = tid; e < nr * nc; e += NT) {
      const int i = e % nr, c = e / nr, r = r0 + i;
      if (r >= j) {
        const double v = r == j ? 1.0 : V[i + (size_t)j * RB];
        double& x = E[i + (size_t)(j + c) * RB];
        x = __fma_rn(-tw[c], v, x);
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < nr * beff; e += NT) {
    const int i = e / beff, c = e % beff;
    jb.Q[(long long)(r0 + i) * jb.lds + jb.q + c] = E[i + (size_t)c * RB];
  }
  if (lead) {
    jb.flag[1] = jb.q + beff;
    jb.flag[0] = (jb.q + beff >= m) ? 1 : 0;
  }
}

size_t inc_group_smem(int b_max) {
  const size_t b = b_max > 0 ? b_max : 1;
  // rows(b) * b <= max(budget, 8 b) for every block width b <= b_max
  const size_t vb = b * 8 > (size_t)GR_BUDGET ? b * 8 : (size_t)GR_BUDGET;
  return sizeof(double) * (vb * 2 + b + 2);
}

}  // namespace

int inc_group_bmax() { return GR_BMAX; }

int inc_group_rows(int b) {
  const int bb = b > 0 ? b : 1;
  return GR_BUDGET / bb > 8 ? GR_BUDGET / bb : 8;
}

int inc_group_capacity(int b_max) {
  int dev = 0, sms = 0, per = 0;
  const size_t sm = inc_group_smem(b_max);
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaFuncSetAttribute(k_inc_group, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_inc_group, NT, sm) != cudaSuccess) return 0;
  return sms * per;
}

cudaError_t launch_inc_group(const IncJob* jobs_dev, const int2* map_dev, int nctas, int b_max, int* err,
                             cudaStream_t st) {
  if (nctas <= 0) return cudaSuccess;
  const size_t sm = inc_group_smem(b_max);
  cudaError_t e = cudaFuncSetAttribute(k_inc_group, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&jobs_dev, (void*)&map_dev, (void*)&err};
  return cudaLaunchCooperativeKernel((const void*)k_inc_group, dim3(nctas), dim3(NT), args, sm, st);
}

cudaError_t launch_inc_qr(const IncJob* jobs_dev, int njobs, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  k_inc_qr<<<njobs, NT, 0, st>>>(jobs_dev);
  return cudaGetLastError();
}

}  // namespace hss
