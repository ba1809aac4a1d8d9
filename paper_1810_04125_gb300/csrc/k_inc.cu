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
// blocks of at most RB rows kept in shared memory), so that the Householder
// QR of a tall block and the formation of Q_k use P SMs.  The cost is the
// group barriers, so the kernel keeps them few:
//  - one group reduction per Householder column: with x the pivot column and
//    u = x - beta e_j, the dots u^T c = x^T c - beta c(j) of the trailing
//    columns need only x^T c and c(j), which every CTA sums over its rows in
//    the same sweep as |x|^2 = x^T x and x(j); the reflector and the updates
//    follow from the reduced sums in every CTA;
//  - Q_k by blocks of QB reflectors in compact-WY form (H_j0 .. H_j1-1 =
//    I - V T V^T, T from V^T V as in the forward recurrence of the block
//    reflector): one reduction of [V^T V, V^T E] per block (its P partials
//    added by slices over the group, then read back by all), E <- E -
//    V (T (V^T E)).
// The P partial sums of a value are added in rank order, so all CTAs hold
// identical scalars.  Same tests, same outputs as k_inc_qr.
constexpr int GR_BUDGET = 6144;   // doubles of V (and of E) per CTA: rows x b
constexpr int GR_BMAX = 1024;     // widest block of the group form (tau table)
constexpr int QB = 16;            // reflectors per block of the Q formation
constexpr int QW = 1024;          // doubles of the block products V^T E per CTA

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

// sum of the P partials base[q * stride], q = 0 .. P-1, added in rank order
// with the loads issued sixteen at a time (they come from L2)
__device__ __forceinline__ double sum_partials(const double* base, size_t stride, int P) {
  double w = 0.0;
  int q = 0;
  for (; q + 16 <= P; q += 16) {
    double t[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) t[u] = __ldcg(base + (size_t)(q + u) * stride);
#pragma unroll
    for (int u = 0; u < 16; ++u) w += t[u];
  }
  for (; q < P; ++q) w += __ldcg(base + (size_t)q * stride);
  return w;
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

// reflectors per block of the Q formation for a block of beff columns
__host__ __device__ __forceinline__ int q_block(int beff) {
  const int nb = beff > 0 ? QW / beff : QB;
  return nb < 1 ? 1 : (nb > QB ? QB : nb);
}

// The partial-sum area of a side (doubles): two parities of P slots of
// 2 b + 2 for the QR columns, P slots of nb (nb + b) for the Q blocks, and
// nb (nb + b) combined values.
__host__ __device__ __forceinline__ size_t part_qr_stride(int b) { return 2 * (size_t)b + 2; }
__host__ __device__ __forceinline__ size_t part_q_stride(int b) { return (size_t)q_block(b) * (q_block(b) + b); }

__global__ void __launch_bounds__(NT, 2) k_inc_group(const IncJob* __restrict__ jobs, const int2* __restrict__ map,
                                                  int* err) {
  extern __shared__ double gsm[];
  const int2 me = map[blockIdx.x];
  const IncJob jb = jobs[me.x];
  const int rank = me.y, P = jb.P;
  const int m = jb.m, b = jb.b, tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int RB = (m + P - 1) / P, r0 = min(m, rank * RB), nr = min(m, r0 + RB) - r0;
  const int bb = max(b, 1);
  double* V = gsm;                               // nr x b, column-major, ld RB
  double* E = gsm + (size_t)RB * bb;             // nr x beff, ld RB
  double* X = gsm + 2 * (size_t)RB * bb;         // QR: d, g, tw (3 b); Q: V^T E then Y (nb x beff)
  double* Gt = X + (3 * (size_t)bb > (size_t)QW ? 3 * (size_t)bb : (size_t)QW);   // Q: V^T V, then T (QB x QB)
  double* s_taus = Gt + 2 * QB * QB;             // tau of every column
  __shared__ double sh[NW];
  __shared__ double s_sc[4];   // alpha, beta, tau, scal of the current column
  __shared__ int s_ok;
  unsigned epoch = 0;
  const size_t S1 = part_qr_stride(b);
  auto slot = [&](int parity, int q) { return jb.part + ((size_t)parity * P + q) * S1; };
  double* qslots = jb.part + 2 * (size_t)P * S1;            // P x S2
  double* qcomb = qslots + (size_t)P * part_q_stride(b);    // S2
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
    for (int c = warp; c < b; c += NW) {
      double w = 0.0;
      for (int i = lane; i < nr; i += 32) { const double h = V[i + (size_t)c * RB]; w = __fma_rn(h, h, w); }
      w = warp_sum(w);
      if (lane == 0) __stcg(slot(parity, rank) + 2 + c, w);
    }
  }
  if (!gbar(jb.bar, P, epoch, err, &s_ok, jb.wait_ns)) return;
  double nS = sum_partials(slot(parity, 0), S1, P), nSh = sum_partials(slot(parity, 0) + 1, S1, P);
  double est = 0.0;
  if (jb.hmt) {   // column totals in rank order, then the largest
    double cm = 0.0;
    for (int c = tid; c < b; c += NT) cm = fmax(cm, sum_partials(slot(parity, 0) + 2 + c, S1, P));
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
  // Householder QR of the block, rows split over the group, one group
  // reduction per column: d_c = x^T c over rows >= j and g_c = c(j) for the
  // columns c >= j (c = j gives |x|^2 and x(j))
  const int p = min(m, b);
  double mn = 1.0 / 0.0, r11 = 0.0;
  double* dd = X;
  double* gg = X + bb;
  double* tw = X + 2 * (size_t)bb;
  for (int j = 0; j < p; ++j) {
    const int nc = b - j;
    const bool ownj = j >= r0 && j < r0 + nr;
    double* out = slot(parity, rank);
    for (int c = warp; c < nc; c += NW) {   // a warp per column
      const double* xc = V + (size_t)j * RB;
      const double* cc = V + (size_t)(j + c) * RB;
      double w = 0.0;
      for (int i = lane; i < nr; i += 32)
        if (r0 + i >= j) w = __fma_rn(xc[i], cc[i], w);
      w = warp_sum(w);
      if (lane == 0) {
        __stcg(out + c, w);
        __stcg(out + nc + c, ownj ? cc[j - r0] : 0.0);
      }
    }
    if (!gbar(jb.bar, P, epoch, err, &s_ok, jb.wait_ns)) return;
    for (int t = tid; t < 2 * nc; t += NT) {   // the P partials of a value, in rank order
      const double w = sum_partials(slot(parity, 0) + t, S1, P);
      if (t < nc) dd[t] = w;
      else gg[t - nc] = w;
    }
    parity ^= 1;
    __syncthreads();
    if (tid == 0) {
      const double alpha = sqrt(dd[0]), x0 = gg[0];
      double beta = 0.0, tau = 0.0, scal = 0.0;
      if (alpha != 0.0) {
        beta = x0 >= 0.0 ? -alpha : alpha;
        tau = (beta - x0) / beta;
        scal = 1.0 / (x0 - beta);
      }
      s_sc[0] = alpha; s_sc[1] = beta; s_sc[2] = tau; s_sc[3] = scal;
      s_taus[j] = tau;
    }
    __syncthreads();
    const double alpha = s_sc[0], beta = s_sc[1], tau = s_sc[2], scal = s_sc[3];
    mn = fmin(mn, alpha);
    if (j == 0) r11 = alpha;
    if (lead) jb.tau[j] = tau;
    // tau v^T c = tau scal (d_c - beta g_c) for the trailing columns
    for (int c = 1 + tid; c < nc; c += NT) tw[c] = tau * (scal * (dd[c] - beta * gg[c]));
    __syncthreads();
    if (tau != 0.0) {
      double* xj = V + (size_t)j * RB;
      // trailing columns: c(r) -= tw_c v(r), v(j) = 1, v(r) = scal x(r) below
      for (int e = tid; e < nr * (nc - 1); e += NT) {
        const int i = e % nr, c = 1 + e / nr, r = r0 + i;
        if (r >= j) {
          const double v = r == j ? 1.0 : scal * xj[i];
          double& x = V[i + (size_t)(j + c) * RB];
          x = __fma_rn(-tw[c], v, x);
        }
      }
      __syncthreads();
      for (int i = tid; i < nr; i += NT) {
        const int r = r0 + i;
        if (r > j) xj[i] *= scal;
        else if (r == j) xj[i] = beta;
      }
    }
    __syncthreads();
  }
  const double rho = jb.rho < 0.0 ? r11 : jb.rho;
  if (lead) { if (!jb.hmt) jb.res[2] = mn; jb.res[3] = r11; }
  if (!jb.hmt && (mn < jb.ea || mn < jb.er * rho)) {
    if (lead) { jb.flag[0] = 1; jb.flag[1] = jb.q; }
    return;
  }
  // Q_k = H_0 ... H_{p-1} [I; 0], first beff columns, by blocks of nb
  // reflectors from the last: E <- (I - V_b T_b V_b^T) E
  const int beff = min(b, m - jb.q);
  const int pq = min(p, beff), nbq = q_block(b);
  const size_t S2 = part_q_stride(b);
  for (int e = tid; e < nr * beff; e += NT) {
    const int i = e % nr, c = e / nr;
    E[i + (size_t)c * RB] = (r0 + i == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  // v_j(r) from V: 0 above row j, 1 at row j, the stored entry below
  auto vref = [&](int i, int jj) -> double {
    const int r = r0 + i;
    return r < jj ? 0.0 : (r == jj ? 1.0 : V[i + (size_t)jj * RB]);
  };
  for (int j1 = pq; j1 > 0;) {
    // block [j0, j1): the columns c < j0 of E and its rows r < j0 are e_c
    // and zero under these reflectors and stay so; the values are
    // [V_b^T V_b (nb x nb), V_b^T E(:, j0:beff) (nb x nw)], one thread each
    // over the own rows
    const int j0 = max(0, j1 - nbq), nb = j1 - j0, nw = beff - j0;
    const int nv = nb * nb + nb * nw;
    const int i0 = max(0, j0 - r0);   // first own row at or below j0
    double* out = qslots + (size_t)rank * S2;
    for (int t = tid; t < nv; t += NT) {
      double w = 0.0;
      if (t < nb * nb) {
        const int a = t / nb, k = t % nb;
        if (a < k)
          for (int i = max(i0, j0 + k - r0); i < nr; ++i) w = __fma_rn(vref(i, j0 + a), vref(i, j0 + k), w);
      } else {
        const int a = (t - nb * nb) / nw, c = j0 + (t - nb * nb) % nw;
        const double* ec = E + (size_t)c * RB;
        for (int i = max(i0, j0 + a - r0); i < nr; ++i) w = __fma_rn(vref(i, j0 + a), ec[i], w);
      }
      __stcg(out + t, w);
    }
    if (!gbar(jb.bar, P, epoch, err, &s_ok, jb.wait_ns)) return;
    {   // this CTA's slice of the values, each the P partials in rank order
      const int v0 = (int)(((long long)nv * rank) / P), v1 = (int)(((long long)nv * (rank + 1)) / P);
      for (int t = v0 + tid; t < v1; t += NT) __stcg(qcomb + t, sum_partials(qslots + t, S2, P));
    }
    if (!gbar(jb.bar, P, epoch, err, &s_ok, jb.wait_ns)) return;
    for (int t = tid; t < nv; t += NT) {
      const double w = __ldcg(qcomb + t);
      if (t < nb * nb) Gt[t] = w;   // Gt[a nb + k] = v_a^T v_k (a < k)
      else X[t - nb * nb] = w;      // X[a nw + c - j0] = v_a^T E(:, c)
    }
    __syncthreads();
    // T_b (upper triangular): T(a, a) = tau_a, T(0:k, k) = -tau_k T(0:k, 0:k)
    // (V^T v_k)(0:k); one warp, column k after column k - 1
    if (warp == 0) {
      double* Tm = Gt + nb * nb;   // nb x nb, row-major
      for (int k = 0; k < nb; ++k) {
        const double tk = s_taus[j0 + k];
        for (int a = lane; a < nb; a += 32) {
          double t = 0.0;
          if (a < k) {
            for (int l = a; l < k; ++l) t = __fma_rn(Tm[a * nb + l], Gt[l * nb + k], t);
            t = -tk * t;
          } else if (a == k) {
            t = tk;
          }
          Tm[a * nb + k] = t;
        }
        __syncwarp();
      }
    }
    __syncthreads();
    // Y = T (V^T E) in place, one thread per column
    {
      const double* Tm = Gt + nb * nb;
      for (int c = tid; c < nw; c += NT) {
        double y[QB];
#pragma unroll
        for (int a = 0; a < QB; ++a) y[a] = a < nb ? X[a * nw + c] : 0.0;
#pragma unroll
        for (int a = 0; a < QB; ++a) {
          if (a >= nb) break;
          double t = 0.0;
#pragma unroll
          for (int k = 0; k < QB; ++k)
            if (k >= a && k < nb) t = __fma_rn(Tm[a * nb + k], y[k], t);
          X[a * nw + c] = t;
        }
      }
    }
    __syncthreads();
    // E(:, j0:beff) -= V_b Y over the own rows at or below j0
    for (int e = tid; e < (nr - i0) * nw; e += NT) {
      const int i = i0 + e % (nr - i0), c = e / (nr - i0);
      double x = E[i + (size_t)(j0 + c) * RB];
      for (int a = 0; a < nb; ++a) x = __fma_rn(-vref(i, j0 + a), X[a * nw + c], x);
      E[i + (size_t)(j0 + c) * RB] = x;
    }
    __syncthreads();
    j1 = j0;
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
  // V and E: rows(b) * b <= max(budget, 8 b) for every block width b <= b_max
  const size_t vb = b * 8 > (size_t)GR_BUDGET ? b * 8 : (size_t)GR_BUDGET;
  const size_t x = 3 * b > (size_t)QW ? 3 * b : (size_t)QW;
  return sizeof(double) * (vb * 2 + x + 2 * QB * QB + b);
}

}  // namespace

int inc_group_bmax() { return GR_BMAX; }

int inc_group_rows(int b) {
  const int bb = b > 0 ? b : 1;
  return GR_BUDGET / bb > 8 ? GR_BUDGET / bb : 8;
}

size_t inc_group_part(int P, int b) {
  return 2 * (size_t)P * part_qr_stride(b) + ((size_t)P + 1) * part_q_stride(b);
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
