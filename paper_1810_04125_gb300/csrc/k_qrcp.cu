// Batched interpolative decomposition by QR with column pivoting (eq. ID):
// for every job, W = S^T (d x m, the sample's rows as columns) is factored
// as W Pi = Q [R1 R2], truncated at the first pivot that fails the rank
// rule, and X = R1^{-1} R2 (= E^T) is formed by blocked back substitution.
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
// Work split.  A job is worked on by a group of P CTAs (P = 1 for small
// jobs; all groups of a launch are co-resident, cooperative launch when
// P > 1).  Column c of W (contiguous, leading dimension ldw) is owned by
// CTA rank c mod P and never moves: a pivot column is retired from its
// owner's list of live columns instead of being swapped; every CTA reads it
// where it lives and builds the same Householder reflector in shared
// memory.  Row j of W then holds row j of R for every column; R1(i, i') =
// W(i, piv[i']) for i < i', R1(i, i) = diag[i]; the surviving columns keep
// R2 in place.
//
// One pass over the trailing matrix per pivot step.  Applying reflector
// H_{j-1} to a column and forming the dot product with the next reflector
// v_j are fused: the pass of step j reads W(r, c) (r >= j), subtracts
// tw_{j-1}(c) v_{j-1}(r), stores it and accumulates v_j(r) times it (both
// reflectors kept unscaled, their scale folded into the coefficients).  Row
// j-1 and the norm down-date only need tw_{j-1}(c) and the old W(j-1, c),
// so the next pivot is known before the pass; the pivot column is brought
// up to date on the fly when it is read.  Inside a CTA eight lanes share a
// live column (a quad of 4 rows each, 16-byte loads) and the warps split
// the rows; the partial dot products meet in shared memory.
//
// Placement.  The CTAs of a group run their pivot steps in lockstep, so two
// of them on one SM are idle in the serial part of a step at the same time
// and the SM's FP64 pipe with them; the block scheduler is free to put
// consecutive blocks on one SM.  A cooperative launch therefore fills every
// co-resident slot and each CTA takes its (job, rank) by the SM it runs on:
// position slot x nsm + (index of its SM), where the host lays the ranks of
// a group out at consecutive positions, i.e. on different SMs, and every SM
// hosts CTAs of several groups whose serial parts need not coincide.
//
// Pivot = largest down-dated squared column norm (lowest index on ties),
// recomputed from the column when cancellation has left less than
// sqrt(eps) of its last exact value; the stop test uses the exact norm of
// the pivot column.  The group barrier is a monotonic counter per job with a
// bounded wait (about 2 s of %globaltimer, or as soon as another CTA has
// recorded an error); data written by one CTA and read by another goes
// through L2 (ld/st .cg).
#include "hss_internal.h"

namespace hss {
namespace {

// Three launch shapes: 128 threads and four CTAs per SM (more co-resident
// groups, so that one group's serial phases overlap others' passes), 256
// threads and two, 512 threads and one (no other group's CTA competing for
// the SM's FP64 pipe).  The registers are budgeted for 512 threads per SM
// in every shape.
constexpr int NT_XWIDE = 512, NT_WIDE = 256, NT_NARROW = 128;
constexpr int NLMAX = 256;   // own columns per CTA (host sizes the groups)
constexpr int PCU = 8;       // loads in flight per thread when the pivot column is read
constexpr int EB = 16;       // rows per block of the back substitution X = R1^{-1} R2

// sum of N partials spaced NLMAX apart, as a balanced tree (fixed order)
template <int N>
__device__ __forceinline__ double tree_sum(const double* p) {
  if constexpr (N == 1) return p[0];
  else return tree_sum<N / 2>(p) + tree_sum<N - N / 2>(p + (N / 2) * NLMAX);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// (k, i) <- the larger key (a non-negative norm's bit pattern), lowest
// column index on ties
__device__ __forceinline__ void key_max(unsigned long long& k, int& i, int& pos, unsigned long long k2, int i2,
                                        int pos2) {
  if (k2 > k || (k2 == k && i2 < i)) { k = k2; i = i2; pos = pos2; }
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
__device__ bool group_barrier(unsigned* bar, int P, unsigned& epoch, int* err, int* s_ok,
                              unsigned long long wait_ns) {
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
      if ((it & 63u) == 0 || it == 1) {   // the first spin too: a short limit is seen at once
        if (*(volatile int*)err) { ok = 0; break; }
        if (gtimer() - t0 > wait_ns) { atomicCAS(err, 0, 6); ok = 0; break; }
      }
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// block-wide sum; every thread gets the same value (fixed order)
template <int NW>
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

// Stop thresholds of pivot step j (0-based): eps_a and eps_r |R_11|, both
// divided by the HMT factor f(j + 1) under rule 1 (zero when f is infinite).
__device__ __forceinline__ void rank_thresholds(const QrcpJob& jb, int d, int j, double r11, double& ta,
                                                double& tr) {
  ta = jb.ea;
  tr = jb.er * r11;
  if (jb.rule == 1) {
    const double den = (double)(d - (j + 1) - 1);
    if (den <= 0.0) { ta = 0.0; tr = 0.0; }
    else {
      const double f = 1.0 + 4.0 * sqrt((double)d) / den * sqrt((double)min(jb.mh, jb.nh));
      ta /= f;
      tr /= f;
    }
  }
}

// shared-memory carve-up (dynamic part): two reflectors of d_max entries,
// then per own live column: partial dots of the warps, tw, top, norm^2,
// norm^2 at the last exact computation, column index, position in the
// group's live list
struct Carve {
  double *v0, *v1, *part, *tw, *top, *nrm, *orig;
  int* lc;
  int* rc;   // columns whose norm is recomputed this step
  int* gp;
};

template <int NW>
__device__ __forceinline__ Carve carve(double* base, int dmax) {
  const int dp = (dmax + 3) & ~3;   // 32-byte aligned reflectors, whole quads
  Carve c;
  c.v0 = base;
  c.v1 = c.v0 + dp;
  c.part = c.v1 + dp;
  c.tw = c.part + NW * NLMAX;
  c.top = c.tw + NLMAX;
  c.nrm = c.top + NLMAX;
  c.orig = c.nrm + NLMAX;
  c.lc = (int*)(c.orig + NLMAX);
  c.rc = c.lc + NLMAX;
  c.gp = c.rc + NLMAX;
  return c;
}

// The position of this CTA in a launch that fills every co-resident slot:
// slot x nsm + the index of its SM among the SMs present, when every SM
// present holds exactly per CTAs of the launch (else blockIdx.x).  place:
// per-SM counters [0, 1024), the bitmap of SMs present [1024, 1056), the
// launch barrier and a flag for an SM id out of range.  Called by every
// thread; false when the launch barrier gave up.
__device__ bool placed_position(unsigned* place, int nsm, int per, int* err, unsigned long long wait_ns, int* pos_out) {
  __shared__ unsigned s_smid, s_slot;
  __shared__ int s_pos, s_ok0;
  unsigned* cnt = place;
  unsigned* bits = place + 1024;
  unsigned* bar = place + 1056;
  unsigned* bad = place + 1057;
  if (threadIdx.x == 0) {
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    s_smid = smid;
    if (smid < 1024u) {
      s_slot = atomicAdd(cnt + smid, 1u);
      atomicOr(bits + (smid >> 5), 1u << (smid & 31u));
    } else {
      s_slot = 0u;
      atomicOr(bad, 1u);
    }
  }
  unsigned ep = 0;
  if (!group_barrier(bar, (int)gridDim.x, ep, err, &s_ok0, wait_ns)) return false;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const unsigned w = __ldcg(bits + lane);
    const unsigned me = s_smid;
    // SMs present, those below this one, and whether each holds per CTAs
    int total = __popc(w), below = 0, even = 1;
    if (me < 1024u) {
      const unsigned mw = me >> 5;
      if ((unsigned)lane < mw) below = __popc(w);
      else if ((unsigned)lane == mw) below = __popc(w & ((1u << (me & 31u)) - 1u));
    }
    for (unsigned r = w; r; r &= r - 1) {
      const int b = __ffs(r) - 1;
      if (__ldcg(cnt + 32 * lane + b) != (unsigned)per) even = 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      total += __shfl_xor_sync(0xffffffffu, total, o);
      below += __shfl_xor_sync(0xffffffffu, below, o);
    }
    even = __all_sync(0xffffffffu, even);
    if (lane == 0) {
      const bool ok = even && total == nsm && __ldcg(bad) == 0u && s_slot < (unsigned)per;
      s_pos = ok ? (int)s_slot * nsm + below : (int)blockIdx.x;
    }
  }
  __syncthreads();
  *pos_out = s_pos;
  return true;
}

template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT) k_qrcp(const QrcpJob* __restrict__ jobs,
                                                   const int2* __restrict__ map, int* err, int dmax,
                                                   unsigned* place, int nsm, int per) {
  constexpr int NW = NT / 32;
  extern __shared__ __align__(16) double smem_d[];
  int pos = (int)blockIdx.x;
  if (map && place && !placed_position(place, nsm, per, err, jobs[0].wait_ns, &pos)) return;
  const int2 me = map ? map[pos] : make_int2(blockIdx.x, 0);
  if (me.x < 0) return;   // an idle slot
  const QrcpJob jb = jobs[me.x];
  const int rank = me.y, P = map ? jb.P : 1;
  const int m = jb.m, d = jb.d, tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const long long ldw = jb.ldw;
  double* W = jb.W;
  double* diag = jb.diag;
  double* liveg = jb.nrm;   // global: +1 live, -1 retired (read by rank 0 at the end)
  Carve S = carve<NW>(smem_d, dmax);
  double* vp = S.v0;        // v_{j-1}
  double* vc = S.v1;        // v_j
  __shared__ double sh[NW];
  __shared__ unsigned long long shk[NW];
  __shared__ int shi[NW], shp[NW];
  __shared__ int s_ok, s_p, s_pos, s_stop, s_nl, s_nrc, s_tl;
  __shared__ double s_xf[4];   // the column moved to the pivot's owner: id, tw, norm^2, orig
  __shared__ double s_twp, s_tau, s_scal, s_r11, s_uj;
  __shared__ double s_th[2][2];   // stop thresholds (eps_a, eps_r |R_11|) by step parity
  unsigned epoch = 0;

  // own columns, W = S^T for them, initial squared norms
  int nl = 0;
  if (rank < m) nl = (m - 1 - rank) / P + 1;
  if (nl > NLMAX || d > dmax) {   // sized by the host; never expected
    if (tid == 0) atomicCAS(err, 0, 9);
    return;
  }
  for (int t = tid; t < nl; t += NT) S.lc[t] = S.gp[t] = rank + P * t;
  for (int r = tid; r < 2 * ((dmax + 3) & ~3); r += NT) S.v0[r] = 0.0;
  __syncthreads();
  for (int t = warp; t < nl; t += NW) {
    const int c = S.lc[t];
    const double* src = jb.S + (long long)c * jb.lds;
    double* dst = W + (long long)c * ldw;
    double s = 0.0;
    for (int r = lane; r < d; r += 32) {
      const double v = src[r];
      dst[r] = v;
      s = __fma_rn(v, v, s);
    }
    s = warp_sum(s);
    if (lane == 0) {
      S.nrm[t] = s;
      S.orig[t] = s;
      S.tw[t] = 0.0;
      liveg[c] = 1.0;
    }
  }
  __syncthreads();

  const int kmax = min(d, m);
  int k = kmax, stopped = 0;
  if (tid == 0) s_nrc = 0;
  __syncthreads();
  const double tol3z = 1.4901161193847656e-08;   // sqrt(2^-52)
  // the reflector of step j is kept unscaled, u_j = x - beta e_j (rows >= j,
  // x the pivot column), H_j = I - tau_j v v^T with v = scal_j u_j; with
  // dot = u_j^T x over a column, row j of R is top - c1 dot and the column
  // update of the next pass is x -= (c2 dot) u_j: c1 = tau scal,
  // c2 = tau scal^2 (no scaling pass over the reflector)
  double c1 = 0.0, c2 = 0.0, uj = 0.0;
  for (int j = 0; j <= kmax; ++j) {
    // ---- (a) finish step j-1 on the own live columns: tw_{j-1} from the
    // partial dots, row j-1 of R, norm down-date; local argmax
    for (int t = tid; t < nl; t += NT) {
      if (j >= 1) {
        const double dot = tree_sum<NW>(S.part + t);
        S.tw[t] = c2 * dot;
        const double rjc = S.top[t] - c1 * dot;
        W[(long long)S.lc[t] * ldw + (j - 1)] = rjc;
        const double v = __fma_rn(-rjc, rjc, S.nrm[t]);
        if (v <= tol3z * S.orig[t]) S.rc[atomicAdd(&s_nrc, 1)] = t;
        else S.nrm[t] = v;
      }
    }
    __syncthreads();
    if (j == kmax) break;
    if (s_nrc > 0) {
      // exact norm^2 of rows >= j of the columns (with H_{j-1} applied)
      for (int q = warp; q < s_nrc; q += NW) {
        const int t = S.rc[q];
        const double* col = W + (long long)S.lc[t] * ldw;
        const double twv = S.tw[t];
        double s2 = 0.0;
        for (int r = j + lane; r < d; r += 32) {
          const double x = __fma_rn(-twv, vp[r], col[r]);
          s2 = __fma_rn(x, x, s2);
        }
        s2 = warp_sum(s2);
        if (lane == 0) { S.nrm[t] = s2; S.orig[t] = s2; }
      }
      __syncthreads();
    }
    // argmax on integer keys: the bit patterns of non-negative doubles are
    // ordered like their values (no FP64 compares on the critical path)
    // the column at the last position of the group's live list goes to the
    // pivot's owner after this step (the live list stays balanced, one
    // position in P per CTA): its owner publishes its state beside the
    // argmax partials
    const int lastpos = m - 1 - j;
    if (tid == 0) s_tl = -1;
    __syncthreads();
    unsigned long long bk = 0ull;
    int bi = 0x7fffffff, bp = -1;
    for (int t = tid; t < nl; t += NT) {
      key_max(bk, bi, bp, (unsigned long long)__double_as_longlong(S.nrm[t]), S.lc[t], t);
      if (S.gp[t] == lastpos) {
        s_tl = t;
        if (P > 1) {
          double* xf = jb.xfer + (j & 1) * 4;
          __stcg(xf, (double)S.lc[t]);
          __stcg(xf + 1, S.tw[t]);
          __stcg(xf + 2, S.nrm[t]);
          __stcg(xf + 3, S.orig[t]);
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, bk, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
      const int p2 = __shfl_xor_sync(0xffffffffu, bp, o);
      key_max(bk, bi, bp, k2, i2, p2);
    }
    if (lane == 0) { shk[warp] = bk; shi[warp] = bi; shp[warp] = bp; }
    __syncthreads();
    if (tid == 0) {
      unsigned long long kk = shk[0];
      int i = shi[0], pos = shp[0];
      for (int w = 1; w < NW; ++w) key_max(kk, i, pos, shk[w], shi[w], shp[w]);
      const double twc = pos >= 0 ? S.tw[pos] : 0.0;
      if (P > 1) {
        // partials of step j in buffer j & 1: a CTA that runs ahead writes the
        // next step's into the other buffer while the group still reads these
        const int pb = (j & 1) * P + rank;
        __stcg((ulonglong2*)jb.redv + pb, make_ulonglong2(kk, (unsigned long long)(unsigned)i));
        __stcg(jb.redt + pb, twc);
      }
      s_p = i;
      s_pos = pos;
      s_twp = twc;
    }
    // ---- (b) the pivot of step j over the group
    if (!group_barrier(jb.bar, P, epoch, err, &s_ok, jb.wait_ns)) return;
    if (P > 1 && warp == 1 && lane < 4) s_xf[lane] = __ldcg(jb.xfer + (j & 1) * 4 + lane);
    if (P > 1 && warp == 0) {
      unsigned long long kk = 0ull;
      int i = 0x7fffffff;
      double tw2 = 0.0;
      const int pb = (j & 1) * P;
      for (int q = lane; q < P; q += 32) {
        const ulonglong2 e = __ldcg((const ulonglong2*)jb.redv + pb + q);
        const double t2 = __ldcg(jb.redt + pb + q);
        const int i2 = (int)(unsigned)e.y;
        if (e.x > kk || (e.x == kk && i2 < i)) { kk = e.x; i = i2; tw2 = t2; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, kk, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, i, o);
        const double t2 = __shfl_xor_sync(0xffffffffu, tw2, o);
        if (k2 > kk || (k2 == kk && i2 < i)) { kk = k2; i = i2; tw2 = t2; }
      }
      if (lane == 0) {
        if (s_p != i) s_pos = -1;   // the pivot is another CTA's column
        s_p = i;
        s_twp = tw2;
      }
    }
    __syncthreads();
    const int p = s_p;
    // ---- (c) pivot column with H_{j-1} applied, exact norm, reflector
    {
      const double* pc = W + (long long)p * ldw;
      const double twp = s_twp;
      double s = 0.0;
      for (int r0 = j + tid; r0 < d; r0 += PCU * NT) {   // PCU loads in flight per thread
        double xv[PCU];
#pragma unroll
        for (int u = 0; u < PCU; ++u) {
          const int r = r0 + u * NT;
          xv[u] = r < d ? (P > 1 ? __ldcg(pc + r) : pc[r]) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < PCU; ++u) {
          const int r = r0 + u * NT;
          if (r < d) {
            const double x = __fma_rn(-twp, vp[r], xv[u]);
            vc[r] = x;
            s = __fma_rn(x, x, s);
          }
        }
      }
      const double ss = block_sum<NW>(s, sh);
      // thread 0: norm, stop test, tau; thread 32 (another warp, so the two
      // FP64 divisions run side by side): the scaling of the reflector
      if (tid == 0 || tid == 32) {
        const double alpha = sqrt(ss);
        double thr_a, thr_r;
        if (j == 0) {
          if (tid == 0) s_r11 = alpha;
          rank_thresholds(jb, d, 0, alpha, thr_a, thr_r);
        } else {
          thr_a = s_th[j & 1][0];
          thr_r = s_th[j & 1][1];
        }
        const int stop = (alpha <= thr_a || alpha <= thr_r) ? 1 : 0;
        const double x0 = vc[j];
        const double beta = x0 >= 0.0 ? -alpha : alpha;
        if (tid == 32) {
          if (!stop) s_scal = 1.0 / (x0 - beta);
        } else {
          s_stop = stop;
          if (!stop) {
            s_tau = (beta - x0) / beta;
            s_uj = x0 - beta;
            // live list update: the pivot leaves; the column at the last
            // position takes the pivot's position, and so moves to the
            // pivot's owner (possibly from another CTA of the group)
            const int pos = s_pos, tl = s_tl;
            int nn = nl;
            auto move = [&](int to, int from) {
              S.lc[to] = S.lc[from]; S.tw[to] = S.tw[from]; S.nrm[to] = S.nrm[from];
              S.orig[to] = S.orig[from]; S.gp[to] = S.gp[from];
            };
            if (pos >= 0) {
              __stcg(diag + j, beta);
              __stcg(jb.piv + j, p);
              liveg[p] = -1.0;
              const int gpos = S.gp[pos];
              if (gpos == lastpos) {            // the pivot was the last column
                move(pos, nn - 1);
                nn -= 1;
              } else if (tl >= 0) {             // the last column is this CTA's too
                move(pos, tl);
                S.gp[pos] = gpos;
                if (tl != nn - 1) move(tl, nn - 1);
                nn -= 1;
              } else {                          // it comes from another CTA
                S.lc[pos] = (int)s_xf[0]; S.tw[pos] = s_xf[1]; S.nrm[pos] = s_xf[2]; S.orig[pos] = s_xf[3];
                S.gp[pos] = gpos;
              }
            } else if (tl >= 0) {               // this CTA's last column went to the pivot's owner
              if (tl != nn - 1) move(tl, nn - 1);
              nn -= 1;
            }
            s_nl = nn;
          }
        }
      }
      if (tid == 64 && j + 1 < kmax) {
        // the thresholds of the next step, beside the two divisions above
        const double r11 = j == 0 ? sqrt(ss) : s_r11;
        rank_thresholds(jb, d, j + 1, r11, s_th[(j + 1) & 1][0], s_th[(j + 1) & 1][1]);
      }
      __syncthreads();
      if (s_stop) { k = j; stopped = 1; break; }
      nl = s_nl;
      c1 = s_tau * s_scal;
      c2 = c1 * s_scal;
      uj = s_uj;   // u_j(j); vc[j] keeps x(j), which the pass replaces by uj
    }
    // ---- (d) the fused pass: rows r >= j of the own live columns,
    //   x = W(r,c) - tw_{j-1}(c) u_{j-1}(r);  W(r,c) = x;  dot += u_j(r) x
    // A warp takes four live columns at a time (a batch), eight lanes per
    // column, lane i of a group one quad (4 rows) of each block of 8 quads,
    // so that every 16-byte load of the warp touches four 128-byte lines.
    // The blocks of a batch are dealt to the warps round robin, two at a
    // time (a unit); a warp walks its units across the batches in order and
    // loads the next unit while it computes the current one, so the loads
    // of one batch overlap the arithmetic of the previous.  At the end of a
    // batch the eight lanes of a column add their partial dots with three
    // shuffles; a batch in which a warp has no block leaves its zero.
    {
      if (tid == 0) s_nrc = 0;   // read for the last time before the pivot step
      const int q0 = j >> 2, q1 = (d + 3) >> 2;
      const int B0 = q0 >> 3, NB = ((q1 + 7) >> 3) - B0;
      const int g = lane >> 3, i8 = lane & 7;
      const int nbat = (nl + 3) >> 2;
      for (int t = lane; t < nl; t += 32) S.part[warp * NLMAX + t] = 0.0;
      __syncwarp();
      // the warp's first block of batch b; units step by two blocks per warp
      auto first_blk = [&](int bb) { return (warp - (bb * NB) % NW + NW) % NW; };
      auto advance = [&](int& bb, int& bk) {
        while (bb < nbat && bk >= NB) {
          ++bb;
          if (bb < nbat) bk = first_blk(bb);
        }
      };
      auto load = [&](int bb, int bk, double2& a01, double2& a23, double2& b01, double2& b23, bool& va,
                      bool& vb) {
        const int t = 4 * bb + g;
        const bool act = t < nl;
        const double* col = W + (long long)(act ? S.lc[t] : 0) * ldw;
        const int qa = 8 * (B0 + bk) + i8, qb = qa + 8 * NW;
        va = act && qa >= q0 && qa < q1;
        vb = act && bk + NW < NB && qb >= q0 && qb < q1;
        if (va) { const double2* pp = (const double2*)(col + 4 * qa); a01 = pp[0]; a23 = pp[1]; }
        if (vb) { const double2* pp = (const double2*)(col + 4 * qb); b01 = pp[0]; b23 = pp[1]; }
      };
      int b = 0, blk = first_blk(0);
      advance(b, blk);
      const double2 z2 = make_double2(0.0, 0.0);
      double2 ca01 = z2, ca23 = z2, cb01 = z2, cb23 = z2;
      bool cva = false, cvb = false;
      if (b < nbat) load(b, blk, ca01, ca23, cb01, cb23, cva, cvb);
      double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;   // four short chains
      while (b < nbat) {
        // the next unit, its loads in flight during this unit's arithmetic
        int nb = b, nbk = blk + 2 * NW;
        advance(nb, nbk);
        double2 na01 = z2, na23 = z2, nb01 = z2, nb23 = z2;
        bool nva = false, nvb = false;
        if (nb < nbat) load(nb, nbk, na01, na23, nb01, nb23, nva, nvb);
        const int t = 4 * b + g;
        const bool act = t < nl;
        double* col = W + (long long)(act ? S.lc[t] : 0) * ldw;
        const double twv = act ? S.tw[t] : 0.0;
        const int qa = 8 * (B0 + blk) + i8, qb = qa + 8 * NW;
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const bool v = h2 ? cvb : cva;
          if (!v) continue;
          const int r = 4 * (h2 ? qb : qa);
          double x[4] = {h2 ? cb01.x : ca01.x, h2 ? cb01.y : ca01.y, h2 ? cb23.x : ca23.x, h2 ? cb23.y : ca23.y};
          const double2 p01 = *(const double2*)(vp + r), p23 = *(const double2*)(vp + r + 2);
          const double2 c01 = *(const double2*)(vc + r), c23 = *(const double2*)(vc + r + 2);
          const double pv[4] = {p01.x, p01.y, p23.x, p23.y};
          const double cv[4] = {r == j ? uj : c01.x, r + 1 == j ? uj : c01.y, r + 2 == j ? uj : c23.x,
                                r + 3 == j ? uj : c23.y};
          if (r >= j && r + 4 <= d) {
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = __fma_rn(-twv, pv[u], x[u]);
            acc0 = __fma_rn(cv[0], x[0], acc0);
            acc1 = __fma_rn(cv[1], x[1], acc1);
            acc2 = __fma_rn(cv[2], x[2], acc2);
            acc3 = __fma_rn(cv[3], x[3], acc3);
            if (r == j) S.top[t] = x[0];
          } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              if (r + u >= j && r + u < d) {
                x[u] = __fma_rn(-twv, pv[u], x[u]);
                if (u == 0) acc0 = __fma_rn(cv[u], x[u], acc0);
                else if (u == 1) acc1 = __fma_rn(cv[u], x[u], acc1);
                else if (u == 2) acc2 = __fma_rn(cv[u], x[u], acc2);
                else acc3 = __fma_rn(cv[u], x[u], acc3);
              }
            }
            if (r <= j && j < r + 4) {
              const int u = j - r;   // select without indexing x (keeps it in registers)
              S.top[t] = u == 0 ? x[0] : (u == 1 ? x[1] : (u == 2 ? x[2] : x[3]));
            }
          }
          double2* pp = (double2*)(col + r);
          pp[0] = make_double2(x[0], x[1]);
          pp[1] = make_double2(x[2], x[3]);
        }
        if (nb != b) {   // the batch is done: its partial dots
          double acc = (acc0 + acc1) + (acc2 + acc3);
          acc += __shfl_xor_sync(0xffffffffu, acc, 4);
          acc += __shfl_xor_sync(0xffffffffu, acc, 2);
          acc += __shfl_xor_sync(0xffffffffu, acc, 1);
          if (act && i8 == 0) S.part[warp * NLMAX + t] = acc;
          acc0 = acc1 = acc2 = acc3 = 0.0;
        }
        b = nb;
        blk = nbk;
        ca01 = na01; ca23 = na23; cb01 = nb01; cb23 = nb23;
        cva = nva; cvb = nvb;
      }
      // swap the reflectors: v_j becomes the one to apply next
      double* tmp = vp;
      vp = vc;
      vc = tmp;
      __syncthreads();
    }
  }

  // every R entry, pivot and liveness flag of the group visible before the solve
  if (!group_barrier(jb.bar, P, epoch, err, &s_ok, jb.wait_ns)) return;

  int accepted = 1;
  if (jb.rule == 1) accepted = stopped ? (k <= d - jb.p) : (k == m);
  // surviving columns after the k pivots, in column order (rank 0)
  if (rank == 0) {
    int base = k;
    for (int c0 = 0; c0 < m; c0 += NT) {
      const int c = c0 + tid;
      const int live = (c < m) && __ldcg(liveg + c) > 0.0;
      const unsigned bal = __ballot_sync(0xffffffffu, live);
      const int wpre = __popc(bal & ((1u << lane) - 1u));
      if (lane == 0) shi[warp] = __popc(bal);
      __syncthreads();
      int off = base;
      for (int w = 0; w < warp; ++w) off += shi[w];
      int tot = 0;
      for (int w = 0; w < NW; ++w) tot += shi[w];
      if (live) __stcg(jb.piv + off + wpre, c);
      __syncthreads();
      base += tot;
    }
  }
  if (jb.do_id && accepted && k > 0 && k < m) {
    // X = R1^{-1} R2 in place on the own surviving columns, by blocks of up
    // to EB rows from the bottom: the diagonal block is solved in shared
    // memory (a thread per column), then the rows above take one update of
    // depth EB, X(r, c) -= sum_b R1(r, i0 + b) X(i0 + b, c) (a thread per
    // row), so an entry of X is read and written once per block, not once
    // per row.  R1(r, i) = W(r, piv[i]) for r < i.
    const int dp = (dmax + 3) & ~3;
    double* rd = S.v0;   // 1 / R_ii
    double* xs = S.v1;   // the block's rows of X, row-major (ld nc)
    double* rb = S.part; // the block of R1, rb[a * EB + b] = R1(i0 + a, i0 + b)
    int* pb = S.rc;      // piv[i0 .. i1)
    for (int i = tid; i < k; i += NT) rd[i] = 1.0 / __ldcg(diag + i);
    for (int c0 = 0; c0 < nl; c0 += dp) {   // own columns in chunks whose block rows fit xs
      const int nc = min(nl - c0, dp);
      const int BR = max(1, min(EB, dp / nc));
      for (int i1 = k; i1 > 0; i1 -= BR) {
        const int i0 = max(0, i1 - BR), nb = i1 - i0;
        __syncthreads();   // xs, rb, pb free; rd written
        for (int a = tid; a < nb; a += NT) pb[a] = __ldcg(jb.piv + i0 + a);
        for (int e = tid; e < nb * nc; e += NT) {
          const int a = e / nc, c = e - a * nc;
          xs[e] = W[(long long)S.lc[c0 + c] * ldw + i0 + a];
        }
        __syncthreads();
        for (int e = tid; e < nb * nb; e += NT) {
          const int a = e / nb, b = e - a * nb;
          rb[a * EB + b] = a < b ? __ldcg(W + (long long)pb[b] * ldw + i0 + a) : 0.0;
        }
        __syncthreads();
        for (int c = tid; c < nc; c += NT) {
          double* col = W + (long long)S.lc[c0 + c] * ldw;
          for (int b = nb - 1; b >= 0; --b) {
            const double x = xs[b * nc + c] * rd[i0 + b];
            xs[b * nc + c] = x;
            col[i0 + b] = x;
            for (int a = 0; a < b; ++a) xs[a * nc + c] = __fma_rn(-rb[a * EB + b], x, xs[a * nc + c]);
          }
        }
        __syncthreads();
        for (int r = tid; r < i0; r += NT) {
          double rv[EB];
#pragma unroll
          for (int b = 0; b < EB; ++b) rv[b] = b < nb ? __ldcg(W + (long long)pb[b] * ldw + r) : 0.0;
          for (int c = 0; c < nc; ++c) {
            double a0 = 0.0, a1 = 0.0;
#pragma unroll
            for (int b = 0; b < EB; b += 2) {
              if (b < nb) a0 = __fma_rn(rv[b], xs[b * nc + c], a0);
              if (b + 1 < nb) a1 = __fma_rn(rv[b + 1], xs[(b + 1) * nc + c], a1);
            }
            double* dst = W + (long long)S.lc[c0 + c] * ldw + r;
            *dst -= a0 + a1;
          }
        }
      }
    }
  }
  if (rank == 0 && tid == 0) { jb.out[0] = k; jb.out[1] = stopped; jb.out[2] = accepted; }
}

size_t smem_for(int dmax, int nt) {
  const size_t dp = ((size_t)dmax + 3) & ~(size_t)3;
  return sizeof(double) * (2 * dp + (nt / 32 + 4) * (size_t)NLMAX) + 3 * sizeof(int) * NLMAX;
}

template <int NT>
int group_capacity(int dmax, int* nsm_out, int* per_out) {
  int dev = 0, sms = 0, per = 0;
  const size_t sm = smem_for(dmax, NT);
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaFuncSetAttribute(k_qrcp<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_qrcp<NT>, NT, sm) != cudaSuccess) return 0;
  if (nsm_out) *nsm_out = sms;
  if (per_out) *per_out = per;
  return sms * per;
}

template <int NT>
cudaError_t launch(const QrcpJob* jobs_dev, const int2* map_dev, int nctas, int dmax, int* err, unsigned* place,
                   int nsm, int per, cudaStream_t st) {
  const size_t sm = smem_for(dmax, NT);
  cudaError_t e = cudaFuncSetAttribute(k_qrcp<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  if (!map_dev) {
    k_qrcp<NT><<<nctas, NT, sm, st>>>(jobs_dev, nullptr, err, dmax, nullptr, 0, 0);
    return cudaGetLastError();
  }
  if (place && nctas != nsm * per) return cudaErrorInvalidValue;   // placement needs every slot filled
  void* args[] = {(void*)&jobs_dev, (void*)&map_dev, (void*)&err, (void*)&dmax, (void*)&place, (void*)&nsm,
                  (void*)&per};
  return cudaLaunchCooperativeKernel((const void*)k_qrcp<NT>, dim3(nctas), dim3(NT), args, sm, st);
}

}  // namespace

int qrcp_cols_per_cta() { return NLMAX; }

// Co-resident CTAs of k_qrcp on this device for sample width dmax, in shape
// 2 (512 threads), 1 (256) or 0 (128).
int qrcp_group_capacity(int dmax, int wide, int* nsm, int* per) {
  if (wide == 2) return group_capacity<NT_XWIDE>(dmax, nsm, per);
  return wide ? group_capacity<NT_WIDE>(dmax, nsm, per) : group_capacity<NT_NARROW>(dmax, nsm, per);
}

// map == nullptr: one CTA per job (ordinary launch); otherwise map[cta] =
// (job, rank) and the launch is cooperative.  dmax: largest d of the jobs.
cudaError_t launch_qrcp(const QrcpJob* jobs_dev, const int2* map_dev, int nctas, int dmax, int wide, int* err,
                        unsigned* place, int nsm, int per, cudaStream_t st) {
  if (nctas <= 0) return cudaSuccess;
  if (wide == 2) return launch<NT_XWIDE>(jobs_dev, map_dev, nctas, dmax, err, place, nsm, per, st);
  return wide ? launch<NT_WIDE>(jobs_dev, map_dev, nctas, dmax, err, place, nsm, per, st)
              : launch<NT_NARROW>(jobs_dev, map_dev, nctas, dmax, err, place, nsm, per, st);
}

}  // namespace hss
