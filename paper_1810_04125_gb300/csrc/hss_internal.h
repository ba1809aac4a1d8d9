// Internal declarations shared by the host driver and the kernels of the
// HSS library.  Nothing here is part of the C ABI (include/hss.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hss.h"

namespace hss {

// Device view of an hss_source plus the leaf id of every index (entries of
// A inside one leaf's diagonal block are "on the diagonal" and are removed
// from the sampled matrix, eq. sample_off_diag at the leaf level).
struct SrcDev {
  int kind, n, dim, pad;
  const double* a;
  const double* b;
  long long ld;
  double p0, p1;
  const int* leaf_id;   // n entries, nondecreasing
};

// Entry A(i, j) in FP64 (the definitions of HSS_SRC_*).
__device__ __forceinline__ double entry(const SrcDev& s, int i, int j) {
  switch (s.kind) {
    case HSS_SRC_DENSE:
      return s.a[(long long)i + (long long)j * s.ld];
    case HSS_SRC_TOEPLITZ:
      return i >= j ? s.a[i - j] : s.b[j - i];
    case HSS_SRC_GAUSS: {
      double r2 = 0.0;
      for (int c = 0; c < s.dim; ++c) {
        double t = s.a[i + c * s.ld] - s.a[j + c * s.ld];
        r2 = __fma_rn(t, t, r2);
      }
      return exp(-r2 / (2.0 * s.p0 * s.p0)) + (i == j ? s.p1 : 0.0);
    }
    default: {  // HSS_SRC_LAPLACE
      if (i == j) return s.p0;
      double r2 = 0.0;
      for (int c = 0; c < 3; ++c) {
        double t = s.a[i + c * s.ld] - s.a[j + c * s.ld];
        r2 = __fma_rn(t, t, r2);
      }
      return 1.0 / (4.0 * 3.141592653589793 * sqrt(r2));
    }
  }
}

// A strided operand view: logical element (i, l) is
//   base[r * rs + l * cs]  with r = rows ? rows[i] : i, and base = p, or p2
//   with r -= split when r >= split (two stacked blocks).
struct Opnd {
  const double* p;
  const double* p2;
  long long rs, cs;
  const int* rows;
  int split;
};

// Generic batched FP64 tile product, one 64 x 64 output tile per CTA:
//   C(rows_c[i], j) = alpha * sum_l A(i, l) B(l, j) + beta * C0(i, j)
//                     + gamma * C(rows_c[i], j)
struct GemmJob {
  Opnd A, B, C0;
  double* C;
  long long c_rs, c_cs;
  const int* c_rows;
  double* C2;           // second output block for rows >= c_split
  int c_split;
  int M, N, K;
  double alpha, beta, gamma;
  // tensor-core form with packed operands (launch_gemm_tc_packed): A as
  // tiles (ti, kt) of 128 rows x 32 k, B^T as tiles (tj, kt) of tile_n rows
  // x 32 k, the three TF32 terms of a tile one after another
  unsigned char* pa;
  unsigned char* pb;
  int nkt;
};
// One tile of an operand to pack: job, operand (0 = A, 1 = B), row tile, k tile.
struct PackUnit { int job, which, tile, kt; };
// One output tile of one job; k0..k1 is its share of K (split-K tiles add
// alpha * partial into C atomically: the job then has beta == 0 and
// gamma == 1, or gamma == 0 with C zeroed beforehand).
struct GemmTile { int job, ti, tj, k0, k1; };

// QR with column pivoting of W = S^T (S: m x d rows, row-major ld lds),
// truncated by the plain rule (rule 0) or the HMT-scaled rule (rule 1),
// followed by X = R1^{-1} R2 when accepted and do_id.  Columns are not
// swapped: piv[0:k] lists the pivot columns, piv[k:m] the others in column
// order, and X(:, t) is left in W(0:k, piv[k + t]).
struct QrcpJob {
  const double* S;
  long long lds;
  int m, d;
  double* W;            // workspace, col-major d x m, ld = ldw
  long long ldw;
  double* nrm;          // workspace m (column liveness)
  double* diag;         // workspace min(d, m): R_jj
  int* piv;             // out: m entries
  int rule;             // 0 plain, 1 HMT
  int mh, nh, p;        // Hankel block sizes and oversampling (HMT)
  int do_id;
  double er, ea;
  int* out;             // out[0] = k, out[1] = stopped, out[2] = accepted
  // group (multi-CTA) form only
  int P;                // CTAs working on this job
  unsigned* bar;        // group barrier counter, zero before the launch
  double* redv;         // 2 P partial maxima as 16-byte (norm bits, column) pairs,
                        // two steps in flight, 16-byte aligned
  double* redt;         // 2 P pending-update coefficients of the candidates
  double* xfer;         // 2 x 4: the column moved between CTAs at a step (id, tw,
                        // norm^2, orig), two steps in flight
  unsigned long long wait_ns;  // bound of one group-barrier wait (%globaltimer ns)
};

// One Incrementing block test on one side of a node (Algorithm 5):
// Sh = (I - Q Q^T)^2 S(:, c0:c0+b), norms, Householder QR of Sh, the four
// tests of eq. stopping_criteria, and on failure Q <- [Q Q_k].
struct IncJob {
  const double* S;      // m x lds row-major local sample
  long long lds;
  int m, c0, b;
  double* Q;            // m x lds row-major, q columns in use
  int q;
  double* Sh;           // workspace m x b col-major (ld m)
  double* T;            // workspace q x b col-major (ld q)
  double* tau;          // workspace b
  double er, ea;
  double rho;           // |(R_1)_11| of the first block, < 0 if none yet
  int hmt;              // 1: the HMT criterion (Lemma 4.1) instead of eq. stopping_criteria
  double hmt_c;         // alpha sqrt(2/pi) of the HMT criterion
  double* res;          // out: [0]=|S_k|_F, [1]=|Sh|_F, [2]=min|diag| (the HMT estimate
                        // with hmt), [3]=|R_11|
  int* flag;            // out: [0]=sufficient, [1]=new q
  // group form (launch_inc_group): P CTAs split the m rows
  int P;
  unsigned* bar;        // group barrier counter, zero before the launch
  double* part;         // inc_group_part(P, b) doubles of partial sums
  unsigned long long wait_ns;  // bound of one group-barrier wait (%globaltimer ns)
};

// Gather of sub-blocks of A: out(i, j) = A(I[i], J[j]) (col-major, ld ldo);
// I or J may be NULL meaning i0 + i / j0 + j.  src: the source of the
// entries (one launch serves the blocks of several matrices).
struct ExtractJob {
  const int* I; int i0, mi;
  const int* J; int j0, nj;
  double* out; long long ldo;
  SrcDev src;
};

// dst[t] = (idx[t] < split ? src[idx[t]] : src2[idx[t] - split]) for t < cnt:
// the skeleton index composition tau.I = [nu1.I nu2.I](tau.J) of Algorithm 2
struct GatherJob {
  const int* src;
  const int* src2;
  const int* idx;
  int* dst;
  int cnt, split;
};

// One node of a compressed handle as the entry kernels read it
// (k_entries.cu): tree, state, ranks, inverse pivot orders (position of each
// sample row in the pivot order), X of U and V, and the blocks D, B12, B21
// (F12, F21: the dense blocks of a node left uncompressed).
struct EntryNode {
  int lo, size, level, parent, ch0, ch1, state;
  int kr, kc, mr, mc;
  const int* pivr;
  const int* pivc;
  int* ipivr;
  int* ipivc;
  const double* Xr;
  const double* Xc;
  const double* D;
  const double* B12;
  const double* B21;
  const double* F12;
  const double* F21;
};

// Launch wrappers (return cudaError_t of the launch).
cudaError_t launch_random_normal(unsigned long long seed, int n, int col0, int ncols,
                                 double* R, long long ldr, int round_mode, cudaStream_t st);
cudaError_t launch_sample_fp64(const SrcDev& src, int ncols, const double* R, long long ldr,
                               double* Sr, double* Sc, long long lds, cudaStream_t st);
// tcgen05 mixed-precision sampling with entries generated in the kernel
// (k_sample_tc.cu); Rp is R packed by launch_pack_r; *used_atomic tells
// whether S had to be zeroed beforehand (K split across CTAs).  toep: for a
// Toeplitz source, its diagonals split into the terms of the precision
// (launch_toeplitz_terms, toeplitz_terms_bytes), else NULL.
cudaError_t launch_sample_tc(const SrcDev& src, int leaf, int precision, int trans, int ncols,
                             const void* Rp, double* S, long long lds, int* err, int* used_atomic,
                             const void* toep, cudaStream_t st);
size_t toeplitz_terms_bytes(int n, int precision);
cudaError_t launch_toeplitz_terms(const SrcDev& src, int precision, void* out, cudaStream_t st);
int sample_tc_ksplit(int n, int ncols, int precision);
// packed form for a dense A: operands split once into canonical tiles in
// global memory, the main loop fed by bulk copies (k_sample_tc.cu)
size_t packed_a_bytes(int n, int precision);
size_t packed_r_bytes(int n, int ncols, int precision);
cudaError_t launch_pack_a(const SrcDev& src, int leaf, int precision, void* out, cudaStream_t st);
cudaError_t launch_pack_r(const double* R, long long ldr, int n, int ncols, int precision, void* out,
                          cudaStream_t st);
int sample_tc_packed_ksplit(int n, int ncols, int precision);
cudaError_t launch_sample_tc_packed(const void* A, const void* Rp, int n, int ncols, int precision,
                                    int trans, double* S, long long lds, int* err, cudaStream_t st);
// out(:, c) = R rounded to the significand of the mixed format (mode 1: 11
// bits, TF32; mode 2: 8 bits, BF16)
cudaError_t launch_round_copy(const double* in, long long ldin, double* out, long long ldout, int n,
                              int ncols, int mode, cudaStream_t st);
cudaError_t launch_extract(const ExtractJob* jobs_dev, int njobs, int max_tiles, cudaStream_t st);
cudaError_t launch_gemm(const GemmJob* jobs_dev, const GemmTile* tiles_dev, int ntiles,
                        cudaStream_t st);
// The same contract with the product on tcgen05 tensor cores, operands split
// into three TF32 terms (k_gemm_tc.cu): tiles of 128 rows x tile_n columns
// (gemm_tc_tile_n); *err records a wait that gave up.
int gemm_tc_tile_n(int max_n);
cudaError_t launch_gemm_tc(const GemmJob* jobs_dev, const GemmTile* tiles_dev, int ntiles, int tile_n,
                           int* err, cudaStream_t st);
// The same product from operands split once into their TF32 terms: the
// pack kernel writes every listed operand tile (bytes per tile:
// gemm_tc_tile_bytes), then one thread per CTA streams a tile pair per k-tile
// by bulk copy and sixteen warps drain the chains.
size_t gemm_tc_tile_bytes(int which, int tile_n);
cudaError_t launch_gemm_tc_pack(const GemmJob* jobs_dev, const PackUnit* units_dev, int nunits, int tile_n,
                                cudaStream_t st);
cudaError_t launch_gemm_tc_packed(const GemmJob* jobs_dev, const GemmTile* tiles_dev, int ntiles, int tile_n,
                                  int* err, cudaStream_t st);
// map == nullptr: one CTA per job; otherwise the launch is cooperative and
// map holds the (job, rank within the job's group) of every position, (-1,
// -1) for an idle one.  With place == nullptr CTA b takes map[b]; with
// place (QRCP_PLACE_WORDS zeroed words) the launch fills every co-resident
// slot (nctas = nsm x per) and CTA takes map[slot x nsm + its SM's index], so
// that the ranks of one group that sit at consecutive positions run on
// different SMs (it falls back to map[b] when the SMs do not hold exactly
// per CTAs each).  d_max: largest d.  A CTA owns at most qrcp_cols_per_cta()
// columns (m / P); W is col-major with ldw a multiple of 4; nrm holds m
// doubles.
// The process-wide launch-shape parameters (hss_set_tuning).
hss_tuning tuning_get();
// wide: 2 = 512 threads and one CTA per SM, 1 = 256 threads and two, 0 = 128
// threads and four.
constexpr int QRCP_PLACE_WORDS = 1024 + 32 + 4;
int qrcp_cols_per_cta();
int qrcp_group_capacity(int d_max, int wide, int* nsm = nullptr, int* per = nullptr);
cudaError_t launch_qrcp(const QrcpJob* jobs_dev, const int2* map_dev, int nctas, int d_max, int wide, int* err,
                        unsigned* place, int nsm, int per, cudaStream_t st);
// With a user sampling operator: S(i, c0 + q) = T(i, q) - sum_{j in leaf(i)}
// A(i, j) R(j, q) (trans = 0) or A(j, i) (trans = 1) for i < n, q < w: the
// leaf diagonal blocks removed from the user's product T (col-major, ld ldt)
// into the row-major samples S (ld lds, column offset applied by the caller).
// Dp + doff[L]: leaf L's block D (col-major, ld = its size); leaf_id gives
// each row's leaf, leaf_lo the nleaves + 1 row bounds.
cudaError_t launch_leaf_diag_sub(const double* Dp, const long long* doff, const int* leaf_id, const int* leaf_lo,
                                 int n, int w, const double* R, long long ldr, const double* T, long long ldt,
                                 double* S, long long lds, int trans, cudaStream_t st);
cudaError_t launch_inc_qr(const IncJob* jobs_dev, int njobs, cudaStream_t st);
// The same test with the rows of each side split over a group of P CTAs
// (map[cta] = (job, rank), cooperative launch); b_max: largest block, at
// most inc_group_bmax().
int inc_group_rows(int b);                 // most rows per CTA for a block of b columns
size_t inc_group_part(int P, int b);       // doubles of a side's partial-sum area (IncJob.part)
int inc_group_bmax();
int inc_group_capacity(int b_max);          // co-resident CTAs
cudaError_t launch_inc_group(const IncJob* jobs_dev, const int2* map_dev, int nctas, int b_max, int* err,
                             cudaStream_t st);
cudaError_t launch_nonfinite(const double* S, long long lds, int n, int c0, int c1,
                             int* flag, cudaStream_t st);
cudaError_t launch_identity_block(double* X, int n, int c0, int w, cudaStream_t st);
cudaError_t launch_gather_int(const GatherJob* jobs_dev, int njobs, int max_cnt, cudaStream_t st);
// entries of a compressed handle (k_entries.cu); err: 1 = index out of
// range, 2 = pivot out of range
cudaError_t launch_inv_piv(const EntryNode* nodes, int nn, int* err, cudaStream_t st);
cudaError_t launch_entry_paths(const EntryNode* nodes, const int* leaf_of, int n, const int* idx, int count,
                               double* out, int kcap, int lp1, int side, int* err, cudaStream_t st);
cudaError_t launch_entry_pairs(const EntryNode* nodes, const int* leaf_of, int n, const int* I, int nr, const int* J,
                               int nc, const double* Wrow, const double* Vcol, int kcap, int lp1, double* out,
                               long long ldo, cudaStream_t st);

}  // namespace hss
