/*
 * hss.h -- C ABI of the GB300 library for adaptive randomized HSS
 * compression (Gorman, Chavez, Ghysels, Mary, Rouet, Li, "Matrix-free
 * construction of HSS representation using adaptive randomized sampling",
 * arXiv:1810.04125).
 *
 * Conventions for every entry point:
 *  - All functions return hss_status (0 = HSS_OK).  None aborts or exits;
 *    the last failure's message is available from hss_last_error().
 *  - "device" pointers are CUDA global-memory pointers of the current
 *    device, owned by the caller and only read (or written, for outputs)
 *    during the call.  "host" pointers are ordinary CPU memory.
 *  - Matrices are FP64.  "col-major" means element (i, j) at p[i + j*ld];
 *    "row-major" means element (i, j) at p[i*ld + j].
 *  - Work is issued on the caller's CUDA stream (NULL = legacy default
 *    stream).  Calls return after their last stream synchronisation,
 *    except hss_matvec, hss_random_normal and hss_sample_offdiag, which
 *    are asynchronous on that stream.
 */
#ifndef HSS_H
#define HSS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HSS_OK = 0,
  HSS_ERR_ARG = 1,            /* invalid argument; nothing was launched        */
  HSS_ERR_NOMEM = 2,          /* device or host allocation failed              */
  HSS_ERR_CUDA = 3,           /* a CUDA call failed (message in last_error)    */
  HSS_ERR_NOT_CONVERGED = 4,  /* d reached d_max with the root not COMPRESSED;
                                 the handle is returned with per-node states
                                 and is usable as a partial result (see
                                 hss_compress)                                 */
  HSS_ERR_NONFINITE = 5,      /* NaN or Inf found in the random samples        */
  HSS_ERR_TIMEOUT = 6,        /* a bounded device wait expired                 */
  HSS_ERR_UNSUPPORTED = 7,    /* option combination not implemented            */
  HSS_ERR_OPERATOR = 8,       /* the user sampling operator returned nonzero   */
  HSS_ERR_IO = 9              /* a file could not be opened, written or renamed */
} hss_status;

/* Sample growth strategy (paper section 2.4): Doubling = Algorithm 4 with
 * the HMT-scaled RRQR stop of eq. RRQRHMTstop; Incrementing = Algorithm 5
 * with the four tests of eq. stopping_criteria. */
enum { HSS_DOUBLING = 0, HSS_INCREMENTING = 1 };

/* Stopping test of the Incrementing strategy (section 2.4).
 *  NEW : the relative and absolute tests of eq. stopping_criteria (the
 *        paper's criterion).
 *  HMT : the probabilistic bound of Lemma 4.1 (eq. HMT_err_bound) in the form
 *        of eq. HMT_IQQH, applied to the node's local sample: a block S_k of
 *        b new columns is sufficient when
 *          alpha sqrt(2/pi) max_i |((I - Q Q^T)^2 S_k)(:, i)|_2 <= eps_a,
 *        which bounds the 2-norm of the part of the sampled operator outside
 *        span(Q) by eps_a except with probability alpha^-b; otherwise the
 *        block's orthonormal basis joins Q.  It knows no relative tolerance:
 *        rtol is ignored, and the final RRQR keeps the pivots with
 *        |R_jj| > eps_a (the paper's Table 3 compares the two criteria).
 *        Incrementing only (HSS_ERR_ARG with Doubling). */
enum { HSS_CRIT_NEW = 0, HSS_CRIT_HMT = 1 };

/* Arithmetic of the sampling product S = A R (the only step that is not
 * FP64 in the mixed forms; the QR, ID, tests and merges are always FP64).
 *  FP64   : plain FP64 products.
 *  TF32X2 : A split as A0 + A1 (two TF32 terms), R rounded once to TF32,
 *           two tensor-core products with FP32 accumulation.
 *  BF16X3 : A split as A0 + A1 + A2 (three BF16 terms), R rounded once to
 *           BF16, three tensor-core products with FP32 accumulation. */
enum { HSS_PREC_FP64 = 0, HSS_PREC_TF32X2 = 1, HSS_PREC_BF16X3 = 2 };

/* Where the entries of A come from (paper section 3.1, "Partially
 * Matrix-Free Interface": sampling plus element extraction A(I, J)). */
enum {
  HSS_SRC_DENSE = 0,     /* a: device col-major n x n, leading dimension ld  */
  HSS_SRC_TOEPLITZ = 1,  /* a: device first column c[0..n-1], A_ij = c[i-j]
                            for i >= j; b: device first row r[0..n-1],
                            A_ij = r[j-i] for j > i (b may equal a)          */
  HSS_SRC_GAUSS = 2,     /* a: device points, col-major n x dim (ld);
                            A_ij = exp(-|x_i - x_j|^2 / (2 p0^2)) + p1 [i==j] */
  HSS_SRC_LAPLACE = 3,   /* a: device points, col-major n x 3 (ld);
                            A_ij = 1 / (4 pi |x_i - x_j|), A_ii = p0          */
  HSS_SRC_EXTRACT = 4    /* the caller's element extraction routine
                            (extract, ctx below; a, b, ld, p0, p1 unused):
                            the matrix is known only through it and the
                            sampling operator opts->op, which is then
                            required                                         */
};

/* One block request of the element extraction routine (section 3.1: the
 * routine returns sub-blocks A(I, J) for row and column index sets):
 * out(i, j) = A(I[i], J[j]) for i < nr, j < nc.  I, J: device int arrays of
 * global indices (0-based); out: device, col-major, leading dimension
 * ldo >= nr.  All three are owned by the library. */
typedef struct hss_block {
  int nr, nc;
  const int* I;
  const int* J;
  double* out;
  long long ldo;
} hss_block;

/* The element extraction routine of an HSS_SRC_EXTRACT source: fills the
 * nblocks requests of `blocks` (a host array, valid during the call) by work
 * it enqueues on `stream` (a cudaStream_t); returns 0, or nonzero on failure
 * (the compression then stops with HSS_ERR_OPERATOR).  As in the paper's
 * level-by-level traversal, the blocks of one tree level come in one call
 * (the B12 and B21 generators of its nodes), the leaf diagonal blocks D in
 * one call before the first sampling pass, and, when d_max is reached
 * without convergence, the dense off-diagonal blocks of the nodes left
 * uncompressed in one more call.  It runs on the host thread that called the
 * compression. */
typedef int (*hss_extract_fn)(void* ctx, int nblocks, const hss_block* blocks, void* stream);

typedef struct hss_source {
  int kind;              /* HSS_SRC_*                                        */
  int n;                 /* matrix order                                     */
  int dim;               /* point dimension (GAUSS, LAPLACE)                 */
  int reserved;
  const double* a;       /* device, see HSS_SRC_*                            */
  const double* b;       /* device, TOEPLITZ first row; NULL otherwise       */
  long long ld;          /* leading dimension of a (DENSE, points)           */
  double p0, p1;         /* kernel parameters, see HSS_SRC_*                 */
  hss_extract_fn extract; /* HSS_SRC_EXTRACT: the extraction routine; NULL
                            otherwise                                        */
  void* ctx;             /* passed to extract unchanged                      */
} hss_source;

/* Node states of Algorithm 3. */
enum { HSS_UNTOUCHED = 0, HSS_PARTIALLY_COMPRESSED = 1, HSS_COMPRESSED = 2 };

/* A user sampling product (section 3.1, the partially matrix-free
 * interface: the construction needs only products with A and A^T and
 * selected entries of A).  apply(ctx, trans, n, ncols, R, ldr, S, lds, stream)
 * must enqueue on `stream` (a cudaStream_t) the product S = A R (trans = 0)
 * or S = A^T R (trans = 1): R and S are device col-major n x ncols with
 * leading dimensions ldr, lds >= n; R is only read, S only written, both
 * owned by the library and valid until the stream reaches the work enqueued
 * after the call returns.  It returns 0, or nonzero on failure (the
 * compression then stops with HSS_ERR_OPERATOR).  The entries of A for the
 * generators (D and B blocks, and the leaf diagonal blocks removed from the
 * samples) come from the hss_source, which must describe the same A (a
 * built-in source, or the caller's extraction routine, HSS_SRC_EXTRACT).
 * The callback runs on the host thread that called the compression, once per
 * orientation and pass. */
typedef int (*hss_apply_fn)(void* ctx, int trans, int n, int ncols, const double* R, long long ldr,
                            double* S, long long lds, void* stream);
typedef struct hss_operator {
  hss_apply_fn apply;
  void* ctx;             /* passed through unchanged                          */
} hss_operator;

typedef struct hss_opts {
  int leaf;              /* leaf size of the halving cluster tree (>= 1)     */
  int strategy;          /* HSS_DOUBLING or HSS_INCREMENTING                  */
  int precision;         /* HSS_PREC_*                                       */
  int level_tol_scaling; /* 1: node tolerances eps/level(tau) (Algorithm 3);
                            0: plain eps                                      */
  double rtol, atol;     /* eps_r, eps_a (> = 0)                              */
  int d0;                /* initial number of random vectors                 */
  int dd;                /* Incrementing step Delta d (ignored by Doubling)  */
  int d_max;             /* cap on the number of random vectors (<= n)       */
  int oversample_p;      /* Doubling oversampling p (paper default 10)       */
  unsigned long long seed; /* Philox key when R == NULL                      */
  const double* R;       /* optional device col-major n x d_max random
                            matrix (ld = n); NULL = generated on the device
                            with Philox4x32-10 (hss_random_normal)            */
  int symmetric;         /* 1: A = A^T (not checked): Algorithm 3 with
                            A^T = A, whose column side copies the row side
                            (S^c = S^r, V = U, B21 = B12^T), so only the row
                            side is sampled, tested and factored; 0: general */
  int criterion;         /* HSS_CRIT_NEW (0, default) or HSS_CRIT_HMT        */
  double hmt_alpha;      /* alpha > 1 of the HMT criterion (Lemma 4.1; the
                            paper's example takes 10); ignored with NEW       */
  const hss_operator* op; /* host; NULL: the library samples A from the
                            source's entries.  Otherwise every pass samples
                            through op (precision must be HSS_PREC_FP64: the
                            product's arithmetic is the operator's) and the
                            library removes the leaf diagonal blocks
                            D_tau R(I_tau) from its result (Algorithm 2)      */
  long long wait_limit_ns; /* bound of each device-side wait of the kernels
                            whose CTAs work on one node side together (QRCP
                            and Incrementing test group barriers), in ns of
                            the GPU's global timer; 0 = about 2 s.  A wait
                            that runs out makes the kernels return and the
                            call fail with HSS_ERR_TIMEOUT; the library stays
                            usable                                           */
} hss_opts;

typedef struct hss_stats {
  int n, n_nodes, levels, d_final, n_adapt, converged;
  int max_rank_r, max_rank_c;
  double ms_total;       /* time of hss_compress on the stream (CUDA events)  */
  double ms_sample;      /* sampling kernels only (events around them)        */
  double ms_rng;         /* random generation and sample checks               */
  double ms_id;          /* QRCP / ID kernels                                 */
  double ms_test;        /* Incrementing projection + QR kernels              */
  double ms_merge;       /* extraction, merge, reduction and bookkeeping      */
  double flop_sample;    /* algorithmic sampling flops, sum of 4 n^2 Delta d
                            (the dense product's count, also with a user
                            operator, whose own work may be far less)       */
  double bytes_sample;   /* algorithmic sampling bytes: one read of A (dense
                            source) + R read + S^r, S^c written, summed      */
  long long launches;    /* kernels launched by the call                      */
  long long sample_launches; /* of which sampling kernels                     */
  long long bytes_h2d;   /* host-to-device bytes copied by the call           */
  long long bytes_d2h;   /* device-to-host bytes copied by the call           */
  double flop_id;        /* algorithmic flops of the QRCP/ID kernels: 2md for
                            the norms, 4(d-j)(m-j-1) + 3(d-j) per pivot step
                            j, k^2 (m-k) for X = R1^{-1} R2                   */
} hss_stats;

typedef struct hss_node_info {
  int lo, size, level, parent, child0, child1; /* tree (level-order index)   */
  int state;             /* HSS_UNTOUCHED / _PARTIALLY_COMPRESSED / _COMPRESSED */
  int mr, mc;            /* rows of the local samples tau.S^r, tau.S^c        */
  int kr, kc;            /* ranks: #J^r (columns of U), #J^c (columns of V)   */
} hss_node_info;

typedef struct hss_matrix_s* hss_matrix;   /* opaque; owns device memory    */

/* Adaptive randomized HSS compression, Algorithm 3 (HSSCompressAdaptive and
 * CompressNodeAdaptive) with Algorithm 2 (ComputeLocalSamples,
 * ReduceLocalSamples), the ID of eq. ID and the strategy of opts->strategy.
 * A: source of the entries of A (device data, or the caller's extraction
 * routine).  out: receives a handle, also on HSS_ERR_NOT_CONVERGED; on any
 * other error *out is NULL.  The handle owns all generator memory until
 * hss_free.
 * HSS_ERR_NOT_CONVERGED (Algorithm 3's loop ends at d_max with the root not
 * COMPRESSED): the node states are those of the last pass, the generators of
 * the COMPRESSED subtrees stand, and the rest of A is kept as it is — for
 * each uncompressed node with children the blocks A(I_nu1, I_nu2) and
 * A(I_nu2, I_nu1) between its children, for the leaves D — so that
 * hss_matvec and hss_to_dense reproduce A exactly outside the compressed
 * subtrees.  When those blocks would take more than half of the free device
 * memory they are not kept, and the handle then serves hss_get_stats,
 * hss_get_node and hss_export_node only (HSS_ERR_ARG from the products). */
hss_status hss_compress(const hss_source* A, const hss_opts* opts, void* stream,
                        hss_matrix* out);

/* The two non-adaptive modes the paper measures its adaptivity against
 * (section 4.3.2, Table 4).  "Known-rank" is hss_compress with
 * opts->d0 == opts->d_max: one pass with a fixed number of random vectors,
 * no growth (HSS_ERR_NOT_CONVERGED if that number is too small).
 * "Hard-restart", this call: without adaptivity a user restarts from scratch
 * with more random vectors when a compression fails.  Attempts with
 * d = d0, 2 d0, 4 d0, ... (the last clipped to d_max), each an hss_compress
 * with d0 = d_max = d on the first d columns of R (opts->R, or the generated
 * R of opts->seed, whose leading columns are the same for every d), nothing
 * carried over between attempts; the strategy's own test decides failure.
 * *out receives the first converged attempt (or the attempt at d_max with
 * HSS_ERR_NOT_CONVERGED, as hss_compress); *restarts (host, may be NULL) the
 * number of failed attempts.  Its stats cover the last attempt only. */
hss_status hss_compress_restart(const hss_source* A, const hss_opts* opts, void* stream,
                                hss_matrix* out, int* restarts);

/* hss_compress for a batch of independent matrices (the paper compresses
 * one matrix per call; the batch has no counterpart there): A[count] and
 * opts[count] (one options struct per matrix; strategies, precisions and
 * sizes may differ), out[count] receives the handles.  The matrices are
 * compressed in lockstep on `stream`, following Algorithm 3's level-by-level
 * traversal (section 3.2) across the whole batch: every step of a level
 * (extraction, merge, Incrementing test, QRCP / ID, reduction) is one launch
 * over the nodes of that level of every matrix (the leaves of all matrices
 * first), and the host reads back ranks and flags once per level for the
 * whole batch.  Matrices run in groups whose estimated device memory fits
 * 60 % of the free memory, largest first.  Each handle's phase times are
 * those of its group; the launch and byte counts of a group are reported
 * with its first matrix.  Errors: on any status other than HSS_OK /
 * HSS_ERR_NOT_CONVERGED every handle is freed, out[] is all NULL and the
 * status is returned (its message in hss_last_error);
 * HSS_ERR_NOT_CONVERGED when some matrix did not converge (all handles
 * valid, as for hss_compress). */
hss_status hss_compress_batched(const hss_source* A, const hss_opts* opts, int count, void* stream,
                                hss_matrix* out);

/* Y = H X (transpose = 0) or Y = H^T X (transpose = 1) for a compressed
 * handle: the O(r n) product of section 2.1 (up-sweep
 * x^_tau = V_tau^T [...], sibling coupling with B12 / B21, down-sweep with
 * U_tau, leaves D_tau); H^T exchanges the roles of U and V, takes D^T and
 * couples with B21^T, B12^T.  A partial result (HSS_ERR_NOT_CONVERGED)
 * couples the children of its uncompressed nodes through the dense blocks
 * it kept.  X, Y: device col-major n x nrhs (ldx, ldy >= n); Y is
 * overwritten.  Asynchronous on the stream. */
hss_status hss_matvec(hss_matrix H, int nrhs, const double* X, long long ldx,
                      double* Y, long long ldy, int transpose, void* stream);

/* Entries of a compressed handle, out(r, c) = H(I[r], J[c]) — the element
 * extraction of section 3.1 applied to an HSS matrix, so that a matrix built
 * from compressed ones (a sum, or a product through hss_matvec) can itself be
 * compressed through a user operator and an extraction source.  For i and j
 * in one leaf the entry is D(i, j); otherwise u_a(i) B v_b(j)^T with a, b the
 * children of the lowest common ancestor holding i and j, u_a(i) the row of
 * the nested basis U_a (eq. nestedUV: a leaf's U = Pi [I; X^T], each level
 * up times the node's own basis) and v_b(j) that of V_b; the dense blocks of
 * a partial result where they apply.  Cost: for each row index the products
 * along its path to the root (sum over its ancestors of k^2), and k per
 * entry.  I (nr), J (nc): device int arrays of indices in [0, n); out: device
 * col-major nr x nc, ld ldo >= nr.  Uses a temporary device buffer; returns
 * after a sync of the stream; HSS_ERR_ARG (entries left zero) when an index
 * is out of range. */
hss_status hss_get_entries(hss_matrix H, int nr, const int* I, int nc, const int* J, double* out,
                           long long ldo, void* stream);

/* The dense matrix H (eq. nestedUV expanded): out (device, col-major n x n,
 * ld >= n) = H applied to identity column blocks of up to 2048 columns with
 * hss_matvec (a temporary n x 2048 device buffer).  For tests and moderate
 * n; returns after a sync of the stream. */
hss_status hss_to_dense(hss_matrix H, double* out, long long ld, void* stream);

hss_status hss_get_stats(hss_matrix H, hss_stats* s);                 /* host */
hss_status hss_get_node(hss_matrix H, int node, hss_node_info* info); /* host */

/* Host copies of one node's generators (any pointer may be NULL):
 * Jr[kr], Jc[kc]  skeleton rows of tau.S^r / tau.S^c, local to the sample
 *                 (pivot order; U(Jr, :) = I);
 * Pr[mr], Pc[mc]  full pivot order (first kr / kc entries are Jr / Jc);
 * Xr (kr x (mr-kr)), Xc (kc x (mc-kc))  col-major R1^{-1} R2, so that
 *                 U = Pi [I; Xr^T] (eq. ID);
 * Ir[kr], Ic[kc]  global skeleton indices tau.I^r, tau.I^c;
 * D (size x size, leaves), B12 (kr(nu1) x kc(nu2)), B21 (kr(nu2) x kc(nu1))
 *                 col-major, non-leaves. */
hss_status hss_export_node(hss_matrix H, int node, int* Jr, int* Jc, int* Pr, int* Pc,
                           double* Xr, double* Xc, int* Ir, int* Ic, double* D,
                           double* B12, double* B21);

void hss_free(hss_matrix H);

/* Launch-shape parameters, process-wide.  The defaults are the built-in
 * heuristics; the package's tuning script times the candidates on the GPU at
 * hand and records the fastest in a table that the Python binding applies
 * when it loads the library.  They change launch shapes only: any choice
 * gives the same method, with rounding differences only. */
typedef struct hss_tuning {
  int qrcp_wide_max_sides;    /* QRCP launches over at most this many node
                                 sides use 256 threads and two CTAs per SM,
                                 larger ones 128 threads and four (default 8) */
  int sample_waves_packed;    /* K split of the packed tensor-core sampling
                                 kernel: CTAs for this many waves of the SMs
                                 (default 4; at least 64 k-tiles per CTA)      */
  int sample_waves_generated; /* the same for the generated-entry kernel
                                 (default 2)                                   */
  int qrcp_min_cols;          /* a node side's QRCP group takes extra CTAs
                                 (beyond one per 256 columns) only while each
                                 keeps at least this many columns (default 4) */
  int qrcp_sm_ctas;           /* CTAs per SM of the QRCP group launches: 1
                                 (512 threads), 2 (256) or 4 (128); 0 = by
                                 qrcp_wide_max_sides (default 0)              */
} hss_tuning;
hss_status hss_set_tuning(const hss_tuning* t);   /* NULL: back to the defaults;
                                                     HSS_ERR_ARG on values < 1
                                                     (qrcp_sm_ctas: not 0, 1, 2
                                                     or 4)                    */
hss_status hss_get_tuning(hss_tuning* t);

/* Checkpoint of a compressed handle (no counterpart in the paper, which
 * keeps its compression in memory; its warm restart of Algorithm 3 is
 * in-process).  hss_save writes to the host file `path` the tree, node
 * states and ranks, statistics and every generator (D, U and V as pivots and
 * X, skeleton indices, B12, B21) in a plain binary format (8-byte magic
 * "HSSGEN01", native byte order); the handle must have converged
 * (HSS_ERR_ARG otherwise).  The file is written as `path`.tmp and renamed to
 * `path` once complete; on failure the temporary file is removed and
 * nothing is left at `path` (HSS_ERR_IO for a failed open, write, close or
 * rename, HSS_ERR_CUDA for a failed copy of the generators to the host).
 * hss_load reads such a file into a new handle on the current device,
 * serving hss_matvec, hss_to_dense, hss_get_node, hss_export_node and
 * hss_get_stats like the original; it cannot resume a compression (the
 * samples are not saved).  Every count, index and pivot is checked on the
 * host before anything is uploaded: the tree must be the halving tree of
 * the saved n and leaf size, every array exactly as long as the ranks
 * imply, the pivots of a node a permutation of its sample rows and its
 * skeleton indices inside its index range.  HSS_ERR_IO when the file cannot
 * be opened, HSS_ERR_ARG when it is not such a checkpoint, is truncated or
 * fails a check; *out is NULL then. */
hss_status hss_save(hss_matrix H, const char* path);
hss_status hss_load(const char* path, hss_matrix* out);

/* hss_free (and a failed compression) keep the handle's device memory in
 * 256 MB chunks, up to 32 GB per device, for the next compression on the same
 * device (after waiting for the device, as cudaFree would).  The work buffers
 * of a call (packed operands, job lists, temporaries) come stream-ordered
 * from a memory pool of the library's own per context, which keeps freed
 * memory reserved, at most the largest set of work buffers one call held at
 * once (the device's default pool is not touched).
 * This call returns the chunks cached for the current device with cudaFree
 * and, after waiting for the device, trims that pool to nothing. */
hss_status hss_release_cached(void);
const char* hss_status_str(hss_status s);
const char* hss_last_error(void);

/* Recursive coordinate bisection of a host point set (col-major n x dim,
 * ld >= n): at each node of size m > leaf, sort by the coordinate of largest
 * extent, ties by original index, and split into floor(m/2) + ceil(m/2).
 * perm (host, n): perm[new] = old.  The halving tree of the permuted points
 * is the cluster tree (paper section 3: binary, possibly imbalanced). */
hss_status hss_rcb_order(const double* points, int n, int dim, long long ld, int leaf,
                         int* perm);

/* Gaussian random matrix R(:, col0:col0+ncols) (Table "helper functions",
 * randn): Philox4x32-10 keyed by seed, counter (i >> 1, column, 0, 0), two
 * 53-bit uniforms, Box-Muller; row i takes the cosine (even i) or sine (odd
 * i) branch.  round_mode 0: FP64; 1: rounded to an 11-bit significand
 * (TF32); 2: rounded to an 8-bit significand (BF16).  R: device col-major,
 * column col0 at R (ld >= n).  Asynchronous. */
hss_status hss_random_normal(unsigned long long seed, int n, int col0, int ncols,
                             double* R, long long ldr, int round_mode, void* stream);

/* The sampling step with the leaf diagonal blocks removed, eq.
 * sample_off_diag at the leaf level:  Sr = (A - D^(L)) R,
 * Sc = (A - D^(L))^T R, where D^(L) = blockdiag of the leaves of the halving
 * tree with the given leaf size.  R: device col-major n x ncols (ldr);
 * Sr, Sc: device row-major n x ncols (row stride lds >= ncols); either may
 * be NULL to skip it.  precision: HSS_PREC_*.  Asynchronous. */
hss_status hss_sample_offdiag(const hss_source* A, int leaf, int precision, int ncols,
                              const double* R, long long ldr, double* Sr, double* Sc,
                              long long lds, void* stream);

/* The same computation as hss_sample_offdiag in its FP64 form (same
 * arguments, same results; precision must be HSS_PREC_FP64 — the mixed
 * forms stage their split operands in temporary buffers, so they return
 * HSS_ERR_UNSUPPORTED here), for callers that cannot let a library allocate
 * device memory:
 * a serving process or framework that owns the whole device-memory budget
 * through its own pool, or a caller that cannot accept the synchronisation
 * or the possible failure of cudaMalloc / cudaMallocAsync in the middle of
 * a run.  It allocates nothing: the per-index leaf table the kernel needs
 * lives in a fixed device array inside the library (4 MiB, held on every
 * GPU that loads the library until the process exits), so n may not
 * exceed 2^20 (larger n returns HSS_ERR_ARG without launching anything).
 * The first call in a CUDA context looks up that array's device address (a
 * one-time set-up per context, which may load the library's device code);
 * make that first call before any stream capture.  A context destroyed and
 * created again (cudaDeviceReset) gets the set-up anew.  All calls share the array and overwrite the first n entries:
 * calls that overlap on the GPU (on different streams, or from different
 * host threads) race on it and must be serialised by the caller.  The
 * paper has no counterpart to this entry point.  Asynchronous. */
hss_status hss_sample_offdiag_noalloc(const hss_source* A, int leaf, int precision, int ncols,
                                      const double* R, long long ldr, double* Sr, double* Sc,
                                      long long lds, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HSS_H */
