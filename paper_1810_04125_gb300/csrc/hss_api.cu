// Host driver and C ABI of the HSS library (include/hss.h).
//
// hss_compress runs Algorithm 3 (HSSCompressAdaptive): sample, then sweep
// the cluster tree bottom-up one level at a time, and grow the sample until
// the root is COMPRESSED.  Every step of a level is one batched launch over
// all nodes of that level (extraction, upward merge, strategy test, ID,
// reduction); the host reads back the ranks and test flags once per level
// (twice for Incrementing) to update the node states of Algorithm 3 and to
// size the next level's buffers.  All arithmetic runs in the kernels.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <queue>
#include <vector>

#include <cuda.h>

#include "hss_internal.h"

#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <mutex>
#include <thread>

using namespace hss;

namespace {

thread_local std::string g_err;

hss_status fail(hss_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define CK(x)                                                                                   \
  do {                                                                                          \
    cudaError_t e_ = (x);                                                                       \
    if (e_ != cudaSuccess)                                                                      \
      return fail(HSS_ERR_CUDA, "%s failed: %s (%s:%d)", #x, cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                                    \
  } while (0)
#define CKS(x)                      \
  do {                              \
    hss_status s_ = (x);            \
    if (s_ != HSS_OK) return s_;    \
  } while (0)

// Chunked bump allocator for memory that lives as long as the handle.
// Arena chunks of the standard size outlive their handle in a per-process
// cache (up to kCacheCap bytes per device) and serve the next compression:
// cudaMalloc and cudaFree of 256 MB chunks cost milliseconds each, and a
// compression takes several.  A handle's release waits for the device first,
// as cudaFree would, so no work still reading a chunk sees it reused.
constexpr size_t kChunk = size_t(256) << 20;
constexpr size_t kCacheCap = size_t(32) << 30;
struct ChunkCache {
  std::mutex mu;
  std::vector<std::pair<int, void*>> free;   // (device, chunk of kChunk bytes)
  size_t held[64] = {0};
};
ChunkCache& chunk_cache() {
  static ChunkCache c;
  return c;
}

typedef CUresult (*ctx_get_current_fn)(CUcontext*);
typedef CUresult (*ctx_get_id_fn)(CUcontext, unsigned long long*);

// Id of the current context (driver entry points looked up through the
// runtime, so the library does not link the driver library itself); false
// when there is no current context yet or the lookup is unavailable.
bool current_context_id(unsigned long long* id) {
  static ctx_get_current_fn get_current = nullptr;
  static ctx_get_id_fn get_id = nullptr;
  if (!get_current || !get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return false;
    get_current = (ctx_get_current_fn)f1;
    get_id = (ctx_get_id_fn)f2;
  }
  CUcontext ctx = nullptr;
  return get_current(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, id) == CUDA_SUCCESS;
}

// Stream-ordered buffers (packed operands, job lists, temporaries) come from
// a memory pool of the library's own, one per context, that keeps the freed
// memory reserved (at most the largest set of buffers one call held at
// once).  The device's default pool returns freed memory to the system at
// every synchronisation, and mapping it again cost milliseconds per
// allocation (a batch of 64 matrices spent 29 % of its time there); the
// default pool's own setting is left alone for the other users of it in the
// process.  hss_release_cached trims the pool.
struct PoolCache {
  std::mutex mu;
  std::vector<std::pair<unsigned long long, cudaMemPool_t>> pools;   // (context id, pool)
};
PoolCache& pool_cache() {
  static PoolCache c;
  return c;
}

cudaError_t lib_pool(cudaMemPool_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  unsigned long long id = 0;
  if (!current_context_id(&id)) {
    cudaFree(nullptr);   // makes the device's primary context current
    if (!current_context_id(&id)) return cudaDeviceGetDefaultMemPool(out, dev);
  }
  PoolCache& c = pool_cache();
  std::lock_guard<std::mutex> lock(c.mu);
  for (auto& q : c.pools)
    if (q.first == id) {
      *out = q.second;
      return cudaSuccess;
    }
  cudaMemPoolProps pp;
  memset(&pp, 0, sizeof pp);
  pp.allocType = cudaMemAllocationTypePinned;
  pp.handleTypes = cudaMemHandleTypeNone;
  pp.location.type = cudaMemLocationTypeDevice;
  pp.location.id = dev;
  cudaMemPool_t pool = nullptr;
  e = cudaMemPoolCreate(&pool, &pp);
  if (e != cudaSuccess) return e;
  unsigned long long keep = ~0ull;
  e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  if (e != cudaSuccess) {
    cudaMemPoolDestroy(pool);
    return e;
  }
  c.pools.push_back({id, pool});
  *out = pool;
  return cudaSuccess;
}

template <class T>
cudaError_t dmalloc_async(T** p, size_t bytes, cudaStream_t st) {
  cudaMemPool_t pool = nullptr;
  cudaError_t e = lib_pool(&pool);
  if (e != cudaSuccess) return e;
  return cudaMallocFromPoolAsync((void**)p, bytes, pool, st);
}

struct Arena {
  std::vector<std::pair<void*, size_t>> chunks;
  char* cur = nullptr;
  size_t left = 0;
  void* alloc(size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    if (bytes > left) {
      const size_t sz = std::max(kChunk, bytes);
      void* p = nullptr;
      int dev = 0;
      if (sz == kChunk && cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) {
        ChunkCache& c = chunk_cache();
        std::lock_guard<std::mutex> lock(c.mu);
        for (size_t i = 0; i < c.free.size(); ++i)
          if (c.free[i].first == dev) {
            p = c.free[i].second;
            c.free.erase(c.free.begin() + i);
            c.held[dev] -= kChunk;
            break;
          }
      }
      if (!p && cudaMalloc(&p, sz) != cudaSuccess) return nullptr;
      chunks.push_back({p, sz});
      cur = (char*)p;
      left = sz;
    }
    void* r = cur;
    cur += bytes;
    left -= bytes;
    return r;
  }
  void release() {
    int dev = -1;
    if (!chunks.empty() && (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)) dev = -1;
    ChunkCache& c = chunk_cache();
    for (auto& ch : chunks) {
      bool kept = false;
      if (ch.second == kChunk && dev >= 0 && dev < 64) {
        std::lock_guard<std::mutex> lock(c.mu);
        if (c.held[dev] + kChunk <= kCacheCap) {
          c.free.push_back({dev, ch.first});
          c.held[dev] += kChunk;
          kept = true;
        }
      }
      if (!kept) cudaFree(ch.first);
    }
    chunks.clear();
    cur = nullptr;
    left = 0;
  }
};

// Growable per-phase scratch (reset before each phase; growing waits for
// the stream, which is idle at these points anyway).
struct Scratch {
  char* base = nullptr;
  size_t cap = 0, used = 0;
  std::vector<size_t> plan;
  void reset() { used = 0; overflow = false; }
  static size_t rnd(size_t b) { return (b + 255) & ~size_t(255); }
  cudaError_t ensure(size_t bytes, cudaStream_t st) {
    if (bytes <= cap) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    if (base) cudaFree(base);
    base = nullptr;
    cap = 0;
    size_t sz = std::max(bytes + bytes / 4, size_t(1) << 20);
    e = cudaMalloc(&base, sz);
    if (e != cudaSuccess) return e;
    cap = sz;
    return cudaSuccess;
  }
  bool overflow = false;   // a take() beyond the capacity (a sizing bug); checked by callers
  void* take(size_t bytes) {
    if (used + rnd(bytes) > cap) {
      overflow = true;
      return base;
    }
    void* r = base + used;
    used += rnd(bytes);
    return r;
  }
  void release() {
    if (base) cudaFree(base);
    base = nullptr;
    cap = used = 0;
  }
};

struct Side {
  double* S = nullptr;   // local sample, m x dmax row-major
  int m = 0, k = 0;
  int* piv = nullptr;    // m
  double* X = nullptr;   // k x (m-k) col-major, ld max(k,1)
  int* I = nullptr;      // k global skeleton indices
  double* Q = nullptr;   // Incrementing basis, m x dmax row-major
  int q = 0, tested = 0;
  double rho = -1.0;
  bool done = false;
  // per-level staging
  int qr_k = 0, qr_acc = 0;
};

struct Node {
  int lo, size, level, parent, ch[2];
  bool leaf;
  int state = HSS_UNTOUCHED;
  Side r, c;
  double* Rr = nullptr;  // tau.R^r = V^T R(I_tau): c.k x dmax row-major
  double* Rc = nullptr;  // tau.R^c = U^T R(I_tau): r.k x dmax row-major
  double* D = nullptr;   // leaf: size x size col-major
  double* B12 = nullptr; // kr(nu1) x kc(nu2) col-major, ld max(kr(nu1),1)
  double* B21 = nullptr; // kr(nu2) x kc(nu1) col-major, ld max(kr(nu2),1)
  // a node that is not COMPRESSED when the compression stops at d_max: the
  // blocks A(I_nu1, I_nu2) (|nu1| x |nu2|) and A(I_nu2, I_nu1), col-major
  double* F12 = nullptr;
  double* F21 = nullptr;
};

// Phase boundaries: CUDA events on the stream (the per-phase times of the
// statistics) and one NVTX range per phase on the calling host thread (the
// phases on a profiler's timeline; no cost without a tool attached).
struct PhaseTimer {
  std::vector<cudaEvent_t> ev;
  std::vector<int> ph;
  bool range_open = false;
  cudaError_t mark(int phase, cudaStream_t st) {
    static const char* const names[] = {"hss sample", "hss id", "hss test", "hss merge", "hss other", "hss rng"};
    if (range_open) nvtxRangePop();
    nvtxRangePushA(phase >= 0 && phase < 6 ? names[phase] : "hss");
    range_open = true;
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    ev.push_back(e);
    ph.push_back(phase);
    return cudaEventRecord(e, st);
  }
  // out[phase] = summed time of the phase; out[PH_N - 1] = total
  void sum(double* out, int nph) {
    for (int i = 0; i < nph; ++i) out[i] = 0.0;
    for (size_t i = 0; i + 1 < ev.size(); ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) == cudaSuccess) {
        out[ph[i]] += ms;
        out[nph - 1] += ms;
      }
    }
  }
  void close_range() {
    if (range_open) nvtxRangePop();
    range_open = false;
  }
  void clear() {
    for (auto e : ev) cudaEventDestroy(e);
    ev.clear();
    ph.clear();
  }
};
enum { PH_SAMPLE = 0, PH_ID = 1, PH_TEST = 2, PH_MERGE = 3, PH_OTHER = 4, PH_RNG = 5, PH_N = 7 };

}  // namespace

struct hss_matrix_s {
  int n = 0, dmax = 0, device = 0;
  hss_opts o{};
  hss_source src{};
  std::vector<Node> nodes;
  std::vector<std::vector<int>> by_level;
  int max_level = 0;
  std::vector<int> bounds;   // sample widths after each growth (Incrementing blocks)
  Arena arena;
  double* R = nullptr;     // n x dmax col-major (ld n)
  double* Sg_r = nullptr;  // n x dmax row-major: leaf samples
  double* Sg_c = nullptr;
  int* leaf_id = nullptr;
  int* leaf_lo = nullptr;  // nleaves + 1 row bounds (with a user operator)
  long long* leaf_doff = nullptr; // offset of each leaf's D in the packed leaf blocks (user operator)
  double* leaf_D = nullptr;       // the leaf blocks D, packed (user operator)
  int* iota = nullptr;
  int d_final = 0, n_adapt = 0, converged = 0;
  int pack_decided = -1;   // mixed forms, generated A: packed tiles (1) or not (0)
  bool sym = false;        // symmetric option: the column side mirrors the row side
  void* packA = nullptr;   // packed tensor-core tiles of a dense A (during compress)
  void* toep_terms = nullptr; // a Toeplitz source's diagonals split into terms (during compress)
  bool usable = false;
  bool partial = false;    // not converged; the uncompressed part kept dense (F12, F21)
  hss_stats st{};
  // progress of the compression (Algorithm 3's outer loop)
  int d = 0, d_prev = 0, slot = 0;
  bool own_R = true, done = false;
  ~hss_matrix_s() {
    if (packA) cudaFree(packA);
    if (toep_terms) cudaFree(toep_terms);
    arena.release();
  }
};

namespace {

// A device buffer reused launch after launch on one stream: a job list
// uploaded for the next launch is copied after the previous launch has
// finished reading it (stream order), so no allocation per launch.
struct DevBuf {
  char* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes, cudaStream_t st) {
    if (bytes <= cap) return cudaSuccess;
    if (p) {
      cudaError_t e = cudaFreeAsync(p, st);
      if (e != cudaSuccess) return e;
    }
    p = nullptr;
    cap = 0;
    const size_t sz = std::max(bytes + bytes / 2, size_t(1) << 20);
    cudaError_t e = dmalloc_async((void**)&p, sz, st);
    if (e != cudaSuccess) return e;
    cap = sz;
    return cudaSuccess;
  }
  void release(cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
    p = nullptr;
    cap = 0;
  }
};

// What the matrices of one compression call share (one matrix for
// hss_compress, all of them for hss_compress_batched): the stream, per-phase
// scratch, the job-list buffer, the device flags and the pinned read-back
// buffer, the phase timer and the counters.
//   d_flag[0..7]: [1] tensor-core sampling wait, [2] QRCP barrier,
//   [3] tensor-core tile product wait, [4] Incrementing test barrier;
//   d_flag[8 + i]: non-finite samples of matrix i.
struct Ctx {
  cudaStream_t st = nullptr;
  Scratch scratch;
  DevBuf jobs;
  DevBuf gpack;   // operands of the tensor-core tile products split into their terms
  int* d_flag = nullptr;
  int nflag = 0;
  int* h_pinned = nullptr;
  size_t h_pinned_cap = 0;
  PhaseTimer timer;
  long long launches = 0, sample_launches = 0, bytes_h2d = 0, bytes_d2h = 0;
  bool trace = false;      // HSS_TRACE=1: one stderr line per launch of the batched phases
  cudaEvent_t trace_ev[2] = {nullptr, nullptr};
  int qrcp_cap = -1, qrcp_cap_d = -1, qrcp_cap_w = -1, qrcp_nsm = 0, qrcp_per = 0;
  explicit Ctx(cudaStream_t s) : st(s) {
    const char* tr = getenv("HSS_TRACE");
    trace = tr && tr[0] == '1';
    if (trace && (cudaEventCreate(&trace_ev[0]) != cudaSuccess || cudaEventCreate(&trace_ev[1]) != cudaSuccess))
      trace = false;
  }
  ~Ctx() {
    timer.close_range();
    timer.clear();
    for (auto& e : trace_ev)
      if (e) cudaEventDestroy(e);
    jobs.release(st);
    gpack.release(st);
    if (d_flag) cudaFreeAsync(d_flag, st);
    scratch.release();
    if (h_pinned) cudaFreeHost(h_pinned);
  }
  hss_status flags(int nmat) {
    nflag = 8 + std::max(nmat, 0);
    CK(dmalloc_async((void**)&d_flag, sizeof(int) * nflag, st));
    CK(cudaMemsetAsync(d_flag, 0, sizeof(int) * nflag, st));
    return HSS_OK;
  }
};

SrcDev make_src(const hss_source& s, const int* leaf_id) {
  SrcDev d;
  d.kind = s.kind;
  d.n = s.n;
  d.dim = s.dim;
  d.pad = 0;
  d.a = s.a;
  d.b = s.b ? s.b : s.a;
  d.ld = s.ld;
  d.p0 = s.p0;
  d.p1 = s.p1;
  d.leaf_id = leaf_id;
  return d;
}

hss_status check_source(const hss_source* A) {
  if (!A) return fail(HSS_ERR_ARG, "source is NULL");
  if (A->n <= 0) return fail(HSS_ERR_ARG, "n must be positive (got %d)", A->n);
  if (A->kind == HSS_SRC_EXTRACT) {
    if (!A->extract) return fail(HSS_ERR_ARG, "an extraction source needs its extract routine");
    return HSS_OK;
  }
  if (!A->a) return fail(HSS_ERR_ARG, "source data pointer is NULL");
  switch (A->kind) {
    case HSS_SRC_DENSE:
      if (A->ld < A->n) return fail(HSS_ERR_ARG, "dense ld %lld < n %d", A->ld, A->n);
      break;
    case HSS_SRC_TOEPLITZ:
      break;
    case HSS_SRC_GAUSS:
      if (A->dim <= 0 || A->ld < A->n) return fail(HSS_ERR_ARG, "points need dim > 0 and ld >= n");
      if (!(A->p0 > 0.0)) return fail(HSS_ERR_ARG, "Gaussian bandwidth p0 must be > 0");
      break;
    case HSS_SRC_LAPLACE:
      if (A->dim != 3 || A->ld < A->n) return fail(HSS_ERR_ARG, "Laplace points need dim == 3, ld >= n");
      break;
    default:
      return fail(HSS_ERR_ARG, "unknown source kind %d", A->kind);
  }
  return HSS_OK;
}

// Halving tree in level order (node 0 = root).
void build_tree(int n, int leaf, std::vector<Node>& nodes) {
  nodes.clear();
  Node root{};
  root.lo = 0; root.size = n; root.level = 0; root.parent = -1; root.ch[0] = root.ch[1] = -1;
  nodes.push_back(root);
  for (size_t i = 0; i < nodes.size(); ++i) {
    if (nodes[i].size > leaf) {
      int h = nodes[i].size / 2;
      Node a{}, b{};
      a.lo = nodes[i].lo; a.size = h;
      b.lo = nodes[i].lo + h; b.size = nodes[i].size - h;
      a.level = b.level = nodes[i].level + 1;
      a.parent = b.parent = (int)i;
      a.ch[0] = a.ch[1] = b.ch[0] = b.ch[1] = -1;
      nodes[i].ch[0] = (int)nodes.size();
      nodes.push_back(a);
      nodes[i].ch[1] = (int)nodes.size();
      nodes.push_back(b);
    }
  }
  for (auto& t : nodes) t.leaf = t.ch[0] < 0;
}

hss_status upload(Ctx& c, void* dst, const void* src, size_t bytes) {
  if (bytes == 0) return HSS_OK;
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c.st));
  c.bytes_h2d += (long long)bytes;
  return HSS_OK;
}

hss_status readback(Ctx& c, const void* src, size_t bytes) {
  if (bytes > c.h_pinned_cap) {
    if (c.h_pinned) cudaFreeHost(c.h_pinned);
    c.h_pinned = nullptr;
    c.h_pinned_cap = 0;
    size_t sz = std::max(bytes, size_t(1) << 16);
    CK(cudaMallocHost((void**)&c.h_pinned, sz));
    c.h_pinned_cap = sz;
  }
  if (bytes) CK(cudaMemcpyAsync(c.h_pinned, src, bytes, cudaMemcpyDeviceToHost, c.st));
  c.bytes_d2h += (long long)bytes;
  CK(cudaStreamSynchronize(c.st));
  return HSS_OK;
}

// Several device ranges copied into the pinned buffer back to back with one
// synchronisation; returns the host offset of each range (8-byte aligned).
hss_status readback_many(Ctx& c, const std::vector<std::pair<const void*, size_t>>& items, std::vector<size_t>& off) {
  off.clear();
  size_t tot = 0;
  for (auto& it : items) {
    off.push_back(tot);
    tot += (it.second + 7) & ~size_t(7);
  }
  if (tot > c.h_pinned_cap) {
    if (c.h_pinned) cudaFreeHost(c.h_pinned);
    c.h_pinned = nullptr;
    c.h_pinned_cap = 0;
    size_t sz = std::max(tot, size_t(1) << 16);
    CK(cudaMallocHost((void**)&c.h_pinned, sz));
    c.h_pinned_cap = sz;
  }
  for (size_t i = 0; i < items.size(); ++i)
    if (items[i].second)
      CK(cudaMemcpyAsync((char*)c.h_pinned + off[i], items[i].first, items[i].second, cudaMemcpyDeviceToHost, c.st));
  c.bytes_d2h += (long long)tot;
  CK(cudaStreamSynchronize(c.st));
  return HSS_OK;
}

// The job lists of one launch, packed into the reused device buffer.
struct Staging {
  std::vector<char> host;
  size_t put(const void* p, size_t bytes) {
    const size_t off = Scratch::rnd(host.size());
    host.resize(off + bytes);
    if (bytes) memcpy(host.data() + off, p, bytes);
    return off;
  }
  hss_status send(Ctx& c, char** dev) {
    CK(c.jobs.ensure(std::max<size_t>(host.size(), 256), c.st));
    *dev = c.jobs.p;
    return upload(c, c.jobs.p, host.data(), host.size());
  }
};

Opnd opnd(const double* p, long long rs, long long cs, const int* rows = nullptr,
          const double* p2 = nullptr, int split = 0x7fffffff) {
  Opnd o;
  o.p = p; o.p2 = p2 ? p2 : p; o.rs = rs; o.cs = cs; o.rows = rows; o.split = split;
  return o;
}

GemmJob gemm_job() {
  GemmJob j;
  memset(&j, 0, sizeof j);
  j.A = opnd(nullptr, 0, 0);
  j.B = opnd(nullptr, 0, 0);
  j.C0 = opnd(nullptr, 0, 0);
  j.c_split = 0x7fffffff;
  j.alpha = 1.0;
  return j;
}

// Runs a list of tile-product jobs (one launch).  tc_prec: HSS_PREC_FP64 for
// the FP64 tile kernel; a mixed precision sends the products that only form
// samples (merge, reduce, test projections) to the tensor-core kernel.
hss_status run_gemms(Ctx& c, const std::vector<GemmJob>& jobs, const char* tag = "gemm",
                     int tc_prec = HSS_PREC_FP64) {
  const bool tc = tc_prec != HSS_PREC_FP64;
  int max_n = 0;
  for (const GemmJob& j : jobs) max_n = std::max(max_n, j.N);
  const int tm = tc ? 128 : 64, tn = tc ? gemm_tc_tile_n(max_n) : 64;
  std::vector<GemmTile> tiles;
  double flop = 0.0;
  long long ntile = 0;
  for (const GemmJob& j : jobs)
    if (j.M > 0 && j.N > 0) ntile += (long long)((j.M + tm - 1) / tm) * ((j.N + tn - 1) / tn);
  for (size_t i = 0; i < jobs.size(); ++i) {
    const GemmJob& j = jobs[i];
    if (j.M <= 0 || j.N <= 0) continue;
    flop += 2.0 * j.M * j.N * j.K;
    // FP64 tiles with a long K on a launch of few tiles: split K so that the
    // launch fills the SMs (partials added atomically; C zeroed first when
    // the job overwrites it)
    int ks = 1;
    const bool contiguous_c = !j.c_rows && j.c_split == 0x7fffffff &&
                              ((j.c_rs == 1 && j.c_cs == j.M) || (j.c_cs == 1 && j.c_rs == j.N));
    if (!tc && j.K >= 512 && j.beta == 0.0 && (j.gamma == 1.0 || (j.gamma == 0.0 && contiguous_c)) &&
        ntile < 2 * 152) {
      ks = (int)std::min<long long>((2 * 152 + ntile - 1) / ntile, j.K / 256);
      ks = std::max(ks, 1);
      if (ks > 1 && j.gamma == 0.0) CK(cudaMemsetAsync(j.C, 0, sizeof(double) * (size_t)j.M * j.N, c.st));
    }
    for (int ti = 0; ti < (j.M + tm - 1) / tm; ++ti)
      for (int tj = 0; tj < (j.N + tn - 1) / tn; ++tj)
        for (int z = 0; z < ks; ++z) {
          // K shares in multiples of the 16-wide k step
          const int kb = (int)((long long)j.K * z / ks) / 16 * 16;
          const int ke = z + 1 == ks ? j.K : (int)((long long)j.K * (z + 1) / ks) / 16 * 16;
          tiles.push_back({(int)i, ti, tj, kb, ke});
        }
  }
  if (tiles.empty()) return HSS_OK;
  if (c.trace) CK(cudaEventRecord(c.trace_ev[0], c.st));
  // tensor-core form: every operand split once into its TF32 terms (tiles
  // in a context buffer reused in stream order) when the jobs are large
  // (on average 2^18 operand elements or more: below that the extra launch
  // and the packed copy cost more than the repeated splitting saves,
  // measured on the batch of 64 matrices) and the tiles take at most 4 GB;
  // else the kernel that splits while it stages
  std::vector<GemmJob> pj;
  std::vector<PackUnit> units;
  bool packed = false;
  if (tc) {
    pj = jobs;
    const size_t ab = gemm_tc_tile_bytes(0, tn), bb = gemm_tc_tile_bytes(1, tn);
    size_t total = 0;
    double elems = 0.0;
    int njob = 0;
    std::vector<size_t> oa(jobs.size(), 0), ob(jobs.size(), 0);
    for (size_t i = 0; i < jobs.size(); ++i) {
      const GemmJob& j = jobs[i];
      if (j.M <= 0 || j.N <= 0 || j.K <= 0) continue;
      const size_t nkt = (j.K + 31) / 32, nrb = (j.M + tm - 1) / tm, ncb = (j.N + tn - 1) / tn;
      oa[i] = total;
      total += nrb * nkt * ab;
      ob[i] = total;
      total += ncb * nkt * bb;
      elems += (double)j.K * ((double)j.M + (double)j.N);
      njob++;
    }
    packed = total > 0 && total <= (size_t(4) << 30) && elems >= 262144.0 * njob;
    if (packed) {
      CK(c.gpack.ensure(total, c.st));
      for (size_t i = 0; i < jobs.size(); ++i) {
        GemmJob& j = pj[i];
        if (j.M <= 0 || j.N <= 0 || j.K <= 0) continue;
        const int nkt = (j.K + 31) / 32, nrb = (j.M + tm - 1) / tm, ncb = (j.N + tn - 1) / tn;
        j.pa = (unsigned char*)c.gpack.p + oa[i];
        j.pb = (unsigned char*)c.gpack.p + ob[i];
        j.nkt = nkt;
        for (int t = 0; t < nrb; ++t)
          for (int kt = 0; kt < nkt; ++kt) units.push_back({(int)i, 0, t, kt});
        for (int t = 0; t < ncb; ++t)
          for (int kt = 0; kt < nkt; ++kt) units.push_back({(int)i, 1, t, kt});
      }
    }
  }
  Staging sg;
  const size_t oj = sg.put(packed ? pj.data() : jobs.data(), jobs.size() * sizeof(GemmJob));
  const size_t ot = sg.put(tiles.data(), tiles.size() * sizeof(GemmTile));
  const size_t ou = packed ? sg.put(units.data(), units.size() * sizeof(PackUnit)) : 0;
  char* dev;
  CKS(sg.send(c, &dev));
  if (packed) {
    CK(launch_gemm_tc_pack((const GemmJob*)(dev + oj), (const PackUnit*)(dev + ou), (int)units.size(), tn, c.st));
    CK(launch_gemm_tc_packed((const GemmJob*)(dev + oj), (const GemmTile*)(dev + ot), (int)tiles.size(), tn,
                             c.d_flag + 3, c.st));
    c.launches += 2;
  } else if (tc) {
    CK(launch_gemm_tc((const GemmJob*)(dev + oj), (const GemmTile*)(dev + ot), (int)tiles.size(), tn,
                      c.d_flag + 3, c.st));
    c.launches++;
  } else {
    CK(launch_gemm((const GemmJob*)(dev + oj), (const GemmTile*)(dev + ot), (int)tiles.size(), c.st));
    c.launches++;
  }
  if (c.trace) {
    CK(cudaEventRecord(c.trace_ev[1], c.st));
    CK(cudaEventSynchronize(c.trace_ev[1]));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c.trace_ev[0], c.trace_ev[1]);
    fprintf(stderr, "[hss trace] %s jobs %zu tiles %zu  %.3f ms  %.1f GFLOP/s\n", tag, jobs.size(), tiles.size(), ms,
            flop / (ms * 1e6));
  }
  return HSS_OK;
}

// One launch over the jobs of every precision present: the FP64 products and
// the products of each mixed form (tensor cores) separately.
struct GemmSet {
  std::vector<GemmJob> by_prec[3];
  void add(int prec, const GemmJob& j) { by_prec[prec < 0 || prec > 2 ? 0 : prec].push_back(j); }
  bool empty() const { return by_prec[0].empty() && by_prec[1].empty() && by_prec[2].empty(); }
};
hss_status run_gemm_set(Ctx& c, const GemmSet& g, const char* tag) {
  for (int p = 0; p < 3; ++p) CKS(run_gemms(c, g.by_prec[p], tag, p));
  return HSS_OK;
}

// Element extraction out(i, j) = A(I[i], J[j]) for lists of blocks (a tree
// level of one or several matrices): one launch of the gather / generator
// kernel for the built-in sources, one call of the caller's routine per
// matrix with an extraction source (section 3.1: all blocks of a level at
// once).
struct ExtractSet {
  std::vector<std::pair<hss_matrix_s*, std::vector<ExtractJob>>> per;
  std::vector<ExtractJob>& of(hss_matrix_s* H) {
    for (auto& e : per)
      if (e.first == H) return e.second;
    per.push_back({H, {}});
    return per.back().second;
  }
};

hss_status run_extract(Ctx& c, ExtractSet& es) {
  std::vector<ExtractJob> dev;
  int max_tiles = 1;
  for (auto& pe : es.per) {
    hss_matrix_s* H = pe.first;
    if (pe.second.empty()) continue;
    if (H->src.kind == HSS_SRC_EXTRACT) {
      std::vector<hss_block> blk;
      for (const ExtractJob& e : pe.second) {
        if (e.mi <= 0 || e.nj <= 0) continue;
        hss_block b;
        b.nr = e.mi; b.nc = e.nj;
        b.I = e.I ? e.I : H->iota + e.i0;
        b.J = e.J ? e.J : H->iota + e.j0;
        b.out = e.out; b.ldo = e.ldo;
        blk.push_back(b);
      }
      if (blk.empty()) continue;
      const int rc = H->src.extract(H->src.ctx, (int)blk.size(), blk.data(), (void*)c.st);
      if (rc != 0) return fail(HSS_ERR_OPERATOR, "user element extraction returned %d (%zu blocks)", rc, blk.size());
      continue;
    }
    const SrcDev s = make_src(H->src, H->leaf_id);
    for (ExtractJob e : pe.second) {
      if (e.mi <= 0 || e.nj <= 0) continue;
      e.src = s;
      dev.push_back(e);
      max_tiles = std::max(max_tiles, ((e.mi + 31) / 32) * ((e.nj + 31) / 32));
    }
  }
  es.per.clear();
  if (dev.empty()) return HSS_OK;
  Staging sg;
  const size_t o = sg.put(dev.data(), dev.size() * sizeof(ExtractJob));
  char* d;
  CKS(sg.send(c, &d));
  CK(launch_extract((const ExtractJob*)(d + o), (int)dev.size(), max_tiles, c.st));
  c.launches++;
  return HSS_OK;
}

hss_status run_gathers(Ctx& c, const std::vector<GatherJob>& g) {
  if (g.empty()) return HSS_OK;
  int mx = 0;
  for (const GatherJob& j : g) mx = std::max(mx, j.cnt);
  Staging sg;
  const size_t o = sg.put(g.data(), g.size() * sizeof(GatherJob));
  char* d;
  CKS(sg.send(c, &d));
  CK(launch_gather_int((const GatherJob*)(d + o), (int)g.size(), mx, c.st));
  c.launches++;
  return HSS_OK;
}

// bound of one device-side group wait: the caller's, else about 2 s
unsigned long long wait_limit(const hss_matrix_s* H) {
  return H->o.wait_limit_ns > 0 ? (unsigned long long)H->o.wait_limit_ns : 2000000000ull;
}

double tol_scale(const hss_matrix_s* H, int level) {
  return H->o.level_tol_scaling ? 1.0 / (double)level : 1.0;
}

// ---------------------------------------------------------------- sampling
// Packed operand for the mixed forms: always for a dense A; for generated
// entries when the split tiles take at most 40 % of the free device memory
// (decided once per compression).
bool use_packed(hss_matrix_s* H) {
  if (H->src.kind == HSS_SRC_DENSE) return true;
  if (H->pack_decided < 0) {
    size_t fr = 0, tot = 0;
    const size_t pb = packed_a_bytes(H->n, H->o.precision);
    H->pack_decided = (cudaMemGetInfo(&fr, &tot) == cudaSuccess && (double)pb <= 0.4 * (double)fr) ? 1 : 0;
  }
  return H->pack_decided == 1;
}

// S^r = A R, S^c = A^T R for columns [c0, c1) of matrix H, the leaf diagonal
// blocks removed (eq. sample_off_diag); the non-finite check writes the
// matrix's flag.  No read-back here: sample_check reads every matrix's flags
// at once.
hss_status sample_columns(Ctx& c, hss_matrix_s* H, int c0, int c1) {
  const int n = H->n, w = c1 - c0;
  if (w <= 0) return HSS_OK;
  cudaStream_t st = c.st;
  CK(c.timer.mark(PH_RNG, st));
  const int rm = H->o.precision == HSS_PREC_TF32X2 ? 1 : (H->o.precision == HSS_PREC_BF16X3 ? 2 : 0);
  if (H->own_R && H->o.R == nullptr) {
    CK(launch_random_normal(H->o.seed, n, c0, w, H->R + (long long)c0 * n, n, rm, st));
    c.launches++;
  } else if (H->own_R) {
    // caller's R made exactly representable in the tensor format (reading P10)
    CK(launch_round_copy(H->o.R + (long long)c0 * n, n, H->R + (long long)c0 * n, n, n, w, rm, st));
    c.launches++;
  }
  SrcDev s = make_src(H->src, H->leaf_id);
  const double* Rc = H->R + (long long)c0 * n;
  const int norient = H->sym ? 1 : 2;   // A^T R is A R for a symmetric A
  if (H->o.op) {
    // the user's product A R (and A^T R), then the leaf diagonal blocks off
    CK(c.timer.mark(PH_SAMPLE, st));
    double* T = nullptr;
    CK(dmalloc_async(&T, sizeof(double) * (size_t)n * w * norient, st));
    for (int side = 0; side < norient; ++side) {
      const int rc = H->o.op->apply(H->o.op->ctx, side, n, w, Rc, n, T + (size_t)side * n * w, n, (void*)st);
      if (rc != 0) {
        cudaFreeAsync(T, st);
        return fail(HSS_ERR_OPERATOR, "user operator returned %d (trans = %d, columns %d..%d)", rc, side, c0, c1);
      }
    }
    CK(launch_leaf_diag_sub(H->leaf_D, H->leaf_doff, H->leaf_id, H->leaf_lo, n, w, Rc, n, T, n, H->Sg_r + c0,
                            H->dmax, 0, st));
    if (!H->sym)
      CK(launch_leaf_diag_sub(H->leaf_D, H->leaf_doff, H->leaf_id, H->leaf_lo, n, w, Rc, n, T + (size_t)n * w, n,
                              H->Sg_c + c0, H->dmax, 1, st));
    c.launches += norient;
    c.sample_launches += norient;
    H->st.sample_launches += norient;
    CK(cudaFreeAsync(T, st));
  } else if (H->o.precision == HSS_PREC_FP64) {
    CK(c.timer.mark(PH_SAMPLE, st));
    CK(launch_sample_fp64(s, w, Rc, n, H->Sg_r + c0, H->sym ? nullptr : H->Sg_c + c0, H->dmax, st));
    c.launches += norient;
    c.sample_launches += norient;
    H->st.sample_launches += norient;
  } else if (use_packed(H)) {
    // dense A, or generated entries whose split tiles fit comfortably in
    // HBM: split once per compression into packed tensor-core tiles, then
    // every pass streams them (a generated A is evaluated once, not once per
    // pass)
    if (!H->packA) {
      const size_t pb = packed_a_bytes(n, H->o.precision);
      CK(c.timer.mark(PH_SAMPLE, st));
      CK(dmalloc_async(&H->packA, pb, st));
      CK(launch_pack_a(s, H->o.leaf, H->o.precision, H->packA, st));
      c.launches++;
      // the split is part of the sampling work: a dense A read once, the
      // packed tiles written once
      H->st.bytes_sample += (H->src.kind == HSS_SRC_DENSE ? 8.0 * n * (double)n : 0.0) + (double)pb;
      CK(c.timer.mark(PH_RNG, st));
    }
    void* packR = nullptr;
    CK(dmalloc_async(&packR, packed_r_bytes(n, w, H->o.precision), st));
    CK(launch_pack_r(Rc, n, n, w, H->o.precision, packR, st));
    c.launches++;
    if (sample_tc_packed_ksplit(n, w, H->o.precision) > 1) {
      CK(cudaMemset2DAsync(H->Sg_r + c0, sizeof(double) * H->dmax, 0, sizeof(double) * w, n, st));
      if (!H->sym) CK(cudaMemset2DAsync(H->Sg_c + c0, sizeof(double) * H->dmax, 0, sizeof(double) * w, n, st));
    }
    CK(c.timer.mark(PH_SAMPLE, st));
    CK(launch_sample_tc_packed(H->packA, packR, n, w, H->o.precision, 0, H->Sg_r + c0, H->dmax, c.d_flag + 1, st));
    if (!H->sym)
      CK(launch_sample_tc_packed(H->packA, packR, n, w, H->o.precision, 1, H->Sg_c + c0, H->dmax, c.d_flag + 1,
                                 st));
    c.launches += norient;
    c.sample_launches += norient;
    H->st.sample_launches += norient;
    CK(c.timer.mark(PH_RNG, st));
    CK(cudaFreeAsync(packR, st));
  } else {
    if (H->src.kind == HSS_SRC_TOEPLITZ && !H->toep_terms) {
      // the diagonals split once per compression: the producers assemble
      // tiles from windows of them
      CK(dmalloc_async(&H->toep_terms, toeplitz_terms_bytes(n, H->o.precision), st));
      CK(launch_toeplitz_terms(s, H->o.precision, H->toep_terms, st));
      c.launches++;
    }
    void* packR = nullptr;
    CK(dmalloc_async(&packR, packed_r_bytes(n, w, H->o.precision), st));
    CK(launch_pack_r(Rc, n, n, w, H->o.precision, packR, st));
    c.launches++;
    if (sample_tc_ksplit(n, w, H->o.precision) > 1) {
      CK(cudaMemset2DAsync(H->Sg_r + c0, sizeof(double) * H->dmax, 0, sizeof(double) * w, n, st));
      if (!H->sym) CK(cudaMemset2DAsync(H->Sg_c + c0, sizeof(double) * H->dmax, 0, sizeof(double) * w, n, st));
    }
    CK(c.timer.mark(PH_SAMPLE, st));
    int at = 0;
    CK(launch_sample_tc(s, H->o.leaf, H->o.precision, 0, w, packR, H->Sg_r + c0, H->dmax, c.d_flag + 1, &at,
                        H->toep_terms, st));
    if (!H->sym)
      CK(launch_sample_tc(s, H->o.leaf, H->o.precision, 1, w, packR, H->Sg_c + c0, H->dmax, c.d_flag + 1, &at,
                          H->toep_terms, st));
    c.launches += norient;
    c.sample_launches += norient;
    H->st.sample_launches += norient;
    CK(c.timer.mark(PH_RNG, st));
    CK(cudaFreeAsync(packR, st));
  }
  CK(c.timer.mark(PH_RNG, st));
  H->st.flop_sample += 2.0 * norient * (double)n * (double)n * (double)w;
  // algorithmic bytes of the sampling kernels: A read once per orientation
  // (FP64: 8 B per entry; packed TF32x2: 8 B; packed BF16x3: 6 B), R read,
  // S written
  double abytes = 0.0;
  if (H->o.op) abytes = 0.0;   // the operator's own traffic is not the library's
  else if (H->src.kind == HSS_SRC_DENSE || (H->o.precision != HSS_PREC_FP64 && H->pack_decided == 1))
    abytes = (H->o.precision == HSS_PREC_BF16X3 ? 6.0 : 8.0) * n * (double)n;
  H->st.bytes_sample += norient * (abytes + 2.0 * 8.0 * n * (double)w);
  int* flag = c.d_flag + 8 + H->slot;
  CK(launch_nonfinite(H->Sg_r, H->dmax, n, c0, c1, flag, st));
  if (!H->sym) CK(launch_nonfinite(H->Sg_c, H->dmax, n, c0, c1, flag, st));
  c.launches += norient;
  return HSS_OK;
}

// One read-back of the sampling flags of every matrix after a sampling round.
hss_status sample_check(Ctx& c, const std::vector<hss_matrix_s*>& Hs) {
  CKS(readback(c, c.d_flag, sizeof(int) * c.nflag));
  if (c.h_pinned[1]) return fail(HSS_ERR_TIMEOUT, "tensor-core sampling gave up waiting (code %d)", c.h_pinned[1]);
  for (hss_matrix_s* H : Hs)
    if (c.h_pinned[8 + H->slot])
      return fail(HSS_ERR_NONFINITE, "NaN or Inf in the random samples (columns up to %d)", H->d);
  return HSS_OK;
}

// ------------------------------------------------------ one pass of Alg. 3
hss_status alloc_side(hss_matrix_s* H, Side& s, bool leaf, double* Sleaf, int m) {
  s.m = m;
  s.S = leaf ? Sleaf : (double*)H->arena.alloc(sizeof(double) * (size_t)std::max(m, 1) * H->dmax);
  s.piv = (int*)H->arena.alloc(sizeof(int) * (size_t)std::max(m, 1));
  if (!s.S || !s.piv) return fail(HSS_ERR_NOMEM, "device arena allocation failed (side, m=%d)", m);
  if (H->o.strategy == HSS_INCREMENTING) {
    s.Q = (double*)H->arena.alloc(sizeof(double) * (size_t)std::max(m, 1) * H->dmax);
    if (!s.Q) return fail(HSS_ERR_NOMEM, "device arena allocation failed (basis Q)");
  }
  return HSS_OK;
}

// Merge jobs (Algorithm 2, non-leaf ComputeLocalSamples) for columns [cs, d).
void merge_jobs(hss_matrix_s* H, Node& t, int cs, int d, std::vector<GemmJob>& jobs) {
  Node& a = H->nodes[t.ch[0]];
  Node& b = H->nodes[t.ch[1]];
  const long long dm = H->dmax;
  const int N = d - cs;
  auto blk = [&](double* dst, const Side& child, const double* Bm, long long brs, long long bcs,
                 const double* Rred, int K) {
    GemmJob j = gemm_job();
    j.M = child.k; j.N = N; j.K = K;
    j.C0 = opnd(child.S + cs, dm, 1, child.piv);
    j.beta = 1.0;
    j.A = opnd(Bm, brs, bcs);
    j.B = opnd(Rred + cs, dm, 1);
    j.alpha = -1.0;
    j.C = dst + cs; j.c_rs = dm; j.c_cs = 1;
    jobs.push_back(j);
  };
  const int k1r = a.r.k, k2r = b.r.k, k1c = a.c.k, k2c = b.c.k;
  // tau.S^r = [nu1.S^r(J) - B12 nu2.R^r ; nu2.S^r(J) - B21 nu1.R^r]
  blk(t.r.S, a.r, t.B12, 1, std::max(k1r, 1), b.Rr, k2c);
  blk(t.r.S + (long long)k1r * dm, b.r, t.B21, 1, std::max(k2r, 1), a.Rr, k1c);
  if (H->sym) return;   // symmetric option: tau.S^c is tau.S^r
  // tau.S^c = [nu1.S^c(J) - B21^T nu2.R^c ; nu2.S^c(J) - B12^T nu1.R^c]
  blk(t.c.S, a.c, t.B21, std::max(k2r, 1), 1, b.Rc, k2r);
  blk(t.c.S + (long long)k1c * dm, b.c, t.B12, std::max(k1r, 1), 1, a.Rc, k1r);
}

// ReduceLocalSamples (Algorithm 2) for columns [cs, d): Rr = V^T x, Rc = U^T x.
void reduce_jobs(hss_matrix_s* H, Node& t, int cs, int d, std::vector<GemmJob>& jobs) {
  const long long dm = H->dmax;
  const int N = d - cs;
  auto one = [&](double* out, const Side& s, Opnd x_rows_gather_base) {
    if (s.k <= 0 || N <= 0) return;
    GemmJob j = gemm_job();
    j.M = s.k; j.N = N; j.K = s.m - s.k;
    Opnd c0 = x_rows_gather_base;
    c0.rows = s.piv;
    j.C0 = c0;
    j.beta = 1.0;
    j.A = opnd(s.X, 1, std::max(s.k, 1));
    Opnd bb = x_rows_gather_base;
    bb.rows = s.piv + s.k;
    j.B = bb;
    j.C = out + cs; j.c_rs = dm; j.c_cs = 1;
    jobs.push_back(j);
  };
  if (t.leaf) {
    Opnd x = opnd(H->R + t.lo + (long long)cs * H->n, 1, H->n);
    one(t.Rr, t.c, x);
    if (!H->sym) one(t.Rc, t.r, x);     // symmetric option: R^c is R^r
  } else {
    Node& a = H->nodes[t.ch[0]];
    Node& b = H->nodes[t.ch[1]];
    one(t.Rr, t.c, opnd(a.Rr + cs, dm, 1, nullptr, b.Rr + cs, a.c.k));
    if (!H->sym) one(t.Rc, t.r, opnd(a.Rc + cs, dm, 1, nullptr, b.Rc + cs, a.r.k));
  }
}

std::mutex& tuning_mutex() {
  static std::mutex m;
  return m;
}
hss_tuning& tuning_ref() {
  static hss_tuning t{8, 4, 2, 4};
  return t;
}

// Most CTAs of one side's group in the Incrementing test (every value of a
// column step adds this many partial sums).
constexpr int INC_GROUP_PMAX = 32;

std::mutex& coop_launch_mutex() {
  static std::mutex m;
  return m;
}

// QRCP/ID over all columns [0, H->d) of the listed node sides (of one or
// several matrices, each at its own d).
struct QrcpReq { hss_matrix_s* H; int node; int side; int rule; };

hss_status run_qrcp(Ctx& c, const std::vector<QrcpReq>& reqs, std::vector<double*>& wbuf) {
  c.scratch.reset();
  if (reqs.empty()) return HSS_OK;
  cudaStream_t st = c.st;
  const size_t nj = reqs.size();
  int dmx = 1;
  for (const QrcpReq& q : reqs) dmx = std::max(dmx, q.H->d);
  // Launch shape.  Every job gets a group of P CTAs, each owning about g of
  // its m columns (g a multiple of 32, at most qrcp_cols_per_cta()), with g
  // the smallest width for which the groups of a batch fit the co-resident
  // CTAs; one cooperative launch per batch (plain launch when every P is 1).
  // few node sides (the top levels): the wide shape, whose groups have half
  // as many CTAs; otherwise the narrow one (or the number of CTAs per SM the
  // tuning fixes).  Shapes: 0 = 128 threads, four CTAs per SM; 1 = 256, two;
  // 2 = 512, one.
  const hss_tuning tun = tuning_get();
  int wide = (int)nj <= tun.qrcp_wide_max_sides ? 1 : 0;
  if (tun.qrcp_sm_ctas) wide = tun.qrcp_sm_ctas == 4 ? 0 : (tun.qrcp_sm_ctas == 2 ? 1 : 2);
  if (c.qrcp_cap_d != dmx || c.qrcp_cap_w != wide) {
    c.qrcp_cap = qrcp_group_capacity(dmx, wide, &c.qrcp_nsm, &c.qrcp_per);
    c.qrcp_cap_d = dmx;
    c.qrcp_cap_w = wide;
  }
  const int cap = c.qrcp_cap, NL = qrcp_cols_per_cta();
  if (cap <= 0) return fail(HSS_ERR_CUDA, "QRCP kernel cannot be resident (d = %d)", dmx);
  auto side_of = [&](const QrcpReq& q) -> Side& { return q.side ? q.H->nodes[q.node].c : q.H->nodes[q.node].r; };
  std::vector<int> mj(nj), P(nj, 1);
  for (size_t i = 0; i < nj; ++i) mj[i] = std::max(side_of(reqs[i]).m, 1);
  struct Batch { size_t b0, b1; bool group; };
  std::vector<Batch> batches;
  bool all_small = nj >= (size_t)cap;
  for (size_t i = 0; i < nj && all_small; ++i) all_small = mj[i] <= NL;
  if (all_small) batches.push_back({0, nj, false});   // one CTA per side fills the GPU: one plain launch
  for (size_t b0 = all_small ? nj : 0; b0 < nj;) {
    // the largest prefix whose groups fit at width NL
    size_t b1 = b0;
    int used = 0;
    while (b1 < nj) {
      const int p = (mj[b1] + NL - 1) / NL;
      if (b1 > b0 && used + p > cap) break;
      used += p;
      ++b1;
    }
    // groups proportional to m filling every co-resident slot (an equal
    // number of CTAs on every SM, so that no SM runs a double share), each
    // CTA with at most NL columns
    for (size_t i = b0; i < b1; ++i) P[i] = std::max(1, (mj[i] + NL - 1) / NL);
    // hand the remaining slots to the jobs with the most work per CTA; the
    // work of a side is sum_j (d - j)(m - j) over its expected pivot steps:
    // the rank of its previous attempt (Doubling repeats a failed side at
    // twice the width) with some growth, else min(m, d)
    std::vector<double> wk(nj, 0.0);
    for (size_t i = b0; i < b1; ++i) {
      const Side& s = side_of(reqs[i]);
      const double m = mj[i], dd = reqs[i].H->d, kmx = std::min(m, dd);
      const double k = s.qr_k > 0 ? std::min(kmx, 1.25 * s.qr_k + 16.0) : kmx;
      wk[i] = dd * m * k - 0.5 * (dd + m) * k * k + k * k * k / 3.0 + 1.0;
    }
    std::priority_queue<std::pair<double, size_t>> pq;
    for (size_t i = b0; i < b1; ++i) pq.push({wk[i] / P[i], i});
    while (used < cap && !pq.empty()) {
      auto top = pq.top();
      pq.pop();
      const size_t i = top.second;
      if (mj[i] / (P[i] + 1) < tun.qrcp_min_cols) continue;   // keep enough columns per CTA
      P[i]++;
      used++;
      pq.push({wk[i] / P[i], i});
    }
    bool group = false;
    for (size_t i = b0; i < b1; ++i) group = group || P[i] > 1;
    batches.push_back({b0, b1, group});
    b0 = b1;
  }
  size_t need = 0;
  for (size_t i = 0; i < nj; ++i) {
    const long long ldw = ((long long)reqs[i].H->d + 3) / 4 * 4;
    need += Scratch::rnd(sizeof(double) * (size_t)ldw * mj[i]) + Scratch::rnd(sizeof(double) * mj[i]) +
            Scratch::rnd(sizeof(double) * (size_t)std::max(1, std::min(mj[i], reqs[i].H->d))) +
            Scratch::rnd(sizeof(double) * 4 * P[i]) + Scratch::rnd(sizeof(double) * 2 * P[i]) +
            Scratch::rnd(sizeof(double) * 8);
  }
  need += Scratch::rnd(sizeof(unsigned) * nj) + Scratch::rnd(sizeof(int) * 3 * nj);
  need += Scratch::rnd(sizeof(unsigned) * QRCP_PLACE_WORDS * batches.size());
  CK(c.scratch.ensure(need, st));
  std::vector<QrcpJob> jobs;
  wbuf.clear();
  unsigned* bars = (unsigned*)c.scratch.take(sizeof(unsigned) * nj);
  int* outs = (int*)c.scratch.take(sizeof(int) * 3 * nj);
  // per batch: the placement counters of its cooperative launch
  unsigned* places = (unsigned*)c.scratch.take(sizeof(unsigned) * QRCP_PLACE_WORDS * batches.size());
  for (size_t i = 0; i < nj; ++i) {
    const QrcpReq& q = reqs[i];
    hss_matrix_s* H = q.H;
    Node& t = H->nodes[q.node];
    Side& s = q.side ? t.c : t.r;
    const int d = H->d;
    const long long ldw = ((long long)d + 3) / 4 * 4;   // 32-byte aligned columns
    QrcpJob j;
    memset(&j, 0, sizeof j);
    j.S = s.S; j.lds = H->dmax; j.m = s.m; j.d = d;
    j.W = (double*)c.scratch.take(sizeof(double) * (size_t)ldw * mj[i]);
    j.ldw = ldw;
    j.nrm = (double*)c.scratch.take(sizeof(double) * mj[i]);
    j.diag = (double*)c.scratch.take(sizeof(double) * std::max(1, std::min(mj[i], d)));
    j.piv = s.piv;
    j.rule = q.rule;
    j.mh = t.size; j.nh = H->n - t.size; j.p = H->o.oversample_p;
    j.do_id = 1;
    double sc = tol_scale(H, t.level);
    // the HMT criterion knows the absolute tolerance only: its final RRQR
    // keeps the pivots above eps_a
    j.er = (H->o.criterion == HSS_CRIT_HMT ? 0.0 : H->o.rtol) * sc; j.ea = H->o.atol * sc;
    j.out = outs + 3 * i;
    j.P = P[i];
    j.bar = bars + i;
    j.redv = (double*)c.scratch.take(sizeof(double) * 4 * P[i]);   // 2 P (key, index) pairs
    j.redt = (double*)c.scratch.take(sizeof(double) * 2 * P[i]);
    j.xfer = (double*)c.scratch.take(sizeof(double) * 8);
    j.wait_ns = wait_limit(H);
    wbuf.push_back(j.W);
    jobs.push_back(j);
  }
  if (c.scratch.overflow) return fail(HSS_ERR_NOMEM, "QRCP scratch sized too small");
  CK(c.timer.mark(PH_ID, st));
  CK(cudaMemsetAsync(bars, 0, sizeof(unsigned) * nj, st));
  CK(cudaMemsetAsync(places, 0, sizeof(unsigned) * QRCP_PLACE_WORDS * batches.size(), st));
  CK(cudaMemsetAsync(c.d_flag + 2, 0, sizeof(int), st));
  if (c.trace) CK(cudaEventRecord(c.trace_ev[0], st));
  // job list and every batch's (job, rank) map in one upload
  Staging sg;
  const size_t oj = sg.put(jobs.data(), jobs.size() * sizeof(QrcpJob));
  std::vector<size_t> omap(batches.size(), 0);
  std::vector<int> nmap(batches.size(), 0);
  for (size_t bi = 0; bi < batches.size(); ++bi) {
    const Batch& b = batches[bi];
    if (!b.group) continue;
    // every co-resident slot, positions slot x nsm + SM index: the groups'
    // ranks in order, so that the CTAs of a group run on different SMs and
    // each SM hosts ranks of several groups; the rest idle
    std::vector<int2> map;
    for (size_t i = b.b0; i < b.b1; ++i)
      for (int r = 0; r < P[i]; ++r) map.push_back(make_int2((int)i, r));
    if ((int)map.size() > cap) return fail(HSS_ERR_CUDA, "QRCP groups exceed the co-resident CTAs");
    map.resize((size_t)cap, make_int2(-1, -1));
    omap[bi] = sg.put(map.data(), map.size() * sizeof(int2));
    nmap[bi] = (int)map.size();
  }
  char* dev;
  CKS(sg.send(c, &dev));
  const QrcpJob* dj = (const QrcpJob*)(dev + oj);
  // A cooperative launch needs all of its CTAs resident at once: compressions
  // running side by side on other host threads take turns with them, the
  // lock held until the launch has finished (the flag read-back below).
  bool any_group = false;
  for (const Batch& b : batches) any_group = any_group || b.group;
  std::unique_lock<std::mutex> coop(coop_launch_mutex(), std::defer_lock);
  if (any_group) coop.lock();
  int ctas_total = 0;
  for (size_t bi = 0; bi < batches.size(); ++bi) {
    const Batch& b = batches[bi];
    if (b.group) {
      const bool place = c.qrcp_nsm * c.qrcp_per == nmap[bi];
      CK(launch_qrcp(dj, (const int2*)(dev + omap[bi]), nmap[bi], dmx, wide, c.d_flag + 2,
                     place ? places + QRCP_PLACE_WORDS * bi : nullptr, c.qrcp_nsm, c.qrcp_per, st));
      ctas_total += nmap[bi];
    } else {
      CK(launch_qrcp(dj + b.b0, nullptr, (int)(b.b1 - b.b0), dmx, wide, c.d_flag + 2, nullptr, 0, 0, st));
      ctas_total += (int)(b.b1 - b.b0);
    }
    c.launches++;
  }
  const int nbatch = (int)batches.size();
  if (c.trace) CK(cudaEventRecord(c.trace_ev[1], st));
  // the flags and the (k, stopped, accepted) triples in one read-back
  std::vector<size_t> off;
  CKS(readback_many(c, {{c.d_flag, sizeof(int) * 8}, {outs, sizeof(int) * 3 * jobs.size()}}, off));
  const int* hf = (const int*)((char*)c.h_pinned + off[0]);
  const int* ho = (const int*)((char*)c.h_pinned + off[1]);
  const int f2 = hf[2], f3 = hf[3];
  if (coop.owns_lock()) coop.unlock();
  if (f2) return fail(HSS_ERR_TIMEOUT, "group QRCP barrier gave up (code %d)", f2);
  if (f3) return fail(HSS_ERR_TIMEOUT, "tensor-core tile product gave up waiting (code %d)", f3);
  double tr_flop = 0.0;
  int tr_m = 0, tr_k = 0;
  double tr_wmax = 0.0;
  for (size_t i = 0; i < reqs.size(); ++i) {
    Side& s = side_of(reqs[i]);
    s.qr_k = ho[3 * i];
    s.qr_acc = ho[3 * i + 2];
    // algorithmic flops: norms, k Householder steps (reflector + trailing
    // dot and update of m-j-1 columns), back substitution for X
    const double m = jobs[i].m, dd = jobs[i].d, k = s.qr_k;
    double f = 2.0 * m * dd;
    for (int j = 0; j < s.qr_k; ++j) f += 4.0 * (dd - j) * (m - j - 1) + 3.0 * (dd - j);
    if (s.qr_acc && k > 0 && m > k) f += k * k * (m - k);
    reqs[i].H->st.flop_id += f;
    tr_flop += f;
    tr_m = std::max(tr_m, jobs[i].m);
    tr_k = std::max(tr_k, s.qr_k);
    tr_wmax = std::max(tr_wmax, f / P[i]);
  }
  if (c.trace) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c.trace_ev[0], c.trace_ev[1]);
    // balance: the work per CTA of the busiest group against the mean
    fprintf(stderr,
            "[hss trace] qrcp level %d jobs %zu batches %d ctas %d max_m %d d %d max_k %d  %.3f ms  %.1f GFLOP/s"
            "  balance %.2f\n",
            reqs[0].H->nodes[reqs[0].node].level, nj, nbatch, ctas_total, tr_m, dmx, tr_k, ms,
            tr_flop / (ms * 1e6), tr_flop / std::max(1.0, tr_wmax * ctas_total));
  }
  return HSS_OK;
}

// After an accepted QRCP: permanent X (compacted out of the workspace) and
// the global skeleton indices tau.I = base(J).
hss_status finalize_id(hss_matrix_s* H, int node, int side, const double* W, std::vector<GemmJob>& copies,
                       std::vector<GatherJob>& gathers) {
  Node& t = H->nodes[node];
  Side& s = side ? t.c : t.r;
  s.k = s.qr_k;
  const int k = s.k, m = s.m, d = H->d;
  s.X = (double*)H->arena.alloc(sizeof(double) * (size_t)std::max(k, 1) * std::max(m - k, 1));
  s.I = (int*)H->arena.alloc(sizeof(int) * (size_t)std::max(k, 1));
  if (!s.X || !s.I) return fail(HSS_ERR_NOMEM, "device arena allocation failed (ID)");
  if (k > 0 && m > k) {
    // X(:, t) = W(0:k, piv[k + t]): element (t, i) of the copy's transposed view
    GemmJob j = gemm_job();
    j.M = m - k; j.N = k; j.K = 0;
    j.C0 = opnd(W, ((long long)d + 3) / 4 * 4, 1, s.piv + k);   // QRCP workspace, ldw
    j.beta = 1.0;
    j.C = s.X; j.c_rs = k; j.c_cs = 1;
    copies.push_back(j);
  }
  if (k > 0) {
    GatherJob g;
    if (t.leaf) {
      g = {H->iota + t.lo, nullptr, s.piv, s.I, k, 0x7fffffff};
    } else {
      Side& a = side ? H->nodes[t.ch[0]].c : H->nodes[t.ch[0]].r;
      Side& b = side ? H->nodes[t.ch[1]].c : H->nodes[t.ch[1]].r;
      g = {a.I, b.I, s.piv, s.I, k, a.k};
    }
    gathers.push_back(g);
  }
  return HSS_OK;
}

// The Incrementing test (Algorithm 5) of the candidate sides of one level of
// every listed matrix: all their untested blocks, one round per block, until
// each side passes or runs out of columns (P18).
hss_status incrementing_tests(Ctx& c, const std::vector<std::pair<hss_matrix_s*, std::vector<int>>>& cands) {
  cudaStream_t st = c.st;
  struct Sd { hss_matrix_s* H; int node, side; };
  auto block_end = [&](hss_matrix_s* H, int tested) {
    for (int bnd : H->bounds)
      if (bnd > tested) return std::min(bnd, H->d);
    return H->d;
  };
  for (;;) {
    std::vector<Sd> sides;
    for (auto& hc : cands) {
      hss_matrix_s* H = hc.first;
      for (int id : hc.second) {
        Node& t = H->nodes[id];
        for (int sd = 0; sd < (H->sym ? 1 : 2); ++sd) {
          Side& s = sd ? t.c : t.r;
          if (s.done) {
            s.tested = H->d;
          } else if (H->d > s.tested) {
            // a block that brings the basis to m columns leaves the side
            // sufficient whatever its test finds (the test passes, or Q_k
            // joins and spans every row, P18): nothing to compute
            const int be = block_end(H, s.tested);
            if (s.q + (be - s.tested) >= s.m) {
              s.tested = be;
              s.done = true;
            } else {
              sides.push_back({H, id, sd});
            }
          }
        }
        if (H->sym) t.c = t.r;
      }
    }
    if (sides.empty()) return HSS_OK;
    CK(c.timer.mark(PH_TEST, st));
    c.scratch.reset();
    size_t need = 0;
    for (auto& x : sides) {
      Side& s = x.side ? x.H->nodes[x.node].c : x.H->nodes[x.node].r;
      size_t b = block_end(x.H, s.tested) - s.tested, m = std::max(s.m, 1);
      const int pg = (int)((m + inc_group_rows((int)b) - 1) / inc_group_rows((int)b));   // fewest CTAs of a group
      need += Scratch::rnd(8 * m * b) + Scratch::rnd(8 * std::max<size_t>(std::max(s.q, s.m), 1) * b) +
              Scratch::rnd(8 * b) + Scratch::rnd(8 * 4) + Scratch::rnd(8) + Scratch::rnd(sizeof(unsigned)) +
              Scratch::rnd(8 * inc_group_part(std::max(pg, INC_GROUP_PMAX), (int)b));
    }
    CK(c.scratch.ensure(need, st));
    std::vector<IncJob> ij;
    GemmSet g1, g2, g3;
    int bmax = 0;
    for (auto& x : sides) {
      hss_matrix_s* H = x.H;
      Node& t = H->nodes[x.node];
      Side& s = x.side ? t.c : t.r;
      IncJob j;
      memset(&j, 0, sizeof j);
      const int b = block_end(H, s.tested) - s.tested, m = s.m;
      bmax = std::max(bmax, b);
      j.S = s.S; j.lds = H->dmax; j.m = m; j.c0 = s.tested; j.b = b;
      j.Q = s.Q; j.q = s.q;
      j.Sh = (double*)c.scratch.take(8 * (size_t)std::max(m, 1) * b);
      j.T = (double*)c.scratch.take(8 * (size_t)std::max(std::max(s.q, m), 1) * b);
      j.tau = (double*)c.scratch.take(8 * (size_t)b);
      double sc = tol_scale(H, t.level);
      j.er = H->o.rtol * sc; j.ea = H->o.atol * sc;
      j.rho = s.rho;
      j.hmt = H->o.criterion == HSS_CRIT_HMT;
      j.hmt_c = j.hmt ? H->o.hmt_alpha * std::sqrt(2.0 / std::acos(-1.0)) : 0.0;
      j.wait_ns = wait_limit(H);
      ij.push_back(j);
      // Sh = S(:, tested:tested+b)
      GemmJob cp = gemm_job();
      cp.M = m; cp.N = b; cp.K = 0;
      cp.C0 = opnd(s.S + s.tested, H->dmax, 1);
      cp.beta = 1.0;
      cp.C = j.Sh; cp.c_rs = 1; cp.c_cs = m;
      g1.add(HSS_PREC_FP64, cp);
      if (s.q > 0) {
        GemmJob t1 = gemm_job();   // T = Q^T Sh
        t1.M = s.q; t1.N = b; t1.K = m;
        t1.A = opnd(s.Q, 1, H->dmax);
        t1.B = opnd(j.Sh, 1, m);
        t1.C = j.T; t1.c_rs = 1; t1.c_cs = s.q;
        g2.add(H->o.precision, t1);
        GemmJob t2 = gemm_job();   // Sh -= Q T
        t2.M = m; t2.N = b; t2.K = s.q;
        t2.A = opnd(s.Q, H->dmax, 1);
        t2.B = opnd(j.T, 1, s.q);
        t2.alpha = -1.0; t2.gamma = 1.0;
        t2.C = j.Sh; t2.c_rs = 1; t2.c_cs = m;
        g3.add(H->o.precision, t2);
      }
    }
    double* res0 = (double*)c.scratch.take(sizeof(double) * 4 * ij.size());
    int* flag0 = (int*)c.scratch.take(sizeof(int) * 2 * ij.size());
    for (size_t i = 0; i < ij.size(); ++i) { ij[i].res = res0 + 4 * i; ij[i].flag = flag0 + 2 * i; }
    CKS(run_gemm_set(c, g1, "test-copy"));
    // (I - Q Q^T)^2; in the mixed forms both products take the tensor
    // cores with the three-term split of the merges (error below 2^-32
    // of |Q||S| per product, under the samples' own noise); the norms,
    // the QR and every decision stay FP64
    for (int rep = 0; rep < 2; ++rep) {
      CKS(run_gemm_set(c, g2, "test-QtS"));
      CKS(run_gemm_set(c, g3, "test-S-QT"));
    }
    // the rows of each side over a group of CTAs (one cooperative launch
    // per batch of sides that fits the co-resident slots); blocks wider
    // than the group kernel takes go to one CTA per side
    // (only when one CTA per side would leave SMs idle and all groups fit
    // two launches; a level with many sides keeps one CTA per side)
    int nsm = 0, cur = 0;
    CK(cudaGetDevice(&cur));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, cur));
    bool grouped = bmax <= inc_group_bmax() && (int)ij.size() < nsm;
    const int gcap = grouped ? inc_group_capacity(bmax) : 0;
    long long gsum = 0;
    for (const IncJob& j : ij) {   // the groups at their row widths fit two launches
      const int rows = inc_group_rows(j.b);
      const int pmin = (j.m + rows - 1) / rows;
      if (pmin > gcap) grouped = false;
      gsum += pmin;
    }
    if (gsum > 2LL * gcap) grouped = false;
    std::vector<int> P(ij.size(), 1);
    std::vector<std::pair<size_t, size_t>> gbatches;
    if (grouped) {
      // the fewest CTAs whose rows fit shared memory, then the remaining
      // resident slots to the sides with the most rows per CTA (at most
      // INC_GROUP_PMAX CTAs and at least 8 rows each): a group's cost is its
      // barriers and its rows per CTA
      long long used = 0;
      std::priority_queue<std::pair<double, size_t>> pq;
      for (size_t i = 0; i < ij.size(); ++i) {
        const int rows = inc_group_rows(ij[i].b);
        P[i] = std::max(1, (ij[i].m + rows - 1) / rows);
        used += P[i];
        pq.push({(double)ij[i].m / P[i], i});
      }
      while (gsum <= gcap && used < gcap && !pq.empty()) {   // one launch: fill its slots
        const size_t i = pq.top().second;
        pq.pop();
        if (P[i] >= INC_GROUP_PMAX || ij[i].m / (P[i] + 1) < 8) continue;
        P[i]++;
        used++;
        pq.push({(double)ij[i].m / P[i], i});
      }
      for (size_t i = 0; i < ij.size(); ++i) {
        ij[i].P = P[i];
        ij[i].bar = (unsigned*)c.scratch.take(sizeof(unsigned));
        ij[i].part = (double*)c.scratch.take(sizeof(double) * inc_group_part(std::max(P[i], INC_GROUP_PMAX), ij[i].b));
      }
      for (size_t b0 = 0; b0 < ij.size();) {
        size_t b1 = b0;
        int used = 0;
        while (b1 < ij.size() && (b1 == b0 || used + P[b1] <= gcap)) used += P[b1++];
        gbatches.push_back({b0, b1});
        b0 = b1;
      }
    }
    if (c.scratch.overflow) return fail(HSS_ERR_NOMEM, "test scratch sized too small");
    Staging sg;
    const size_t oj = sg.put(ij.data(), ij.size() * sizeof(IncJob));
    std::vector<size_t> omap;
    std::vector<int> nmap;
    for (auto& gb : gbatches) {
      std::vector<int2> map;
      for (size_t i = gb.first; i < gb.second; ++i)
        for (int r = 0; r < P[i]; ++r) map.push_back(make_int2((int)i, r));
      omap.push_back(sg.put(map.data(), map.size() * sizeof(int2)));
      nmap.push_back((int)map.size());
    }
    char* dev;
    CKS(sg.send(c, &dev));
    const IncJob* dj = (const IncJob*)(dev + oj);
    if (c.trace) CK(cudaEventRecord(c.trace_ev[0], st));
    std::unique_lock<std::mutex> coop(coop_launch_mutex(), std::defer_lock);
    if (grouped) {
      CK(cudaMemsetAsync(c.d_flag + 4, 0, sizeof(int), st));
      for (size_t i = 0; i < ij.size(); ++i) CK(cudaMemsetAsync(ij[i].bar, 0, sizeof(unsigned), st));
      coop.lock();
      for (size_t b = 0; b < gbatches.size(); ++b) {
        CK(launch_inc_group(dj, (const int2*)(dev + omap[b]), nmap[b], bmax, c.d_flag + 4, st));
        c.launches++;
      }
    } else {
      CK(launch_inc_qr(dj, (int)ij.size(), st));
      c.launches++;
    }
    if (c.trace) {
      CK(cudaEventRecord(c.trace_ev[1], st));
      CK(cudaEventSynchronize(c.trace_ev[1]));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, c.trace_ev[0], c.trace_ev[1]);
      int mm = 0, qq = 0;
      for (auto& x : sides) {
        const Side& s = x.side ? x.H->nodes[x.node].c : x.H->nodes[x.node].r;
        mm = std::max(mm, s.m);
        qq = std::max(qq, s.q);
      }
      fprintf(stderr, "[hss trace] inc_qr sides %zu max_m %d max_q %d b %d  %.3f ms\n", sides.size(), mm, qq, bmax, ms);
    }
    // the barrier flag, the test flags and the norms in one read-back
    std::vector<size_t> off;
    CKS(readback_many(c, {{c.d_flag + 4, sizeof(int)}, {flag0, sizeof(int) * 2 * ij.size()},
                          {res0, sizeof(double) * 4 * ij.size()}}, off));
    if (coop.owns_lock()) coop.unlock();
    const int bar_err = *(const int*)((char*)c.h_pinned + off[0]);
    if (grouped && bar_err)
      return fail(HSS_ERR_TIMEOUT, "Incrementing test group barrier gave up (code %d)", bar_err);
    const int* flags = (const int*)((char*)c.h_pinned + off[1]);
    const double* res = (const double*)((char*)c.h_pinned + off[2]);
    for (size_t i = 0; i < sides.size(); ++i) {
      hss_matrix_s* H = sides[i].H;
      Side& s = sides[i].side ? H->nodes[sides[i].node].c : H->nodes[sides[i].node].r;
      s.tested = block_end(H, s.tested);
      s.q = flags[2 * i + 1];
      if (s.rho < 0.0 && res[4 * i + 3] >= 0.0) s.rho = res[4 * i + 3];
      s.done = flags[2 * i] != 0;
    }
  }
}

// One pass of Algorithm 3 (the sweep of CompressNodeAdaptive over the tree)
// for every listed matrix, in lockstep: step s takes level max_level - s of
// each matrix (the leaves of all of them first), and every phase of a step
// is one launch over the nodes of all matrices at that step.
hss_status run_pass(Ctx& c, const std::vector<hss_matrix_s*>& act) {
  cudaStream_t st = c.st;
  int depth = 0;
  for (hss_matrix_s* H : act) depth = std::max(depth, H->max_level);
  for (int sstep = 0; sstep < depth; ++sstep) {
    struct Lv { hss_matrix_s* H; int lev; std::vector<int> cand, upd; };
    std::vector<Lv> L;
    for (hss_matrix_s* H : act) {
      const int lev = H->max_level - sstep;
      if (lev < 1) continue;
      Lv lv{H, lev, {}, {}};
      for (int id : H->by_level[lev]) {
        Node& t = H->nodes[id];
        if (!t.leaf && (H->nodes[t.ch[0]].state != HSS_COMPRESSED || H->nodes[t.ch[1]].state != HSS_COMPRESSED))
          continue;
        (t.state == HSS_COMPRESSED ? lv.upd : lv.cand).push_back(id);
      }
      if (!lv.cand.empty() || !lv.upd.empty()) L.push_back(std::move(lv));
    }
    if (L.empty()) continue;
    CK(c.timer.mark(PH_MERGE, st));
    // --- extraction of D (new leaves) and B12/B21 (new non-leaves)
    ExtractSet ex;
    for (Lv& lv : L) {
      hss_matrix_s* H = lv.H;
      auto add_ex = [&](const int* I, int i0, int mi, const int* J, int j0, int nj, double* out, long long ldo) {
        if (mi <= 0 || nj <= 0) return;
        ExtractJob e;
        memset(&e, 0, sizeof e);
        e.I = I; e.i0 = i0; e.mi = mi; e.J = J; e.j0 = j0; e.nj = nj; e.out = out; e.ldo = ldo;
        ex.of(H).push_back(e);
      };
      for (int id : lv.cand) {
        Node& t = H->nodes[id];
        if (t.state != HSS_UNTOUCHED) continue;
        if (t.leaf) {
          if (!t.D) {   // (already there with a user operator)
            t.D = (double*)H->arena.alloc(sizeof(double) * (size_t)t.size * t.size);
            if (!t.D) return fail(HSS_ERR_NOMEM, "device arena allocation failed (D)");
            add_ex(nullptr, t.lo, t.size, nullptr, t.lo, t.size, t.D, t.size);
          }
          CKS(alloc_side(H, t.r, true, H->Sg_r + (long long)t.lo * H->dmax, t.size));
          if (H->sym) t.c = t.r;
          else CKS(alloc_side(H, t.c, true, H->Sg_c + (long long)t.lo * H->dmax, t.size));
        } else {
          Node& a = H->nodes[t.ch[0]];
          Node& b = H->nodes[t.ch[1]];
          t.B12 = (double*)H->arena.alloc(sizeof(double) * (size_t)std::max(a.r.k, 1) * std::max(b.c.k, 1));
          t.B21 = (double*)H->arena.alloc(sizeof(double) * (size_t)std::max(b.r.k, 1) * std::max(a.c.k, 1));
          if (!t.B12 || !t.B21) return fail(HSS_ERR_NOMEM, "device arena allocation failed (B)");
          add_ex(a.r.I, 0, a.r.k, b.c.I, 0, b.c.k, t.B12, std::max(a.r.k, 1));
          add_ex(b.r.I, 0, b.r.k, a.c.I, 0, a.c.k, t.B21, std::max(b.r.k, 1));
          CKS(alloc_side(H, t.r, false, nullptr, a.r.k + b.r.k));
          if (H->sym) t.c = t.r;
          else CKS(alloc_side(H, t.c, false, nullptr, a.c.k + b.c.k));
        }
      }
    }
    CKS(run_extract(c, ex));
    // --- local samples of non-leaf nodes (upward merge)
    GemmSet mj;
    for (Lv& lv : L) {
      hss_matrix_s* H = lv.H;
      std::vector<GemmJob> j;
      for (int id : lv.cand) {
        Node& t = H->nodes[id];
        if (!t.leaf) merge_jobs(H, t, t.state == HSS_UNTOUCHED ? 0 : H->d_prev, H->d, j);
      }
      for (int id : lv.upd) {
        Node& t = H->nodes[id];
        if (!t.leaf) merge_jobs(H, t, H->d_prev, H->d, j);
      }
      for (auto& g : j) mj.add(H->o.precision, g);
    }
    CKS(run_gemm_set(c, mj, "merge"));

    // --- strategy test on the candidates
    std::vector<QrcpReq> reqs;
    std::vector<std::pair<hss_matrix_s*, std::vector<int>>> inc;
    for (Lv& lv : L) {
      hss_matrix_s* H = lv.H;
      if (H->o.strategy == HSS_DOUBLING) {
        for (int id : lv.cand) {
          reqs.push_back({H, id, 0, 1});
          if (!H->sym) reqs.push_back({H, id, 1, 1});
        }
      } else if (!lv.cand.empty()) {
        inc.push_back({H, lv.cand});
      }
    }
    if (!inc.empty()) {
      CKS(incrementing_tests(c, inc));
      for (auto& hc : inc) {
        hss_matrix_s* H = hc.first;
        for (int id : hc.second) {
          Node& t = H->nodes[id];
          if (H->sym) t.c = t.r;
          if (t.r.done && t.c.done) {
            reqs.push_back({H, id, 0, 0});
            if (!H->sym) reqs.push_back({H, id, 1, 0});
          } else {
            t.state = HSS_PARTIALLY_COMPRESSED;
          }
        }
      }
    }
    std::vector<double*> wbuf;
    CKS(run_qrcp(c, reqs, wbuf));
    CK(c.timer.mark(PH_MERGE, st));
    std::vector<GemmJob> copies;
    std::vector<GatherJob> gathers;
    std::vector<std::pair<hss_matrix_s*, int>> accepted;
    // the requests come as (row side, column side) pairs, or one row-side
    // request per node with the symmetric option (the column side copies it)
    for (size_t i = 0; i < reqs.size();) {
      hss_matrix_s* H = reqs[i].H;
      const size_t per = H->sym ? 1 : 2;
      Node& t = H->nodes[reqs[i].node];
      if (H->sym) t.c = t.r;
      if (t.r.qr_acc && t.c.qr_acc) {
        CKS(finalize_id(H, reqs[i].node, 0, wbuf[i], copies, gathers));
        if (H->sym) t.c = t.r;
        else CKS(finalize_id(H, reqs[i].node, 1, wbuf[i + 1], copies, gathers));
        t.state = HSS_COMPRESSED;
        t.Rr = (double*)H->arena.alloc(sizeof(double) * (size_t)std::max(t.c.k, 1) * H->dmax);
        t.Rc = H->sym ? t.Rr : (double*)H->arena.alloc(sizeof(double) * (size_t)std::max(t.r.k, 1) * H->dmax);
        if (!t.Rr || !t.Rc) return fail(HSS_ERR_NOMEM, "device arena allocation failed (reduced R)");
        accepted.push_back({H, reqs[i].node});
      } else {
        t.state = HSS_PARTIALLY_COMPRESSED;
      }
      i += per;
    }
    CKS(run_gathers(c, gathers));
    CKS(run_gemms(c, copies, "x-copy"));
    GemmSet rj;
    for (auto& a : accepted) {
      std::vector<GemmJob> j;
      reduce_jobs(a.first, a.first->nodes[a.second], 0, a.first->d, j);
      for (auto& g : j) rj.add(a.first->o.precision, g);
    }
    for (Lv& lv : L) {
      std::vector<GemmJob> j;
      for (int id : lv.upd) reduce_jobs(lv.H, lv.H->nodes[id], lv.H->d_prev, lv.H->d, j);
      for (auto& g : j) rj.add(lv.H->o.precision, g);
    }
    CKS(run_gemm_set(c, rj, "reduce"));
  }
  // the roots: COMPRESSED once both children are (Algorithm 3), keeping
  // B12 = A(nu1.I^r, nu2.I^c), B21 = A(nu2.I^r, nu1.I^c), or D for a root leaf
  ExtractSet ex;
  for (hss_matrix_s* H : act) {
    Node& root = H->nodes[0];
    if (!(root.leaf || (H->nodes[root.ch[0]].state == HSS_COMPRESSED &&
                        H->nodes[root.ch[1]].state == HSS_COMPRESSED)))
      continue;
    if (root.state == HSS_UNTOUCHED) {
      auto add = [&](const int* I, int i0, int mi, const int* J, int j0, int nj, double* out, long long ldo) {
        if (mi <= 0 || nj <= 0) return;
        ExtractJob e;
        memset(&e, 0, sizeof e);
        e.I = I; e.i0 = i0; e.mi = mi; e.J = J; e.j0 = j0; e.nj = nj; e.out = out; e.ldo = ldo;
        ex.of(H).push_back(e);
      };
      if (root.leaf) {
        if (!root.D) {
          root.D = (double*)H->arena.alloc(sizeof(double) * (size_t)root.size * root.size);
          if (!root.D) return fail(HSS_ERR_NOMEM, "device arena allocation failed (D)");
          add(nullptr, 0, root.size, nullptr, 0, root.size, root.D, root.size);
        }
      } else {
        Node& a = H->nodes[root.ch[0]];
        Node& b = H->nodes[root.ch[1]];
        root.B12 = (double*)H->arena.alloc(sizeof(double) * (size_t)std::max(a.r.k, 1) * std::max(b.c.k, 1));
        root.B21 = (double*)H->arena.alloc(sizeof(double) * (size_t)std::max(b.r.k, 1) * std::max(a.c.k, 1));
        if (!root.B12 || !root.B21) return fail(HSS_ERR_NOMEM, "device arena allocation failed (B)");
        add(a.r.I, 0, a.r.k, b.c.I, 0, b.c.k, root.B12, std::max(a.r.k, 1));
        add(b.r.I, 0, b.r.k, a.c.I, 0, a.c.k, root.B21, std::max(b.r.k, 1));
      }
    }
    root.state = HSS_COMPRESSED;
  }
  CKS(run_extract(c, ex));
  return HSS_OK;
}

// When d_max is reached with the root not COMPRESSED (Algorithm 3's loop
// ends there), the generators of the compressed subtrees stand, and the
// rest of A is kept as it is: for every node with children that is not
// COMPRESSED, the blocks A(I_nu1, I_nu2) and A(I_nu2, I_nu1) between its
// children (the leaves keep D).  The products and the dense expansion then
// reproduce A exactly outside the compressed subtrees.  The blocks take
// sum 2 |nu1| |nu2| doubles; when that exceeds half of the free device
// memory they are not kept and the handle holds no usable generators.
hss_status keep_dense_blocks(Ctx& c, hss_matrix_s* H) {
  double need = 0.0;
  for (auto& t : H->nodes)
    if (!t.leaf && t.state != HSS_COMPRESSED)
      need += 2.0 * 8.0 * (double)H->nodes[t.ch[0]].size * (double)H->nodes[t.ch[1]].size;
  size_t fr = 0, tot = 0;
  CK(cudaMemGetInfo(&fr, &tot));
  if (need > 0.5 * (double)fr) return HSS_OK;
  ExtractSet ex;
  for (auto& t : H->nodes) {
    if (t.leaf || t.state == HSS_COMPRESSED) continue;
    const Node& a = H->nodes[t.ch[0]];
    const Node& b = H->nodes[t.ch[1]];
    t.F12 = (double*)H->arena.alloc(sizeof(double) * (size_t)a.size * b.size);
    t.F21 = (double*)H->arena.alloc(sizeof(double) * (size_t)b.size * a.size);
    if (!t.F12 || !t.F21) return fail(HSS_ERR_NOMEM, "device allocation of the uncompressed blocks failed");
    ExtractJob e;
    memset(&e, 0, sizeof e);
    e.i0 = a.lo; e.mi = a.size; e.j0 = b.lo; e.nj = b.size; e.out = t.F12; e.ldo = a.size;
    ex.of(H).push_back(e);
    e.i0 = b.lo; e.mi = b.size; e.j0 = a.lo; e.nj = a.size; e.out = t.F21; e.ldo = b.size;
    ex.of(H).push_back(e);
  }
  CK(c.timer.mark(PH_MERGE, c.st));
  CKS(run_extract(c, ex));
  H->partial = true;
  return HSS_OK;
}

// Everything a compression needs before its first pass: tree, leaf labels,
// sample and R buffers, and (with a user operator) the packed leaf blocks D.
hss_status setup(Ctx& c, const hss_source* A, const hss_opts* o, hss_matrix_s* H, ExtractSet& leafD) {
  const int n = A->n;
  H->n = n;
  H->o = *o;
  H->src = *A;
  H->dmax = std::min(o->d_max, n);
  CK(cudaGetDevice(&H->device));
  build_tree(n, o->leaf, H->nodes);
  H->max_level = 0;
  for (auto& t : H->nodes) H->max_level = std::max(H->max_level, t.level);
  H->by_level.assign(H->max_level + 1, {});
  for (size_t i = 0; i < H->nodes.size(); ++i) H->by_level[H->nodes[i].level].push_back((int)i);
  // leaf id per index, iota
  std::vector<int> lid(n), io(n);
  {
    int cnt = 0;
    for (auto& t : H->nodes)
      if (t.leaf) {
        for (int i = t.lo; i < t.lo + t.size; ++i) lid[i] = cnt;
        ++cnt;
      }
    for (int i = 0; i < n; ++i) io[i] = i;
  }
  const size_t nd = (size_t)n * H->dmax;
  H->leaf_id = (int*)H->arena.alloc(sizeof(int) * n);
  H->iota = (int*)H->arena.alloc(sizeof(int) * n);
  H->Sg_r = (double*)H->arena.alloc(sizeof(double) * nd);
  H->sym = o->symmetric != 0;
  H->Sg_c = H->sym ? H->Sg_r : (double*)H->arena.alloc(sizeof(double) * nd);
  const bool mixed = o->precision != HSS_PREC_FP64;
  H->own_R = (o->R == nullptr) || mixed;
  if (H->own_R) H->R = (double*)H->arena.alloc(sizeof(double) * nd);
  else H->R = const_cast<double*>(o->R);
  if (!H->leaf_id || !H->iota || !H->Sg_r || !H->Sg_c || !H->R)
    return fail(HSS_ERR_NOMEM, "device allocation of %zu bytes for samples failed", 3 * nd * 8);
  CKS(upload(c, H->leaf_id, lid.data(), sizeof(int) * n));
  CKS(upload(c, H->iota, io.data(), sizeof(int) * n));
  if (o->op) {
    std::vector<int> lb;
    for (auto& t : H->nodes)
      if (t.leaf) lb.push_back(t.lo);
    lb.push_back(n);
    H->leaf_lo = (int*)H->arena.alloc(sizeof(int) * lb.size());
    if (!H->leaf_lo) return fail(HSS_ERR_NOMEM, "device allocation of the leaf bounds failed");
    CKS(upload(c, H->leaf_lo, lb.data(), sizeof(int) * lb.size()));
    // the leaf blocks D_tau = A(I_tau, I_tau) first, packed: every sampling
    // pass removes D_tau R(I_tau) from the operator's product (Algorithm 2)
    std::vector<long long> off;
    long long tot = 0;
    for (auto& t : H->nodes)
      if (t.leaf) {
        off.push_back(tot);
        tot += (long long)t.size * t.size;
      }
    H->leaf_D = (double*)H->arena.alloc(sizeof(double) * (size_t)tot);
    H->leaf_doff = (long long*)H->arena.alloc(sizeof(long long) * off.size());
    if (!H->leaf_D || !H->leaf_doff) return fail(HSS_ERR_NOMEM, "device allocation of the leaf blocks failed");
    CKS(upload(c, H->leaf_doff, off.data(), sizeof(long long) * off.size()));
    size_t q = 0;
    for (auto& t : H->nodes)
      if (t.leaf) {
        t.D = H->leaf_D + off[q++];
        ExtractJob e;
        memset(&e, 0, sizeof e);
        e.i0 = t.lo; e.mi = t.size; e.j0 = t.lo; e.nj = t.size; e.out = t.D; e.ldo = t.size;
        leafD.of(H).push_back(e);
      }
  }
  H->d = std::min(o->d0, H->dmax);
  H->d_prev = 0;
  H->bounds.assign(1, H->d);
  return HSS_OK;
}

// HSSCompressAdaptive (Algorithm 3) for a list of matrices in lockstep: all
// first samples, then passes of the tree sweep (run_pass) over the matrices
// that are not done, each followed by the growth of the sample of those
// whose root is not COMPRESSED (Doubling: d more columns; Incrementing: dd),
// until every root is COMPRESSED or at d_max.  One read-back of the sampling
// flags per round of sampling.
hss_status compress_all(Ctx& c, const std::vector<const hss_source*>& A, const std::vector<const hss_opts*>& O,
                        std::vector<hss_matrix_s*>& Hs) {
  CKS(c.flags((int)Hs.size()));
  CK(c.timer.mark(PH_OTHER, c.st));
  ExtractSet leafD;
  for (size_t i = 0; i < Hs.size(); ++i) {
    Hs[i]->slot = (int)i;
    CKS(setup(c, A[i], O[i], Hs[i], leafD));
  }
  if (!leafD.per.empty()) {
    CK(c.timer.mark(PH_MERGE, c.st));
    CKS(run_extract(c, leafD));
  }
  for (hss_matrix_s* H : Hs) CKS(sample_columns(c, H, 0, H->d));
  CKS(sample_check(c, Hs));
  std::vector<hss_matrix_s*> act = Hs;
  while (!act.empty()) {
    CKS(run_pass(c, act));
    std::vector<hss_matrix_s*> next;
    for (hss_matrix_s* H : act) {
      if (H->nodes[0].state == HSS_COMPRESSED) { H->converged = 1; H->done = true; continue; }
      if (H->d >= H->dmax) { H->done = true; continue; }
      int dd = (H->o.strategy == HSS_DOUBLING) ? H->d : H->o.dd;
      dd = std::min(dd, H->dmax - H->d);
      CKS(sample_columns(c, H, H->d, H->d + dd));
      H->d_prev = H->d;
      H->d += dd;
      H->bounds.push_back(H->d);
      H->n_adapt++;
      next.push_back(H);
    }
    if (!next.empty()) CKS(sample_check(c, next));
    act.swap(next);
  }
  CK(c.timer.mark(PH_OTHER, c.st));
  for (hss_matrix_s* H : Hs) {
    if (H->packA) {
      CK(cudaFreeAsync(H->packA, c.st));
      H->packA = nullptr;
    }
    if (H->toep_terms) {
      CK(cudaFreeAsync(H->toep_terms, c.st));
      H->toep_terms = nullptr;
    }
    if (!H->converged) CKS(keep_dense_blocks(c, H));
  }
  CKS(readback(c, c.d_flag + 3, sizeof(int)));
  if (c.h_pinned[0]) return fail(HSS_ERR_TIMEOUT, "tensor-core tile product gave up waiting (code %d)", c.h_pinned[0]);
  double ph[PH_N];
  c.timer.sum(ph, PH_N);
  for (size_t i = 0; i < Hs.size(); ++i) {
    hss_matrix_s* H = Hs[i];
    H->d_final = H->d;
    H->usable = H->converged != 0 || H->partial;
    // the phases of a batched call are shared by its matrices; the launch and
    // byte counts are the call's, reported with its first matrix
    H->st.ms_sample = ph[PH_SAMPLE];
    H->st.ms_rng = ph[PH_RNG];
    H->st.ms_id = ph[PH_ID];
    H->st.ms_test = ph[PH_TEST];
    H->st.ms_merge = ph[PH_MERGE] + ph[PH_OTHER];
    H->st.ms_total = ph[PH_N - 1];
    H->st.launches = i == 0 ? c.launches : 0;
    H->st.bytes_h2d = i == 0 ? c.bytes_h2d : 0;
    H->st.bytes_d2h = i == 0 ? c.bytes_d2h : 0;
    H->st.n = H->n;
    H->st.n_nodes = (int)H->nodes.size();
    H->st.levels = H->max_level + 1;
    H->st.d_final = H->d_final;
    H->st.n_adapt = H->n_adapt;
    H->st.converged = H->converged;
    for (size_t q = 1; q < H->nodes.size(); ++q) {
      H->st.max_rank_r = std::max(H->st.max_rank_r, H->nodes[q].r.k);
      H->st.max_rank_c = std::max(H->st.max_rank_c, H->nodes[q].c.k);
    }
  }
  return HSS_OK;
}

hss_status check_opts(const hss_source* A, const hss_opts* o) {
  CKS(check_source(A));
  if (!o) return fail(HSS_ERR_ARG, "opts is NULL");
  if (o->leaf < 1) return fail(HSS_ERR_ARG, "leaf must be >= 1 (got %d)", o->leaf);
  if (o->d0 < 1 || o->d_max < 1) return fail(HSS_ERR_ARG, "d0 and d_max must be >= 1");
  if (o->strategy != HSS_DOUBLING && o->strategy != HSS_INCREMENTING)
    return fail(HSS_ERR_ARG, "unknown strategy %d", o->strategy);
  if (o->strategy == HSS_INCREMENTING && o->dd < 1) return fail(HSS_ERR_ARG, "dd must be >= 1");
  if (o->precision < HSS_PREC_FP64 || o->precision > HSS_PREC_BF16X3)
    return fail(HSS_ERR_ARG, "unknown precision %d", o->precision);
  if (!(o->rtol >= 0.0) || !(o->atol >= 0.0)) return fail(HSS_ERR_ARG, "tolerances must be >= 0");
  if (o->wait_limit_ns < 0) return fail(HSS_ERR_ARG, "wait_limit_ns must be >= 0");
  if (o->oversample_p < 0) return fail(HSS_ERR_ARG, "oversample_p must be >= 0");
  if (o->op && (!o->op->apply || o->precision != HSS_PREC_FP64))
    return fail(HSS_ERR_ARG, "a user operator needs an apply function and HSS_PREC_FP64");
  if (A->kind == HSS_SRC_EXTRACT && !o->op)
    return fail(HSS_ERR_ARG, "an extraction source is sampled through a user operator (opts->op)");
  if (o->criterion != HSS_CRIT_NEW && o->criterion != HSS_CRIT_HMT)
    return fail(HSS_ERR_ARG, "unknown criterion %d", o->criterion);
  if (o->criterion == HSS_CRIT_HMT) {
    if (o->strategy != HSS_INCREMENTING)
      return fail(HSS_ERR_ARG, "the HMT criterion is a test of the Incrementing strategy");
    if (!(o->hmt_alpha > 1.0) || !std::isfinite(o->hmt_alpha))
      return fail(HSS_ERR_ARG, "hmt_alpha must be finite and > 1 (got %g)", o->hmt_alpha);
  }
  return HSS_OK;
}

}  // namespace

// ======================================================================= ABI
// ------------------------------------------------ checkpoint of generators
namespace {
constexpr char kMagic[8] = {'H', 'S', 'S', 'G', 'E', 'N', '0', '1'};

bool put(FILE* f, const void* p, size_t bytes) { return bytes == 0 || fwrite(p, 1, bytes, f) == bytes; }
bool get(FILE* f, void* p, size_t bytes) { return bytes == 0 || fread(p, 1, bytes, f) == bytes; }

// one device array: its element count (-1 when absent), then the elements.
// Returns 0, or 1 on a write failure, 2 on a failed device copy.
template <class T>
int put_array(FILE* f, const T* dev, long long count) {
  const long long c = dev ? count : -1;
  if (!put(f, &c, sizeof c)) return 1;
  if (c <= 0) return 0;
  std::vector<T> h((size_t)c);
  if (cudaMemcpy(h.data(), dev, sizeof(T) * (size_t)c, cudaMemcpyDeviceToHost) != cudaSuccess) return 2;
  return put(f, h.data(), sizeof(T) * (size_t)c) ? 0 : 1;
}

// Reads one array into host memory: its element count must be `want`
// (-1: absent), or any count in [0, max_count] when want == -2 (checked by
// the caller afterwards); *present tells whether it was there.
template <class T>
bool get_array(FILE* f, std::vector<T>& h, bool* present, long long want, long long max_count = 0) {
  long long c = 0;
  if (!get(f, &c, sizeof c)) return false;
  if (want == -2 ? (c < 0 || c > max_count) : c != want) return false;
  *present = c >= 0;
  h.clear();
  if (c <= 0) return true;
  h.resize((size_t)c);
  return get(f, h.data(), sizeof(T) * (size_t)c);
}

template <class T>
hss_status upload_array(Arena& arena, const std::vector<T>& h, bool present, T** dev) {
  *dev = nullptr;
  if (!present) return HSS_OK;
  *dev = (T*)arena.alloc(sizeof(T) * std::max<size_t>(h.size(), 1));
  if (!*dev) return fail(HSS_ERR_NOMEM, "device allocation for a checkpoint array failed");
  if (!h.empty()) CK(cudaMemcpy(*dev, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
  return HSS_OK;
}
}  // namespace

extern "C" {

const char* hss_status_str(hss_status s) {
  switch (s) {
    case HSS_OK: return "HSS_OK";
    case HSS_ERR_ARG: return "HSS_ERR_ARG";
    case HSS_ERR_NOMEM: return "HSS_ERR_NOMEM";
    case HSS_ERR_CUDA: return "HSS_ERR_CUDA";
    case HSS_ERR_NOT_CONVERGED: return "HSS_ERR_NOT_CONVERGED";
    case HSS_ERR_NONFINITE: return "HSS_ERR_NONFINITE";
    case HSS_ERR_TIMEOUT: return "HSS_ERR_TIMEOUT";
    case HSS_ERR_UNSUPPORTED: return "HSS_ERR_UNSUPPORTED";
    case HSS_ERR_OPERATOR: return "HSS_ERR_OPERATOR";
    case HSS_ERR_IO: return "HSS_ERR_IO";
  }
  return "HSS_ERR_UNKNOWN";
}

const char* hss_last_error(void) { return g_err.c_str(); }

hss_status hss_compress(const hss_source* A, const hss_opts* o, void* stream, hss_matrix* out) {
  if (!out) return fail(HSS_ERR_ARG, "out is NULL");
  *out = nullptr;
  CKS(check_opts(A, o));
  cudaStream_t st = (cudaStream_t)stream;
  hss_matrix_s* H = new (std::nothrow) hss_matrix_s();
  if (!H) return fail(HSS_ERR_NOMEM, "host allocation failed");
  hss_status s;
  {
    Ctx c(st);
    std::vector<hss_matrix_s*> Hs{H};
    s = compress_all(c, {A}, {o}, Hs);
  }
  if (s != HSS_OK) {
    cudaStreamSynchronize(st);
    delete H;
    return s;
  }
  *out = H;
  if (!H->converged)
    return fail(HSS_ERR_NOT_CONVERGED, "root not compressed at d = d_max = %d", H->d_final);
  return HSS_OK;
}

hss_status hss_compress_restart(const hss_source* A, const hss_opts* o, void* stream, hss_matrix* out,
                                int* restarts) {
  if (restarts) *restarts = 0;
  if (!A || !o || !out) return fail(HSS_ERR_ARG, "NULL argument");
  *out = nullptr;
  const int cap = std::min(o->d_max, A->n);
  hss_opts a = *o;
  int d = std::min(o->d0, cap), k = 0;
  for (;;) {
    a.d0 = a.d_max = d;
    hss_matrix H = nullptr;
    const hss_status s = hss_compress(A, &a, stream, &H);
    if (s != HSS_ERR_NOT_CONVERGED || d >= cap) {   // converged, failed, or the last attempt
      *out = H;
      if (restarts) *restarts = k;
      return s;
    }
    hss_free(H);
    d = (int)std::min<long long>(2LL * d, cap);
    ++k;
  }
}

hss_status hss_compress_batched(const hss_source* A, const hss_opts* opts, int count, void* stream,
                                hss_matrix* out) {
  if (count < 0) return fail(HSS_ERR_ARG, "count must be >= 0 (got %d)", count);
  if (count == 0) return HSS_OK;
  if (!A || !opts || !out) return fail(HSS_ERR_ARG, "NULL argument");
  for (int i = 0; i < count; ++i) out[i] = nullptr;
  for (int i = 0; i < count; ++i) {
    hss_status s = check_opts(&A[i], &opts[i]);
    if (s != HSS_OK) return fail(s, "matrix %d: %s", i, g_err.c_str());
  }
  cudaStream_t st = (cudaStream_t)stream;
  // Groups of matrices compressed in lockstep, each group's estimated device
  // memory (samples, R, bases, packed tensor-core operand) within 60 % of
  // the free memory; largest first.
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return A[a].n > A[b].n; });
  auto footprint = [&](int i) {
    const double n = A[i].n, dm = std::min(opts[i].d_max, A[i].n);
    double b = 8.0 * n * dm * (opts[i].symmetric ? 3.0 : 4.0);      // R, S^r, S^c, node samples
    if (opts[i].strategy == HSS_INCREMENTING) b += 8.0 * n * dm * 2.0;   // bases Q
    if (opts[i].precision != HSS_PREC_FP64 && A[i].kind == HSS_SRC_DENSE)
      b += (double)packed_a_bytes(A[i].n, opts[i].precision);
    return b;
  };
  size_t fr = 0, tot = 0;
  CK(cudaMemGetInfo(&fr, &tot));
  // memory the library already holds for reuse counts as free: the idle
  // part of its work-buffer pool and the cached arena chunks of this device
  double avail = (double)fr;
  {
    cudaMemPool_t pool = nullptr;
    unsigned long long res = 0, used = 0;
    if (lib_pool(&pool) == cudaSuccess &&
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &res) == cudaSuccess &&
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess && res > used)
      avail += (double)(res - used);
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) {
      ChunkCache& cc = chunk_cache();
      std::lock_guard<std::mutex> lock(cc.mu);
      avail += (double)cc.held[dev];
    }
  }
  const double budget = 0.6 * avail;
  hss_status first = HSS_OK;
  int at = -1;
  for (size_t g0 = 0; g0 < order.size() && first == HSS_OK;) {
    size_t g1 = g0;
    double used = 0.0;
    while (g1 < order.size() && (g1 == g0 || used + footprint(order[g1]) <= budget)) used += footprint(order[g1++]);
    std::vector<hss_matrix_s*> Hs;
    std::vector<const hss_source*> As;
    std::vector<const hss_opts*> Os;
    for (size_t q = g0; q < g1; ++q) {
      hss_matrix_s* H = new (std::nothrow) hss_matrix_s();
      if (!H) { first = fail(HSS_ERR_NOMEM, "host allocation failed"); break; }
      out[order[q]] = H;
      Hs.push_back(H);
      As.push_back(&A[order[q]]);
      Os.push_back(&opts[order[q]]);
    }
    if (first != HSS_OK) break;
    Ctx c(st);
    first = compress_all(c, As, Os, Hs);
    if (first != HSS_OK) at = order[g0];
    g0 = g1;
  }
  if (first != HSS_OK) {
    const std::string msg = g_err;
    cudaStreamSynchronize(st);
    for (int i = 0; i < count; ++i) {
      hss_free(out[i]);
      out[i] = nullptr;
    }
    return fail(first, "batch group starting at matrix %d: %s", at, msg.c_str());
  }
  for (int i = 0; i < count; ++i)
    if (!out[i]->converged) return fail(HSS_ERR_NOT_CONVERGED, "matrix %d: root not compressed at d_max", i);
  return HSS_OK;
}

void hss_free(hss_matrix H) { delete H; }

hss_status hss_set_tuning(const hss_tuning* t) {
  const hss_tuning def{8, 4, 2, 4, 0};
  if (t && (t->qrcp_wide_max_sides < 1 || t->sample_waves_packed < 1 || t->sample_waves_generated < 1 ||
            t->qrcp_min_cols < 1))
    return fail(HSS_ERR_ARG, "tuning values must be >= 1");
  if (t && t->qrcp_sm_ctas != 0 && t->qrcp_sm_ctas != 1 && t->qrcp_sm_ctas != 2 && t->qrcp_sm_ctas != 4)
    return fail(HSS_ERR_ARG, "qrcp_sm_ctas must be 0, 1, 2 or 4");
  std::lock_guard<std::mutex> lock(tuning_mutex());
  tuning_ref() = t ? *t : def;
  return HSS_OK;
}

hss_status hss_get_tuning(hss_tuning* t) {
  if (!t) return fail(HSS_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lock(tuning_mutex());
  *t = tuning_ref();
  return HSS_OK;
}

hss_status hss_release_cached(void) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  ChunkCache& c = chunk_cache();
  std::lock_guard<std::mutex> lock(c.mu);
  for (size_t i = 0; i < c.free.size();) {
    if (c.free[i].first == dev) {
      cudaFree(c.free[i].second);
      c.free.erase(c.free.begin() + i);
    } else {
      ++i;
    }
  }
  if (dev >= 0 && dev < 64) c.held[dev] = 0;
  // and the work-buffer pool's reserved memory, once the device is idle
  cudaMemPool_t pool = nullptr;
  CK(lib_pool(&pool));
  CK(cudaDeviceSynchronize());
  CK(cudaMemPoolTrimTo(pool, 0));
  return HSS_OK;
}


hss_status hss_save(hss_matrix H, const char* path) {
  if (!H || !path) return fail(HSS_ERR_ARG, "NULL argument");
  if (!H->usable || !H->converged)
    return fail(HSS_ERR_ARG, "only a converged handle can be saved");
  // written to path.tmp and renamed into place once complete, so a failed
  // save never leaves a partial file at path
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = fopen(tmp.c_str(), "wb");
  if (!f) return fail(HSS_ERR_IO, "cannot open %s for writing", tmp.c_str());
  const int hdr[8] = {H->n, (int)H->nodes.size(), H->max_level, H->usable ? 1 : 0, H->converged, H->d_final,
                      H->n_adapt, H->o.leaf};
  const long long sst = (long long)sizeof(hss_stats);
  int err = (put(f, kMagic, sizeof kMagic) && put(f, hdr, sizeof hdr) && put(f, &sst, sizeof sst) &&
             put(f, &H->st, sizeof(hss_stats))) ? 0 : 1;
  for (size_t i = 0; !err && i < H->nodes.size(); ++i) {
    const Node& t = H->nodes[i];
    const int rec[12] = {t.lo, t.size, t.level, t.parent, t.ch[0], t.ch[1], t.leaf ? 1 : 0, t.state,
                         t.r.m, t.r.k, t.c.m, t.c.k};
    err = put(f, rec, sizeof rec) ? 0 : 1;
    for (const Side* sd : {&t.r, &t.c}) {
      if (!err) err = put_array(f, i ? sd->piv : (int*)nullptr, sd->m);
      if (!err) err = put_array(f, i ? sd->X : (double*)nullptr, (long long)sd->k * (sd->m - sd->k));
      if (!err) err = put_array(f, i ? sd->I : (int*)nullptr, sd->k);
    }
    long long nb12 = 0, nb21 = 0;
    if (!t.leaf) {
      const Node& a = H->nodes[t.ch[0]];
      const Node& b = H->nodes[t.ch[1]];
      nb12 = (long long)a.r.k * b.c.k;
      nb21 = (long long)b.r.k * a.c.k;
    }
    if (!err) err = put_array(f, t.leaf ? t.D : (double*)nullptr, (long long)t.size * t.size);
    if (!err) err = put_array(f, t.leaf ? (double*)nullptr : t.B12, nb12);
    if (!err) err = put_array(f, t.leaf ? (double*)nullptr : t.B21, nb21);
  }
  if (fclose(f) != 0 && !err) err = 1;
  if (!err && rename(tmp.c_str(), path) != 0) err = 1;
  if (err) {
    remove(tmp.c_str());
    return err == 2 ? fail(HSS_ERR_CUDA, "copying the generators to the host failed")
                    : fail(HSS_ERR_IO, "writing %s failed", path);
  }
  return HSS_OK;
}

hss_status hss_load(const char* path, hss_matrix* out) {
  if (!path || !out) return fail(HSS_ERR_ARG, "NULL argument");
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) return fail(HSS_ERR_IO, "cannot open %s", path);
  // The whole file is read and checked on the host first; nothing reaches
  // the device unless every count, index and pivot is consistent.
  char magic[8];
  int hdr[8];
  long long sst = 0;
  hss_stats st{};
  bool ok = get(f, magic, sizeof magic) && memcmp(magic, kMagic, sizeof kMagic) == 0 && get(f, hdr, sizeof hdr) &&
            get(f, &sst, sizeof sst) && sst == (long long)sizeof(hss_stats) && get(f, &st, sizeof(hss_stats));
  const int n = ok ? hdr[0] : 0, leaf = ok ? hdr[7] : 0;
  // the tree must be the halving tree of (n, leaf) the saver used, node by node
  std::vector<Node> tree;
  int max_level = 0;
  ok = ok && n > 0 && leaf >= 1 && hdr[3] == 1 && hdr[4] == 1;
  if (ok) {
    build_tree(n, leaf, tree);
    for (auto& t : tree) max_level = std::max(max_level, t.level);
    ok = (int)tree.size() == hdr[1] && hdr[2] == max_level;
  }
  const int nn = ok ? (int)tree.size() : 0;
  struct HostSide { std::vector<int> piv, I; std::vector<double> X; bool hp = false, hx = false, hi = false; };
  struct HostNode { HostSide sd[2]; std::vector<double> D, B12, B21; bool hd = false, hb12 = false, hb21 = false; };
  std::vector<HostNode> hn(nn);
  for (int i = 0; ok && i < nn; ++i) {
    Node& t = tree[i];
    int rec[12];
    ok = get(f, rec, sizeof rec);
    if (!ok) break;
    ok = rec[0] == t.lo && rec[1] == t.size && rec[2] == t.level && rec[3] == t.parent && rec[4] == t.ch[0] &&
         rec[5] == t.ch[1] && (rec[6] != 0) == t.leaf && rec[7] == HSS_COMPRESSED;
    t.state = HSS_COMPRESSED;
    t.r.m = rec[8]; t.r.k = rec[9]; t.c.m = rec[10]; t.c.k = rec[11];
    if (i == 0) ok = ok && t.r.m == 0 && t.r.k == 0 && t.c.m == 0 && t.c.k == 0;
    else
      ok = ok && t.r.k >= 0 && t.r.k <= t.r.m && t.c.k >= 0 && t.c.k <= t.c.m && t.r.m <= t.size &&
           t.c.m <= t.size && (!t.leaf || (t.r.m == t.size && t.c.m == t.size));
    for (int q = 0; q < 2 && ok; ++q) {
      const Side& sd = q ? t.c : t.r;
      HostSide& h = hn[i].sd[q];
      const int m = sd.m, k = sd.k;
      ok = get_array(f, h.piv, &h.hp, i ? m : -1) && get_array(f, h.X, &h.hx, i ? (long long)k * (m - k) : -1) &&
           get_array(f, h.I, &h.hi, i ? k : -1);
      // the pivots a permutation of [0, m), the skeleton indices inside the
      // node's index range
      std::vector<char> seen((size_t)std::max(m, 0), 0);
      for (int v : h.piv) {
        if (!ok) break;
        ok = v >= 0 && v < m && !seen[(size_t)v];
        if (ok) seen[(size_t)v] = 1;
      }
      for (int v : h.I) ok = ok && v >= t.lo && v < t.lo + t.size;
    }
    HostNode& h = hn[i];
    ok = ok && get_array(f, h.D, &h.hd, t.leaf ? (long long)t.size * t.size : -1) &&
         get_array(f, h.B12, &h.hb12, t.leaf ? -1 : -2, (long long)n * n) &&
         get_array(f, h.B21, &h.hb21, t.leaf ? -1 : -2, (long long)n * n);
  }
  // the sample rows and the B blocks agree with the children's ranks (the
  // products index with them)
  for (int i = 0; ok && i < nn; ++i) {
    const Node& t = tree[i];
    if (t.leaf) continue;
    const Node& a = tree[t.ch[0]];
    const Node& b = tree[t.ch[1]];
    ok = hn[i].B12.size() == (size_t)a.r.k * b.c.k && hn[i].B21.size() == (size_t)b.r.k * a.c.k;
    if (i > 0) ok = ok && t.r.m == a.r.k + b.r.k && t.c.m == a.c.k + b.c.k;
  }
  // nothing may follow the last node
  char extra;
  ok = ok && fread(&extra, 1, 1, f) == 0;
  fclose(f);
  if (!ok) return fail(HSS_ERR_ARG, "%s is not a readable HSS generator checkpoint", path);

  hss_matrix_s* H = new (std::nothrow) hss_matrix_s();
  if (!H) return fail(HSS_ERR_NOMEM, "host allocation failed");
  H->n = n;
  H->max_level = max_level;
  H->usable = true;
  H->converged = 1;
  H->d_final = hdr[5];
  H->n_adapt = hdr[6];
  H->o.leaf = leaf;
  H->st = st;
  H->st.n = n;
  H->st.n_nodes = nn;
  H->st.levels = max_level + 1;
  H->nodes = tree;
  H->by_level.assign(max_level + 1, {});
  hss_status e = cudaGetDevice(&H->device) == cudaSuccess ? HSS_OK : fail(HSS_ERR_CUDA, "no CUDA device");
  for (int i = 0; e == HSS_OK && i < nn; ++i) {
    Node& t = H->nodes[i];
    for (int q = 0; q < 2 && e == HSS_OK; ++q) {
      Side& sd = q ? t.c : t.r;
      const HostSide& h = hn[i].sd[q];
      e = upload_array(H->arena, h.piv, h.hp, &sd.piv);
      if (e == HSS_OK) e = upload_array(H->arena, h.X, h.hx, &sd.X);
      if (e == HSS_OK) e = upload_array(H->arena, h.I, h.hi, &sd.I);
    }
    if (e == HSS_OK) e = upload_array(H->arena, hn[i].D, hn[i].hd, &t.D);
    if (e == HSS_OK) e = upload_array(H->arena, hn[i].B12, hn[i].hb12, &t.B12);
    if (e == HSS_OK) e = upload_array(H->arena, hn[i].B21, hn[i].hb21, &t.B21);
    H->by_level[t.level].push_back(i);
  }
  if (e != HSS_OK) {
    delete H;
    return e;
  }
  *out = H;
  return HSS_OK;
}

hss_status hss_get_stats(hss_matrix H, hss_stats* s) {
  if (!H || !s) return fail(HSS_ERR_ARG, "NULL argument");
  *s = H->st;
  return HSS_OK;
}

hss_status hss_get_node(hss_matrix H, int node, hss_node_info* info) {
  if (!H || !info) return fail(HSS_ERR_ARG, "NULL argument");
  if (node < 0 || node >= (int)H->nodes.size()) return fail(HSS_ERR_ARG, "node %d out of range", node);
  const Node& t = H->nodes[node];
  info->lo = t.lo; info->size = t.size; info->level = t.level; info->parent = t.parent;
  info->child0 = t.ch[0]; info->child1 = t.ch[1]; info->state = t.state;
  info->mr = t.r.m; info->mc = t.c.m; info->kr = t.r.k; info->kc = t.c.k;
  return HSS_OK;
}

hss_status hss_export_node(hss_matrix H, int node, int* Jr, int* Jc, int* Pr, int* Pc, double* Xr,
                           double* Xc, int* Ir, int* Ic, double* D, double* B12, double* B21) {
  if (!H) return fail(HSS_ERR_ARG, "NULL handle");
  if (node < 0 || node >= (int)H->nodes.size()) return fail(HSS_ERR_ARG, "node %d out of range", node);
  const Node& t = H->nodes[node];
  auto cp = [&](void* dst, const void* src, size_t bytes) -> hss_status {
    if (!dst || !bytes) return HSS_OK;
    if (!src) return fail(HSS_ERR_ARG, "node %d has no such generator", node);
    CK(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
    return HSS_OK;
  };
  if (t.state == HSS_COMPRESSED && node != 0) {
    CKS(cp(Jr, t.r.piv, sizeof(int) * t.r.k));
    CKS(cp(Jc, t.c.piv, sizeof(int) * t.c.k));
    CKS(cp(Pr, t.r.piv, sizeof(int) * t.r.m));
    CKS(cp(Pc, t.c.piv, sizeof(int) * t.c.m));
    CKS(cp(Xr, t.r.X, sizeof(double) * (size_t)t.r.k * (t.r.m - t.r.k)));
    CKS(cp(Xc, t.c.X, sizeof(double) * (size_t)t.c.k * (t.c.m - t.c.k)));
    CKS(cp(Ir, t.r.I, sizeof(int) * t.r.k));
    CKS(cp(Ic, t.c.I, sizeof(int) * t.c.k));
  }
  if (t.leaf) CKS(cp(D, t.D, sizeof(double) * (size_t)t.size * t.size));
  if (!t.leaf && t.state == HSS_COMPRESSED) {
    const Node& a = H->nodes[t.ch[0]];
    const Node& b = H->nodes[t.ch[1]];
    CKS(cp(B12, t.B12, sizeof(double) * (size_t)a.r.k * b.c.k));
    CKS(cp(B21, t.B21, sizeof(double) * (size_t)b.r.k * a.c.k));
  }
  return HSS_OK;
}

hss_status hss_to_dense(hss_matrix H, double* out, long long ld, void* stream) {
  if (!H || !out) return fail(HSS_ERR_ARG, "NULL argument");
  if (!H->usable) return fail(HSS_ERR_ARG, "handle holds no usable generators");
  if (ld < H->n) return fail(HSS_ERR_ARG, "ld %lld < n %d", ld, H->n);
  cudaStream_t st = (cudaStream_t)stream;
  const int n = H->n, blk = std::min(n, 2048);
  double* X = nullptr;
  CK(dmalloc_async((void**)&X, sizeof(double) * (size_t)n * blk, st));
  for (int c0 = 0; c0 < n; c0 += blk) {
    const int w = std::min(blk, n - c0);
    hss_status e = HSS_OK;
    if (launch_identity_block(X, n, c0, w, st) != cudaSuccess)
      e = fail(HSS_ERR_CUDA, "identity block launch failed");
    if (e == HSS_OK) e = hss_matvec(H, w, X, n, out + (long long)c0 * ld, ld, 0, stream);
    if (e != HSS_OK) {
      cudaFreeAsync(X, st);
      return e;
    }
  }
  CK(cudaFreeAsync(X, st));
  CK(cudaStreamSynchronize(st));
  return HSS_OK;
}

hss_status hss_matvec(hss_matrix H, int nrhs, const double* X, long long ldx, double* Y,
                      long long ldy, int transpose, void* stream) {
  if (!H || !X || !Y) return fail(HSS_ERR_ARG, "NULL argument");
  if (!H->usable) return fail(HSS_ERR_ARG, "handle holds no usable generators");
  if (nrhs < 0 || ldx < H->n || ldy < H->n) return fail(HSS_ERR_ARG, "bad nrhs / leading dimension");
  if (transpose != 0 && transpose != 1) return fail(HSS_ERR_ARG, "transpose must be 0 or 1");
  if (nrhs == 0) return HSS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  Ctx c(st);
  const bool tr = transpose != 0;
  const int nn = (int)H->nodes.size();
  // H^T has the roles of U and V exchanged, D^T at the leaves and
  // B12' = B21^T, B21' = B12^T: the up-sweep runs with the "in" side
  // (V for H, U for H^T), the down-sweep with the "out" side
  auto in_side = [&](const Node& t) -> const Side& { return tr ? t.r : t.c; };
  auto out_side = [&](const Node& t) -> const Side& { return tr ? t.c : t.r; };
  // per-node x^ (in-side k x nrhs) and y^ (out-side k x nrhs), row-major
  std::vector<size_t> offx(nn), offy(nn);
  size_t tot = 0;
  for (int i = 1; i < nn; ++i) {
    offx[i] = tot; tot += (size_t)in_side(H->nodes[i]).k * nrhs;
    offy[i] = tot; tot += (size_t)out_side(H->nodes[i]).k * nrhs;
  }
  double* buf = nullptr;
  CK(dmalloc_async((void**)&buf, sizeof(double) * std::max<size_t>(tot, 1), st));
  auto xh = [&](int i) { return buf + offx[i]; };
  auto yh = [&](int i) { return buf + offy[i]; };
  const long long R_ = nrhs;
  // up-sweep: x^_tau = V_tau^T [x(I_tau) | x^_nu1; x^_nu2]
  for (int lev = H->max_level; lev >= 1; --lev) {
    std::vector<GemmJob> jobs;
    for (int id : H->by_level[lev]) {
      Node& t = H->nodes[id];
      const Side& s = in_side(t);
      if (s.k <= 0) continue;
      Opnd x = t.leaf ? opnd(X + t.lo, 1, ldx)
                      : opnd(xh(t.ch[0]), R_, 1, nullptr, xh(t.ch[1]), in_side(H->nodes[t.ch[0]]).k);
      GemmJob j = gemm_job();
      j.M = s.k; j.N = nrhs; j.K = s.m - s.k;
      j.C0 = x; j.C0.rows = s.piv; j.beta = 1.0;
      j.A = opnd(s.X, 1, std::max(s.k, 1));
      j.B = x; j.B.rows = s.piv + s.k;
      j.C = xh(id); j.c_rs = R_; j.c_cs = 1;
      jobs.push_back(j);
    }
    hss_status e = run_gemms(c, jobs);
    if (e != HSS_OK) { cudaFreeAsync(buf, st); return e; }
  }
  // down-sweep; nodes that are not COMPRESSED (a partial result) couple
  // their children through the dense blocks instead (after the leaves)
  std::vector<std::vector<GemmJob>> dense(H->max_level + 1);
  for (int lev = 0; lev < H->max_level; ++lev) {
    std::vector<GemmJob> p0, p1;
    for (int id : H->by_level[lev]) {
      Node& t = H->nodes[id];
      if (t.leaf) continue;
      const int a = t.ch[0], b = t.ch[1];
      const Node& na = H->nodes[a];
      const Node& nb = H->nodes[b];
      const bool root = (id == 0);
      const Side& ts = out_side(t);
      if (t.state != HSS_COMPRESSED) {
        // y^ of the children starts at zero; Y(I_nu1) += A12 X(I_nu2),
        // Y(I_nu2) += A21 X(I_nu1) (transposed: A21^T, A12^T)
        for (int c : {a, b}) {
          const Side& cs = out_side(H->nodes[c]);
          if (cs.k <= 0) continue;
          GemmJob z = gemm_job();
          z.M = cs.k; z.N = nrhs; z.K = 0; z.alpha = 0.0;
          z.C = yh(c); z.c_rs = R_; z.c_cs = 1;
          p1.push_back(z);
        }
        for (int q = 0; q < 2; ++q) {
          const Node& to = q ? nb : na;
          const Node& from = q ? na : nb;
          GemmJob g = gemm_job();
          g.M = to.size; g.N = nrhs; g.K = from.size;
          // A(I_to, I_from): F12 (to = nu1) or F21, col-major ld |I_to|;
          // its transpose is the other block read across
          const double* F = tr ? (q ? t.F12 : t.F21) : (q ? t.F21 : t.F12);
          g.A = tr ? opnd(F, from.size, 1) : opnd(F, 1, to.size);
          g.B = opnd(X + from.lo, 1, ldx);
          g.gamma = 1.0;
          g.C = Y + to.lo; g.c_rs = 1; g.c_cs = ldy;
          dense[lev].push_back(g);
        }
        continue;
      }
      if (!root && ts.k > 0) {
        // [y^_nu1; y^_nu2] = U_tau y^_tau, U = Pi [I; Xr^T]
        GemmJob c = gemm_job();
        c.M = ts.k; c.N = nrhs; c.K = 0;
        c.C0 = opnd(yh(id), R_, 1); c.beta = 1.0;
        c.C = yh(a); c.C2 = yh(b); c.c_split = out_side(na).k; c.c_rows = ts.piv;
        c.c_rs = R_; c.c_cs = 1;
        p0.push_back(c);
        if (ts.m > ts.k) {
          GemmJob g = gemm_job();
          g.M = ts.m - ts.k; g.N = nrhs; g.K = ts.k;
          g.A = opnd(ts.X, std::max(ts.k, 1), 1);
          g.B = opnd(yh(id), R_, 1);
          g.C = yh(a); g.C2 = yh(b); g.c_split = out_side(na).k; g.c_rows = ts.piv + ts.k;
          g.c_rs = R_; g.c_cs = 1;
          p0.push_back(g);
        }
      }
      const double gam = (root || ts.k == 0) ? 0.0 : 1.0;
      // y^_nu1 (+)= B12 x^_nu2 ; y^_nu2 (+)= B21 x^_nu1  (transposed:
      // B21^T x^_nu2 and B12^T x^_nu1; B12 is kr(nu1) x kc(nu2), ld max(kr(nu1), 1))
      const int ld12 = std::max(na.r.k, 1), ld21 = std::max(nb.r.k, 1);
      GemmJob g1 = gemm_job();
      g1.M = out_side(na).k; g1.N = nrhs; g1.K = in_side(nb).k;
      g1.A = tr ? opnd(t.B21, ld21, 1) : opnd(t.B12, 1, ld12);
      g1.B = opnd(xh(b), R_, 1);
      g1.gamma = gam;
      g1.C = yh(a); g1.c_rs = R_; g1.c_cs = 1;
      p1.push_back(g1);
      GemmJob g2 = gemm_job();
      g2.M = out_side(nb).k; g2.N = nrhs; g2.K = in_side(na).k;
      g2.A = tr ? opnd(t.B12, ld12, 1) : opnd(t.B21, 1, ld21);
      g2.B = opnd(xh(a), R_, 1);
      g2.gamma = gam;
      g2.C = yh(b); g2.c_rs = R_; g2.c_cs = 1;
      p1.push_back(g2);
    }
    hss_status e = run_gemms(c, p0);
    if (e == HSS_OK) e = run_gemms(c, p1);
    if (e != HSS_OK) { cudaFreeAsync(buf, st); return e; }
  }
  // leaves: Y(I) = D X(I) + U y^  (D^T and V y^ transposed)
  std::vector<GemmJob> l0, l1;
  for (int id = 0; id < nn; ++id) {
    Node& t = H->nodes[id];
    if (!t.leaf) continue;
    GemmJob g = gemm_job();
    g.M = t.size; g.N = nrhs; g.K = t.size;
    g.A = tr ? opnd(t.D, t.size, 1) : opnd(t.D, 1, t.size);
    g.B = opnd(X + t.lo, 1, ldx);
    g.C = Y + t.lo; g.c_rs = 1; g.c_cs = ldy;
    l0.push_back(g);
    const Side& ts = out_side(t);
    if (id == 0 || ts.k <= 0) continue;
    GemmJob c = gemm_job();
    c.M = ts.k; c.N = nrhs; c.K = 0;
    c.C0 = opnd(yh(id), R_, 1); c.beta = 1.0; c.gamma = 1.0;
    c.C = Y + t.lo; c.c_rows = ts.piv; c.c_rs = 1; c.c_cs = ldy;
    l1.push_back(c);
    if (ts.m > ts.k) {
      GemmJob e2 = gemm_job();
      e2.M = ts.m - ts.k; e2.N = nrhs; e2.K = ts.k;
      e2.A = opnd(ts.X, std::max(ts.k, 1), 1);
      e2.B = opnd(yh(id), R_, 1);
      e2.gamma = 1.0;
      e2.C = Y + t.lo; e2.c_rows = ts.piv + ts.k; e2.c_rs = 1; e2.c_cs = ldy;
      l1.push_back(e2);
    }
  }
  hss_status e = run_gemms(c, l0);
  if (e == HSS_OK) e = run_gemms(c, l1);
  // dense couplings of a partial result, one launch per level (the blocks
  // of one level write disjoint rows of Y)
  for (int lev = 0; lev <= H->max_level && e == HSS_OK; ++lev) e = run_gemms(c, dense[lev]);
  cudaFreeAsync(buf, st);
  return e;
}

hss_status hss_get_entries(hss_matrix H, int nr, const int* I, int nc, const int* J, double* out, long long ldo,
                           void* stream) {
  if (!H) return fail(HSS_ERR_ARG, "NULL handle");
  if (!H->usable) return fail(HSS_ERR_ARG, "handle holds no usable generators");
  if (nr < 0 || nc < 0 || ldo < std::max(nr, 1)) return fail(HSS_ERR_ARG, "bad sizes (nr %d, nc %d, ldo %lld)", nr, nc, ldo);
  if (nr == 0 || nc == 0) return HSS_OK;
  if (!I || !J || !out) return fail(HSS_ERR_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  const int nn = (int)H->nodes.size(), n = H->n;
  int kcap = 1;
  size_t ninv = 0;
  std::vector<int> leaf_of(n);
  for (int id = 0; id < nn; ++id) {
    const Node& t = H->nodes[id];
    kcap = std::max(kcap, std::max(t.r.k, t.c.k));
    if (id) ninv += (size_t)t.r.m + (size_t)t.c.m;
    if (t.leaf)
      for (int i = t.lo; i < t.lo + t.size; ++i) leaf_of[i] = id;
  }
  const int lp1 = H->max_level + 1;
  // rows and columns in chunks whose path vectors take at most 512 MB each
  // (and at most 65535 columns: one grid row per column)
  const long long per = (long long)lp1 * kcap;
  const int chunk =
      (int)std::max<long long>(1, std::min<long long>({(long long)std::max(nr, nc), (64LL << 20) / per, 65535LL}));
  const size_t b_nodes = Scratch::rnd(sizeof(EntryNode) * nn), b_inv = Scratch::rnd(sizeof(int) * std::max<size_t>(ninv, 1)),
               b_leaf = Scratch::rnd(sizeof(int) * n), b_vec = Scratch::rnd(sizeof(double) * (size_t)chunk * per);
  char* buf = nullptr;
  CK(dmalloc_async((void**)&buf, b_nodes + b_inv + b_leaf + 2 * b_vec + 256, st));
  EntryNode* dn = (EntryNode*)buf;
  int* inv = (int*)(buf + b_nodes);
  int* dleaf = (int*)(buf + b_nodes + b_inv);
  double* Wrow = (double*)(buf + b_nodes + b_inv + b_leaf);
  double* Vcol = Wrow + (size_t)chunk * per;
  int* err = (int*)(buf + b_nodes + b_inv + b_leaf + 2 * b_vec);
  std::vector<EntryNode> hn(nn);
  size_t o = 0;
  for (int id = 0; id < nn; ++id) {
    const Node& t = H->nodes[id];
    EntryNode& e = hn[id];
    memset(&e, 0, sizeof e);
    e.lo = t.lo; e.size = t.size; e.level = t.level; e.parent = t.parent; e.ch0 = t.ch[0]; e.ch1 = t.ch[1];
    e.state = t.state;
    e.D = t.D; e.B12 = t.B12; e.B21 = t.B21; e.F12 = t.F12; e.F21 = t.F21;
    if (id && t.state == HSS_COMPRESSED) {
      e.kr = t.r.k; e.kc = t.c.k; e.mr = t.r.m; e.mc = t.c.m;
      e.pivr = t.r.piv; e.pivc = t.c.piv; e.Xr = t.r.X; e.Xc = t.c.X;
      e.ipivr = inv + o; o += t.r.m;
      e.ipivc = inv + o; o += t.c.m;
    }
  }
  hss_status s = HSS_OK;
  Ctx c(st);
  auto run = [&]() -> hss_status {
    CK(cudaMemsetAsync(err, 0, sizeof(int), st));
    CK(cudaMemsetAsync(inv, 0xff, sizeof(int) * std::max<size_t>(ninv, 1), st));   // -1: no position
    CKS(upload(c, dn, hn.data(), sizeof(EntryNode) * nn));
    CKS(upload(c, dleaf, leaf_of.data(), sizeof(int) * n));
    CK(launch_inv_piv(dn, nn, err, st));
    for (int c0 = 0; c0 < nc; c0 += chunk) {
      const int w = std::min(chunk, nc - c0);
      CK(launch_entry_paths(dn, dleaf, n, J + c0, w, Vcol, kcap, lp1, 1, err, st));
      for (int r0 = 0; r0 < nr; r0 += chunk) {
        const int h = std::min(chunk, nr - r0);
        CK(launch_entry_paths(dn, dleaf, n, I + r0, h, Wrow, kcap, lp1, 0, err, st));
        CK(launch_entry_pairs(dn, dleaf, n, I + r0, h, J + c0, w, Wrow, Vcol, kcap, lp1,
                              out + r0 + (long long)c0 * ldo, ldo, st));
      }
    }
    int herr = 0;
    CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (herr == 1) return fail(HSS_ERR_ARG, "an index of I or J is outside [0, %d)", n);
    if (herr) return fail(HSS_ERR_CUDA, "inconsistent pivots in the handle (code %d)", herr);
    return HSS_OK;
  };
  s = run();
  cudaFreeAsync(buf, st);
  return s;
}

hss_status hss_rcb_order(const double* points, int n, int dim, long long ld, int leaf, int* perm) {
  if (!points || !perm || n <= 0 || dim <= 0 || ld < n || leaf < 1)
    return fail(HSS_ERR_ARG, "bad arguments to hss_rcb_order");
  for (int i = 0; i < n; ++i) perm[i] = i;
  std::vector<std::pair<int, int>> stack{{0, n}};
  std::vector<int> tmp;
  while (!stack.empty()) {
    auto [lo, m] = stack.back();
    stack.pop_back();
    if (m <= leaf) continue;
    int best = 0;
    double bext = -1.0;
    for (int c = 0; c < dim; ++c) {
      double mn = points[perm[lo] + c * ld], mx = mn;
      for (int i = lo + 1; i < lo + m; ++i) {
        double v = points[perm[i] + c * ld];
        mn = std::min(mn, v);
        mx = std::max(mx, v);
      }
      if (mx - mn > bext) { bext = mx - mn; best = c; }
    }
    const double* col = points + best * ld;
    std::sort(perm + lo, perm + lo + m, [&](int x, int y) {
      double a = col[x], b = col[y];
      return a < b || (a == b && x < y);
    });
    int h = m / 2;
    stack.push_back({lo + h, m - h});
    stack.push_back({lo, h});
  }
  return HSS_OK;
}

hss_status hss_random_normal(unsigned long long seed, int n, int col0, int ncols, double* R,
                             long long ldr, int round_mode, void* stream) {
  if (!R || n <= 0 || ncols < 0 || col0 < 0 || ldr < n || round_mode < 0 || round_mode > 2)
    return fail(HSS_ERR_ARG, "bad arguments to hss_random_normal");
  CK(launch_random_normal(seed, n, col0, ncols, R, ldr, round_mode, (cudaStream_t)stream));
  return HSS_OK;
}

hss_status hss_sample_offdiag(const hss_source* A, int leaf, int precision, int ncols, const double* R,
                              long long ldr, double* Sr, double* Sc, long long lds, void* stream) {
  CKS(check_source(A));
  if (A->kind == HSS_SRC_EXTRACT) return fail(HSS_ERR_ARG, "sampling needs a source with entries on the device");
  const int n = A->n;
  if (leaf < 1 || ncols < 0 || !R || ldr < n || lds < ncols)
    return fail(HSS_ERR_ARG, "bad arguments to hss_sample_offdiag");
  if (precision < HSS_PREC_FP64 || precision > HSS_PREC_BF16X3)
    return fail(HSS_ERR_ARG, "unknown precision %d", precision);
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<Node> nodes;
  build_tree(n, leaf, nodes);
  std::vector<int> lid(n);
  int cnt = 0;
  for (auto& t : nodes)
    if (t.leaf) {
      for (int i = t.lo; i < t.lo + t.size; ++i) lid[i] = cnt;
      ++cnt;
    }
  int* d_lid = nullptr;
  CK(dmalloc_async((void**)&d_lid, sizeof(int) * n, st));
  CK(cudaMemcpyAsync(d_lid, lid.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
  SrcDev s = make_src(*A, d_lid);
  if (precision == HSS_PREC_FP64) {
    CK(launch_sample_fp64(s, ncols, R, ldr, Sr, Sc, lds, st));
    CK(cudaFreeAsync(d_lid, st));
    return HSS_OK;
  }
  // mixed forms: R rounded once to the tensor format, K split with atomics
  double* Rr = nullptr;
  int* err = nullptr;
  CK(dmalloc_async((void**)&Rr, sizeof(double) * (size_t)n * std::max(ncols, 1), st));
  CK(dmalloc_async((void**)&err, sizeof(int), st));
  CK(cudaMemsetAsync(err, 0, sizeof(int), st));
  CK(launch_round_copy(R, ldr, Rr, n, n, ncols, precision == HSS_PREC_TF32X2 ? 1 : 2, st));
  void* pA = nullptr;
  void* pR = nullptr;
  void* tt = nullptr;
  const bool packed = A->kind == HSS_SRC_DENSE;
  CK(dmalloc_async(&pR, packed_r_bytes(n, ncols, precision), st));
  CK(launch_pack_r(Rr, n, n, ncols, precision, pR, st));
  if (packed) {
    CK(dmalloc_async(&pA, packed_a_bytes(n, precision), st));
    CK(launch_pack_a(s, leaf, precision, pA, st));
  } else if (A->kind == HSS_SRC_TOEPLITZ) {
    CK(dmalloc_async(&tt, toeplitz_terms_bytes(n, precision), st));
    CK(launch_toeplitz_terms(s, precision, tt, st));
  }
  for (int side = 0; side < 2; ++side) {
    double* S = side ? Sc : Sr;
    if (!S) continue;
    const int ks = packed ? sample_tc_packed_ksplit(n, ncols, precision) : sample_tc_ksplit(n, ncols, precision);
    if (ks > 1) CK(cudaMemset2DAsync(S, sizeof(double) * lds, 0, sizeof(double) * ncols, n, st));
    int at = 0;
    if (packed) CK(launch_sample_tc_packed(pA, pR, n, ncols, precision, side, S, lds, err, st));
    else CK(launch_sample_tc(s, leaf, precision, side, ncols, pR, S, lds, err, &at, tt, st));
  }
  if (packed) CK(cudaFreeAsync(pA, st));
  if (tt) CK(cudaFreeAsync(tt, st));
  CK(cudaFreeAsync(pR, st));
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaFreeAsync(Rr, st));
  CK(cudaFreeAsync(err, st));
  CK(cudaFreeAsync(d_lid, st));
  CK(cudaStreamSynchronize(st));
  if (herr) return fail(HSS_ERR_TIMEOUT, "tensor-core sampling gave up waiting (code %d)", herr);
  return HSS_OK;
}

}  // extern "C"

// ===================================================================
// Sampling without any device allocation.
//
// hss_sample_offdiag allocates (stream-ordered) a small table that tells the
// sampling kernel which leaf every index belongs to.  Some callers cannot
// let a library allocate device memory: a serving process or framework that
// owns the whole device-memory budget through its own pool, or a caller that
// cannot accept the synchronisation or the possible failure of cudaMalloc /
// cudaMallocAsync in the middle of a run.  hss_sample_offdiag_noalloc keeps
// that table in a fixed device array that is part of the library image
// instead: it exists on every GPU that loads the library, until the process
// exits, and bounds n by HSS_NOALLOC_MAX_N.
// ===================================================================
#define HSS_NOALLOC_MAX_N (1 << 20)   /* 4 MiB of leaf labels */

static __device__ __align__(256) int g_noalloc_leaf_label[HSS_NOALLOC_MAX_N];

namespace {

// leaf label of index i = first index of the leaf of the halving tree that
// contains i (equal within a leaf, nondecreasing over i)
__global__ void k_noalloc_leaf_label(int* label, int n, int leaf) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int lo = 0, size = n;
  while (size > leaf) {
    int h = size / 2;
    if (i < lo + h) size = h;
    else { lo += h; size -= h; }
  }
  label[i] = lo;
}

std::mutex g_noalloc_mu;
// (context id, device address of the label array in that context): a
// context that is destroyed and created again (cudaDeviceReset) reloads the
// library's module at another address and gets a new id, so a cached
// address never outlives its context
std::vector<std::pair<unsigned long long, int*>> g_noalloc_ptr;

// Device address of the label array in the current context, looked up once
// per context (host code must not pass the symbol itself to a kernel).  The
// first lookup in a context may load the library's device code; later calls
// only read the table.
hss_status noalloc_table(int** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  unsigned long long id = 0;
  bool have_id = current_context_id(&id);
  if (have_id)
    for (auto& e : g_noalloc_ptr)
      if (e.first == id) {
        *out = e.second;
        return HSS_OK;
      }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_leaf_label);
  if (e != cudaSuccess || !p)
    return fail(HSS_ERR_CUDA, "cudaGetSymbolAddress of the leaf-label array failed: %s", cudaGetErrorString(e));
  if (!have_id) have_id = current_context_id(&id);   // the lookup made the primary context current
  if (have_id) g_noalloc_ptr.push_back({id, (int*)p});
  *out = (int*)p;
  return HSS_OK;
}

}  // namespace

extern "C" hss_status hss_sample_offdiag_noalloc(const hss_source* A, int leaf, int precision,
                                                 int ncols, const double* R, long long ldr,
                                                 double* Sr, double* Sc, long long lds,
                                                 void* stream) {
  CKS(check_source(A));
  if (A->kind == HSS_SRC_EXTRACT) return fail(HSS_ERR_ARG, "sampling needs a source with entries on the device");
  const int n = A->n;
  if (leaf < 1 || ncols < 0 || !R || ldr < n || lds < ncols)
    return fail(HSS_ERR_ARG, "bad arguments to hss_sample_offdiag_noalloc");
  if (n > HSS_NOALLOC_MAX_N)
    return fail(HSS_ERR_ARG, "n = %d exceeds the fixed table of hss_sample_offdiag_noalloc (%d)", n,
                HSS_NOALLOC_MAX_N);
  if (precision != HSS_PREC_FP64)
    return fail(HSS_ERR_UNSUPPORTED, "hss_sample_offdiag_noalloc takes HSS_PREC_FP64 only (the mixed forms "
                                     "need temporary operand buffers)");
  int* label = nullptr;
  CKS(noalloc_table(&label));
  cudaStream_t st = (cudaStream_t)stream;
  k_noalloc_leaf_label<<<(n + 255) / 256, 256, 0, st>>>(label, n, leaf);
  CK(cudaGetLastError());
  SrcDev s = make_src(*A, label);
  CK(launch_sample_fp64(s, ncols, R, ldr, Sr, Sc, lds, st));
  return HSS_OK;
}

namespace hss {
hss_tuning tuning_get() {
  std::lock_guard<std::mutex> lock(tuning_mutex());
  return tuning_ref();
}
}  // namespace hss
