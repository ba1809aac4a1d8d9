// Entries of a compressed HSS matrix, H(I, J) for index sets I and J
// (section 2.1, eq. nestedUV): for i and j in one leaf, D(i, j); otherwise,
// with a and b the children of their lowest common ancestor tau that hold
// i and j,
//     H(i, j) = u_a(i) B_ab v_b(j)^T,
// where B_ab is tau's B12 (a first) or B21, and u_a(i) is row i of the
// nested basis of a: at a leaf the row of U = Pi [I; X^T] (eq. ID), one level
// up u_parent(i) = u_a(i) U_parent(rows of a's block, :) (the basis of a
// node is its children's bases times its own small one).  The same for
// v_b(j) with V.  A node that was not COMPRESSED (a partial result) keeps
// its blocks A(I_nu1, I_nu2), A(I_nu2, I_nu1) dense.
//
// Three kernels: the inverse pivot orders of every node side; one CTA per
// requested row index walking its leaf's path to the root and storing
// W_i(level) = u_a(i) B_ab for every ancestor a (and one CTA per column index
// storing v_b(j)); one thread per requested entry finding the common
// ancestor and forming one dot product.
#include "hss_internal.h"

namespace hss {
namespace {

// inv[piv[q]] = q for every node side (one CTA per side)
__global__ void k_inv_piv(const EntryNode* __restrict__ nodes, int nn, int* __restrict__ err) {
  const int side = blockIdx.x & 1, id = blockIdx.x >> 1;
  if (id >= nn) return;
  const EntryNode& t = nodes[id];
  const int m = side ? t.mc : t.mr;
  const int* piv = side ? t.pivc : t.pivr;
  int* inv = side ? t.ipivc : t.ipivr;
  if (!piv || !inv) return;
  for (int q = threadIdx.x; q < m; q += blockDim.x) {
    const int p = piv[q];
    if (p < 0 || p >= m) { atomicCAS(err, 0, 2); continue; }
    inv[p] = q;
  }
}

// Row (side 0) or column (side 1) vectors of the nested basis along the path
// of index idx[r] to the root.  side 0 stores W(level(a)) = u_a(i) B_ab for
// every ancestor a whose parent is COMPRESSED; side 1 stores v_a(j).
// out: (count x (levels + 1) x kcap) doubles; shared memory 2 kcap doubles.
__global__ void k_entry_paths(const EntryNode* __restrict__ nodes, const int* __restrict__ leaf_of, int n,
                              const int* __restrict__ idx, int count, double* __restrict__ out, int kcap, int lp1,
                              int side, int* __restrict__ err) {
  extern __shared__ double sm[];
  double* u = sm;
  double* u2 = sm + kcap;
  const int r = blockIdx.x;
  if (r >= count) return;
  const int i = idx[r];
  if (i < 0 || i >= n) {   // reported; the pair kernel skips the entry
    if (threadIdx.x == 0) atomicCAS(err, 0, 1);
    return;
  }
  int a = leaf_of[i];
  // the root is a leaf (D only), or the leaf's parent was left uncompressed
  // (its couplings are dense blocks; the leaf has no basis)
  if (nodes[a].parent < 0 || nodes[nodes[a].parent].state != HSS_COMPRESSED) return;
  double* base = out + (long long)r * lp1 * kcap;
  {
    const EntryNode& t = nodes[a];
    const int k = side ? t.kc : t.kr;
    const int* inv = side ? t.ipivc : t.ipivr;
    const double* X = side ? t.Xc : t.Xr;
    const int pos = inv[i - t.lo];
    if (pos < 0 || pos >= t.size) {   // not a permutation (never from a compression)
      if (threadIdx.x == 0) atomicCAS(err, 0, 2);
      return;
    }
    for (int c = threadIdx.x; c < k; c += blockDim.x)
      u[c] = pos < k ? (c == pos ? 1.0 : 0.0) : X[c + (long long)(pos - k) * max(k, 1)];
  }
  __syncthreads();
  for (;;) {
    const EntryNode& t = nodes[a];
    const EntryNode& p = nodes[t.parent];
    if (p.state != HSS_COMPRESSED) break;   // dense coupling above: no basis rows needed
    const int ka = side ? t.kc : t.kr;
    const int first = p.ch0 == a;
    const EntryNode& b = nodes[first ? p.ch1 : p.ch0];
    double* dst = base + (long long)t.level * kcap;
    if (side == 0) {
      // W = u_a(i) B_ab: B12 is kr(nu1) x kc(nu2) with ld max(kr(nu1), 1),
      // B21 is kr(nu2) x kc(nu1) with ld max(kr(nu2), 1)
      const double* B = first ? p.B12 : p.B21;
      const int ld = max(ka, 1);
      for (int c = threadIdx.x; c < b.kc; c += blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < ka; ++q) s = __fma_rn(u[q], B[q + (long long)c * ld], s);
        dst[c] = s;
      }
    } else {
      for (int c = threadIdx.x; c < ka; c += blockDim.x) dst[c] = u[c];
    }
    if (p.parent < 0) break;   // a is a child of the root
    // u_parent(i) = u_a(i) U_p(off + q, :), U_p(s, c) = [pos_s == c] for the
    // skeleton rows, X_p(c, pos_s - k_p) for the others
    const int kp = side ? p.kc : p.kr;
    const int* inv = side ? p.ipivc : p.ipivr;
    const double* X = side ? p.Xc : p.Xr;
    const int off = first ? 0 : (side ? b.kc : b.kr);
    const int mp = side ? p.mc : p.mr;
    for (int c = threadIdx.x; c < kp; c += blockDim.x) {
      double s = 0.0;
      for (int q = 0; q < ka; ++q) {
        const int pos = inv[off + q];
        if (pos < 0 || pos >= mp) {   // not a permutation (never from a compression)
          atomicCAS(err, 0, 2);
          continue;
        }
        s = __fma_rn(u[q], pos < kp ? (pos == c ? 1.0 : 0.0) : X[c + (long long)(pos - kp) * max(kp, 1)], s);
      }
      u2[c] = s;
    }
    __syncthreads();
    double* tmp = u;
    u = u2;
    u2 = tmp;
    a = t.parent;
  }
}

// out(r, c) = H(I[r], J[c]) for one chunk of rows and columns
__global__ void k_entry_pairs(const EntryNode* __restrict__ nodes, const int* __restrict__ leaf_of, int n,
                              const int* __restrict__ I, int nr, const int* __restrict__ J, int nc,
                              const double* __restrict__ Wrow, const double* __restrict__ Vcol, int kcap, int lp1,
                              double* __restrict__ out, long long ldo) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (r >= nr || c >= nc) return;
  const int i = I[r], j = J[c];
  double* dst = out + r + (long long)c * ldo;
  if (i < 0 || i >= n || j < 0 || j >= n) { *dst = 0.0; return; }
  int a = leaf_of[i], b = leaf_of[j];
  if (a == b) {
    const EntryNode& t = nodes[a];
    *dst = t.D[(i - t.lo) + (long long)(j - t.lo) * t.size];
    return;
  }
  while (nodes[a].level > nodes[b].level) a = nodes[a].parent;
  while (nodes[b].level > nodes[a].level) b = nodes[b].parent;
  while (nodes[a].parent != nodes[b].parent) { a = nodes[a].parent; b = nodes[b].parent; }
  const EntryNode& ta = nodes[a];
  const EntryNode& tb = nodes[b];
  const EntryNode& p = nodes[ta.parent];
  if (p.state != HSS_COMPRESSED) {
    const double* F = p.ch0 == a ? p.F12 : p.F21;   // A(I_a, I_b), ld |a|
    *dst = F[(i - ta.lo) + (long long)(j - tb.lo) * ta.size];
    return;
  }
  const double* w = Wrow + ((long long)r * lp1 + ta.level) * kcap;
  const double* v = Vcol + ((long long)c * lp1 + tb.level) * kcap;
  double s0 = 0.0, s1 = 0.0;
  int q = 0;
  for (; q + 1 < tb.kc; q += 2) {
    s0 = __fma_rn(w[q], v[q], s0);
    s1 = __fma_rn(w[q + 1], v[q + 1], s1);
  }
  if (q < tb.kc) s0 = __fma_rn(w[q], v[q], s0);
  *dst = s0 + s1;
}

}  // namespace

cudaError_t launch_inv_piv(const EntryNode* nodes, int nn, int* err, cudaStream_t st) {
  if (nn <= 0) return cudaSuccess;
  k_inv_piv<<<2 * nn, 256, 0, st>>>(nodes, nn, err);
  return cudaGetLastError();
}

cudaError_t launch_entry_paths(const EntryNode* nodes, const int* leaf_of, int n, const int* idx, int count,
                               double* out, int kcap, int lp1, int side, int* err, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const size_t sm = sizeof(double) * 2 * (size_t)kcap;
  cudaError_t e = cudaFuncSetAttribute(k_entry_paths, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_entry_paths<<<count, 128, sm, st>>>(nodes, leaf_of, n, idx, count, out, kcap, lp1, side, err);
  return cudaGetLastError();
}

cudaError_t launch_entry_pairs(const EntryNode* nodes, const int* leaf_of, int n, const int* I, int nr, const int* J,
                               int nc, const double* Wrow, const double* Vcol, int kcap, int lp1, double* out,
                               long long ldo, cudaStream_t st) {
  if (nr <= 0 || nc <= 0) return cudaSuccess;
  k_entry_pairs<<<dim3((nr + 127) / 128, nc), 128, 0, st>>>(nodes, leaf_of, n, I, nr, J, nc, Wrow, Vcol, kcap, lp1,
                                                            out, ldo);
  return cudaGetLastError();
}

}  // namespace hss
