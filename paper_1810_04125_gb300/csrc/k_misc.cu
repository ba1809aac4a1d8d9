// Element extraction A(I, J) for the generators D_tau = A(I_tau, I_tau) and
// B12 = A(nu1.I^r, nu2.I^c), B21 = A(nu2.I^r, nu1.I^c) (Algorithm 3,
// section 3.1), all blocks of one tree level in one launch; plus small
// helpers (finiteness check of the samples, index gathers for
// tau.I^r = [nu1.I^r nu2.I^r](tau.J^r) of Algorithm 2).
#include "hss_internal.h"

namespace hss {
namespace {

// grid: (tile, job); each CTA fills 32 x 32 tiles of its job, striding
// over the job's tiles.
__global__ void k_extract(const ExtractJob* __restrict__ jobs) {
  const ExtractJob jb = jobs[blockIdx.y];
  const SrcDev& src = jb.src;
  const int tiles_i = (jb.mi + 31) / 32, tiles_j = (jb.nj + 31) / 32;
  const int ntiles = tiles_i * tiles_j;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int ti = t % tiles_i, tj = t / tiles_i;
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
      int il = e % 32, jl = e / 32;
      int i = ti * 32 + il, j = tj * 32 + jl;
      if (i >= jb.mi || j >= jb.nj) continue;
      int gi = jb.I ? jb.I[i] : jb.i0 + i;
      int gj = jb.J ? jb.J[j] : jb.j0 + j;
      jb.out[(long long)i + (long long)j * jb.ldo] = entry(src, gi, gj);
    }
  }
}

// With a user sampling operator the leaf diagonal blocks come off the
// user's product (Algorithm 2 at a leaf: (A R)(I_tau) - D_tau R(I_tau)): a
// CTA takes a 32 x 32 tile (rows i0.., columns q0..), forms its rows' leaf
// block products in FP64 from the packed blocks D (leaf L at Dp + doff[L],
// col-major) and writes the tile transposed into the row-major samples
// through shared memory.
__global__ void __launch_bounds__(256) k_leaf_diag_sub(const double* __restrict__ Dp,
                                                     const long long* __restrict__ doff,
                                                     const int* __restrict__ leaf_id,
                                                     const int* __restrict__ leaf_lo, int n, int w,
                                                     const double* __restrict__ R, long long ldr,
                                                     const double* __restrict__ T, long long ldt,
                                                     double* __restrict__ S, long long lds, int trans) {
  __shared__ double tile[32][33];
  const int i0 = blockIdx.x * 32, q0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int qq = ty; qq < 32; qq += 8) {
    const int i = i0 + tx, q = q0 + qq;
    double v = 0.0;
    if (i < n && q < w) {
      const int L = leaf_id[i];
      const int lo = leaf_lo[L], hi = leaf_lo[L + 1], m = hi - lo;
      const double* D = Dp + doff[L];
      const double* Rq = R + (long long)q * ldr;
      double acc = 0.0;
      // A(i, j) = D(i - lo, j - lo); the transposed product takes A(j, i)
      for (int j = lo; j < hi; ++j)
        acc = __fma_rn(trans ? D[(j - lo) + (long long)(i - lo) * m] : D[(i - lo) + (long long)(j - lo) * m], Rq[j],
                       acc);
      v = T[(long long)q * ldt + i] - acc;
    }
    tile[qq][tx] = v;
  }
  __syncthreads();
  for (int ii = ty; ii < 32; ii += 8) {
    const int i = i0 + ii, q = q0 + tx;
    if (i < n && q < w) S[(long long)i * lds + q] = tile[tx][ii];
  }
}

__global__ void k_nonfinite(const double* __restrict__ S, long long lds, int n, int c0, int c1,
                            int* flag) {
  int w = c1 - c0;
  long long total = (long long)n * w;
  int bad = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long i = t / w;
    int c = c0 + (int)(t % w);
    double v = S[i * lds + c];
    if (!isfinite(v)) bad = 1;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

// grid: (chunk, job)
__global__ void k_gather_int(const GatherJob* __restrict__ jobs) {
  const GatherJob jb = jobs[blockIdx.y];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < jb.cnt; t += gridDim.x * blockDim.x) {
    const int r = jb.idx[t];
    jb.dst[t] = (r < jb.split) ? jb.src[r] : jb.src2[r - jb.split];
  }
}

// X(i, j) = (i == c0 + j): columns c0 .. c0 + w - 1 of the identity (n x w,
// column-major, ld n)
__global__ void k_identity_block(double* X, int n, int c0, int w) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * w) return;
  const int i = (int)(e % n), j = (int)(e / n);
  X[e] = (i == c0 + j) ? 1.0 : 0.0;
}

}  // namespace

cudaError_t launch_identity_block(double* X, int n, int c0, int w, cudaStream_t st) {
  const long long tot = (long long)n * w;
  if (tot <= 0) return cudaSuccess;
  k_identity_block<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(X, n, c0, w);
  return cudaGetLastError();
}

// Every job's source must have its entries on the device (kinds DENSE ..
// LAPLACE); the host checks that before it builds the list.
cudaError_t launch_extract(const ExtractJob* jobs_dev, int njobs, int max_tiles, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  int gx = max_tiles < 1 ? 1 : (max_tiles > 64 ? 64 : max_tiles);
  for (int j0 = 0; j0 < njobs; j0 += 65535) {
    const int nj = njobs - j0 < 65535 ? njobs - j0 : 65535;
    k_extract<<<dim3(gx, nj), 256, 0, st>>>(jobs_dev + j0);
  }
  return cudaGetLastError();
}

cudaError_t launch_leaf_diag_sub(const double* Dp, const long long* doff, const int* leaf_id, const int* leaf_lo,
                                 int n, int w, const double* R, long long ldr, const double* T, long long ldt,
                                 double* S, long long lds, int trans, cudaStream_t st) {
  if (n <= 0 || w <= 0) return cudaSuccess;
  dim3 grid((n + 31) / 32, (w + 31) / 32);
  k_leaf_diag_sub<<<grid, 256, 0, st>>>(Dp, doff, leaf_id, leaf_lo, n, w, R, ldr, T, ldt, S, lds, trans);
  return cudaGetLastError();
}

cudaError_t launch_nonfinite(const double* S, long long lds, int n, int c0, int c1, int* flag,
                             cudaStream_t st) {
  if (n <= 0 || c1 <= c0) return cudaSuccess;
  k_nonfinite<<<152 * 4, 256, 0, st>>>(S, lds, n, c0, c1, flag);
  return cudaGetLastError();
}

cudaError_t launch_gather_int(const GatherJob* jobs_dev, int njobs, int max_cnt, cudaStream_t st) {
  if (njobs <= 0 || max_cnt <= 0) return cudaSuccess;
  const int gx = (max_cnt + 127) / 128 < 8 ? (max_cnt + 127) / 128 : 8;
  for (int j0 = 0; j0 < njobs; j0 += 65535) {
    const int nj = njobs - j0 < 65535 ? njobs - j0 : 65535;
    k_gather_int<<<dim3(gx, nj), 128, 0, st>>>(jobs_dev + j0);
  }
  return cudaGetLastError();
}

}  // namespace hss
