// Gaussian random matrix R (randn of the paper's helper-function table).
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): ten rounds of the
// bijection (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2),
// hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)) with the Weyl key schedule.  Entry
// R(i, c) uses counter (i >> 1, c, 0, 0); words (w0, w1) and (w2, w3) give
// two 53-bit uniforms; Box-Muller turns them into the pair used by rows
// 2p (cosine branch) and 2p + 1 (sine branch).
#include <algorithm>

#include "hss_internal.h"

namespace hss {
namespace {

__device__ __forceinline__ void philox_round(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
  uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
  uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
  c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
}

__device__ __forceinline__ double round_sig(double x, int bits) {
  // nearest value with a `bits`-bit significand, ties to even
  int e;
  double m = frexp(x, &e);
  double s = (double)(1 << bits);
  return ldexp(rint(m * s) / s, e);
}

__global__ void k_random_normal(unsigned long long seed, int n, int col0, int ncols,
                                double* R, long long ldr, int round_mode) {
  const int npairs = (n + 1) / 2;
  long long total = (long long)npairs * ncols;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int p = (int)(t % npairs);
    int c = (int)(t / npairs);
    uint32_t w[4] = {(uint32_t)p, (uint32_t)(col0 + c), 0u, 0u};
    uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFull), k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
      philox_round(w, k0, k1);
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    double u1 = ((double)(w[0] >> 5) * 67108864.0 + (double)(w[1] >> 6)) * 0x1.0p-53;
    double u2 = ((double)(w[2] >> 5) * 67108864.0 + (double)(w[3] >> 6)) * 0x1.0p-53;
    double rad = sqrt(-2.0 * log1p(-u1));
    double s, co;
    sincospi(2.0 * u2, &s, &co);
    double z0 = rad * co, z1 = rad * s;
    if (round_mode == 1) { z0 = round_sig(z0, 11); z1 = round_sig(z1, 11); }
    if (round_mode == 2) { z0 = round_sig(z0, 8); z1 = round_sig(z1, 8); }
    double* col = R + (long long)c * ldr;
    col[2 * p] = z0;
    if (2 * p + 1 < n) col[2 * p + 1] = z1;
  }
}

__global__ void k_round_copy(const double* in, long long ldin, double* out, long long ldout, int n,
                             int ncols, int mode) {
  long long total = (long long)n * ncols;
  const int bits = mode == 1 ? 11 : 8;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % n);
    long long c = t / n;
    out[i + c * ldout] = round_sig(in[i + c * ldin], bits);
  }
}

}  // namespace

cudaError_t launch_round_copy(const double* in, long long ldin, double* out, long long ldout, int n,
                              int ncols, int mode, cudaStream_t st) {
  if (n <= 0 || ncols <= 0) return cudaSuccess;
  long long total = (long long)n * ncols;
  int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 32);
  k_round_copy<<<blocks, 256, 0, st>>>(in, ldin, out, ldout, n, ncols, mode);
  return cudaGetLastError();
}

cudaError_t launch_random_normal(unsigned long long seed, int n, int col0, int ncols,
                                 double* R, long long ldr, int round_mode, cudaStream_t st) {
  if (n <= 0 || ncols <= 0) return cudaSuccess;
  long long total = (long long)((n + 1) / 2) * ncols;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_random_normal<<<blocks, 256, 0, st>>>(seed, n, col0, ncols, R, ldr, round_mode);
  return cudaGetLastError();
}

}  // namespace hss
