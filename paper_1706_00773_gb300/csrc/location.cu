// location.cu -- the rank-2 location vector of Sec. 2.2 (Algorithms 1a-1c).
//
// Residues (eq. (2) with its sign corrected, eq. (3)'s convention
// f(x) = 1 + sum_i alpha_i / (lam_i - x)):
//   alpha_p = u_p^T adj(I - Sigma M~_p) Sigma u_p,   M~_p = sum_{i != p} u_i u_i^T / (lam_p - lam_i)
// (I + Sigma U^T D_p U with D_p = diag(1/(lam_j - lam_p)) equals I - Sigma M~_p).
// One warp per pole forms M~_p (2x2) from every other term; one block then
// runs the scan of Algorithm 1a (both sigma > 0), 1b (both < 0, from the
// right) or 1c (opposite signs, started from the sign of alpha_1).  L[0] holds
// the roots below lam_1, L[i] those in (lam_i, lam_{i+1}), L[n] those above
// lam_n; where the listings read the undefined residue past either end, the
// last interval takes the roots not placed yet.  With opposite signs a root
// can sit one pole below its old eigenvalue, so up to i+1 roots lie below
// lam_{i+1} and 1c's 0-or-2 choice is made against that bound.
#include "eig_internal.cuh"

namespace eig {
namespace {

__global__ void residues_rank2_kernel(int n, const double* __restrict__ lam,
                                      const double* __restrict__ U, int ldu, double s0, double s1,
                                      double* __restrict__ alpha) {
  const int lane = threadIdx.x & 31;
  const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (p >= n) return;
  const double lp = lam[p];
  double m00 = 0.0, m01 = 0.0, m11 = 0.0;
  for (int i = lane; i < n; i += 32) {
    if (i == p) continue;
    const double r = 1.0 / (lp - lam[i]);
    const double a = U[i], b = U[ldu + i];
    m00 = fma(a * r, a, m00);
    m01 = fma(a * r, b, m01);
    m11 = fma(b * r, b, m11);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    m00 += __shfl_xor_sync(0xffffffffu, m00, off);
    m01 += __shfl_xor_sync(0xffffffffu, m01, off);
    m11 += __shfl_xor_sync(0xffffffffu, m11, off);
  }
  if (lane == 0) {
    // B = I - Sigma M~ ; adj(B) = [[B11, -B01], [-B10, B00]]
    const double b00 = 1.0 - s0 * m00, b01 = -s0 * m01;
    const double b10 = -s1 * m01, b11 = 1.0 - s1 * m11;
    const double u0 = U[p], u1 = U[ldu + p];
    const double v0 = s0 * u0, v1 = s1 * u1;  // Sigma u
    const double a0 = b11 * v0 - b01 * v1;    // adj(B) Sigma u
    const double a1 = -b10 * v0 + b00 * v1;
    alpha[p] = u0 * a0 + u1 * a1;
  }
}

// The greedy scans of Algorithms 1a-1c carry one bit of state: before the
// step that fills interval i, (i - 1) - M (1a, 1b) or i - M (1c) is 0 or 1.
// A residue sign change puts 2 roots in the interval when the bit is 1 and 0
// when it is 0, and flips the bit; equal signs put 1 root and keep it.  So the
// bit before a step is its start value XOR the parity of the sign changes
// before it: one block scans those parities, then each thread writes its
// chunk of L.  1b runs the same steps from the right.
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads) location_scan_kernel(int n, const double* __restrict__ a,
                                                                     int variant, int* __restrict__ L) {
  __shared__ int warp_par[kScanThreads / 32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int steps = n - 1;
  const int chunk = (steps + kScanThreads - 1) / kScanThreads;
  const int lo = 1 + t * chunk;
  const int hi = min(steps + 1, lo + chunk);
  auto interval = [&](int s) { return variant == 1 ? n - s : s; };
  int par = 0;
  for (int s = lo; s < hi; ++s) {
    const int j = interval(s);
    par ^= (a[j - 1] * a[j] > 0.0) ? 0 : 1;
  }
  // exclusive XOR scan over the block
  int incl = par;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl ^= v;
  }
  if (lane == 31) warp_par[w] = incl;
  __syncthreads();
  if (w == 0) {
    int v = warp_par[lane];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, v, off);
      if (lane >= off) v ^= u;
    }
    warp_par[lane] = v;  // inclusive over warps
  }
  __syncthreads();
  const int before_warp = (w > 0) ? warp_par[w - 1] : 0;
  const int total = warp_par[kScanThreads / 32 - 1];
  const int d0 = (variant == 2 && a[0] > 0.0) ? 1 : 0;
  int d = d0 ^ before_warp ^ (incl ^ par);
  for (int s = lo; s < hi; ++s) {
    const int j = interval(s);
    if (a[j - 1] * a[j] > 0.0) {
      L[j] = 1;
    } else {
      L[j] = d ? 2 : 0;
      d ^= 1;
    }
  }
  if (t == 0) {
    const int dn = d0 ^ total;
    if (variant == 0) {
      L[0] = 0;
      L[n] = 1 + dn;
    } else if (variant == 1) {
      L[n] = 0;
      L[0] = 1 + dn;
    } else {
      L[0] = (a[0] > 0.0) ? 0 : 1;
      L[n] = dn;
    }
  }
}

}  // namespace
}  // namespace eig

using namespace eig;

extern "C" int eig_location_rank2(int64_t n, const double* lambda, const double* U,
                                  const int8_t* sigma, double* alpha, int32_t* L, void* stream) {
  if (n < 2 || n > (int64_t)0x3fffffff || !lambda || !U || !alpha || !L) return EIG_EINVAL;
  const int s0 = sigma ? sigma[0] : 1, s1 = sigma ? sigma[1] : 1;
  if ((s0 != 1 && s0 != -1) || (s1 != 1 && s1 != -1)) return EIG_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int variant = (s0 > 0 && s1 > 0) ? 0 : (s0 < 0 && s1 < 0) ? 1 : 2;
  residues_rank2_kernel<<<(unsigned)((n + 7) / 8), 256, 0, s>>>((int)n, lambda, U, (int)n, (double)s0,
                                                               (double)s1, alpha);
  location_scan_kernel<<<1, kScanThreads, 0, s>>>((int)n, alpha, variant, L);
  if (cudaGetLastError() != cudaSuccess) return EIG_ECUDA;
  return EIG_OK;
}
