// perturb.cu -- the first-order perturbation estimate of eq. (11), the paper's
// comparison method for a small K (Sec. 3):
//   mu_j = lam_j + u_j^T Sigma u_j,
//   v_j  = q_j + sum_{i != j} (u_i^T Sigma u_j) / (lam_j - lam_i) q_i,
// i.e. X = Q W with W = I + E, E_ij = (U Sigma U^T)_ij / (lam_j - lam_i).
// (The printed v_j update names v_j^0 and lam_i - lam_j where the standard first
// order has q_i and lam_j - lam_i.)  A pair with lam_i == lam_j contributes 0: the
// formula has no first-order term inside a repeated eigenvalue's eigenspace.
// The product X = Q W runs on the update's own GEMMs.
#include "eig_internal.cuh"

namespace eig {
namespace {

constexpr int kPwThreads = 256;

// Element (a, b) of the output at out[a + b*n] (a contiguous): W[a][b] in the
// plain layout, W[b][a] when transposed (W^T column-major, the layout the
// tensor-core slicer reads to give per-column exponents of W).
template <int KMAX>
__global__ void __launch_bounds__(kPwThreads) perturb_w_kernel(int n, int k, const double* __restrict__ lam,
                                                               const double* __restrict__ U,
                                                               unsigned long long negmask, int transposed,
                                                               double* __restrict__ out) {
  const int a = blockIdx.x * kPwThreads + threadIdx.x;
  double ua[KMAX];
  double la = 0.0;
  if (a < n) {
    la = lam[a];
#pragma unroll
    for (int c = 0; c < KMAX; ++c) ua[c] = (c < k) ? U[(size_t)c * n + a] : 0.0;
  }
  for (int b = blockIdx.y; b < n; b += gridDim.y) {
    if (a >= n) continue;
    const double lb = lam[b];
    double dot = 0.0;
#pragma unroll
    for (int c = 0; c < KMAX; ++c) {
      if (c < k) {
        const double ub = U[(size_t)c * n + b];
        dot = fma(ua[c], ((negmask >> c) & 1ull) ? -ub : ub, dot);
      }
    }
    // row i, column j of W
    const double li = transposed ? lb : la, lj = transposed ? la : lb;
    const bool diag = (a == b);
    const double d = lj - li;
    double v;
    if (diag) {
      v = 1.0;
    } else if (d != 0.0) {
      v = dot / d;
    } else {
      v = 0.0;
    }
    out[(size_t)b * n + a] = v;
  }
}

__global__ void perturb_mu_kernel(int n, int k, const double* __restrict__ lam, const double* __restrict__ U,
                                  unsigned long long negmask, double* __restrict__ mu) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = 0.0;
  for (int c = 0; c < k; ++c) {
    const double u = U[(size_t)c * n + j];
    s = fma(((negmask >> c) & 1ull) ? -u : u, u, s);
  }
  mu[j] = lam[j] + s;
}

}  // namespace

cudaError_t launch_perturb_w(int64_t n, int k, const double* lam, const double* U, unsigned long long negmask,
                             bool transposed, double* W, cudaStream_t s) {
  if (n < 1 || k < 1 || k > EIG_MAX_K) return cudaErrorInvalidValue;
  dim3 grid((unsigned)((n + kPwThreads - 1) / kPwThreads), (unsigned)(n < 65535 ? n : 65535));
  if (k <= 4) {
    perturb_w_kernel<4><<<grid, kPwThreads, 0, s>>>((int)n, k, lam, U, negmask, transposed ? 1 : 0, W);
  } else if (k <= 8) {
    perturb_w_kernel<8><<<grid, kPwThreads, 0, s>>>((int)n, k, lam, U, negmask, transposed ? 1 : 0, W);
  } else {
    perturb_w_kernel<16><<<grid, kPwThreads, 0, s>>>((int)n, k, lam, U, negmask, transposed ? 1 : 0, W);
  }
  return cudaGetLastError();
}

cudaError_t launch_perturb_mu(int64_t n, int k, const double* lam, const double* U, unsigned long long negmask,
                              double* mu, cudaStream_t s) {
  perturb_mu_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((int)n, k, lam, U, negmask, mu);
  return cudaGetLastError();
}

}  // namespace eig
