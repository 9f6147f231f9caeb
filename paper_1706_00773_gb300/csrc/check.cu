// check.cu -- optional FP64 quality check of an update on sampled columns:
// residual |A' x - mu x|_2 with A' = Q diag(lam) Q^T + K Sigma K^T applied
// through the OLD Q and lam, and the Gram matrix of the sampled x.  These are
// the accuracy metrics (B) and (C) of the paper's Figs. 6-7.
#include <math.h>

#include "eig_internal.cuh"

namespace eig {
namespace {

constexpr int kChkThreads = 256;

__device__ double block_sum_chk(double v, double* sh) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int s = kChkThreads / 2; s > 0; s >>= 1) {
    if (t < s) sh[t] += sh[t + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

__global__ void gather_cols_kernel(int64_t n, const double* __restrict__ X,
                                   const int* __restrict__ cols, int nc, double* __restrict__ Xs) {
  const int s = blockIdx.y;
  const double* src = X + (int64_t)cols[s] * n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    Xs[i + (int64_t)s * n] = src[i];
}

__global__ void scale_rows_kernel(int64_t n, int nc, const double* __restrict__ lam,
                                  double* __restrict__ Z) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * nc;
       e += (int64_t)gridDim.x * blockDim.x)
    Z[e] *= lam[e % n];
}

// One CTA per sampled column s: y = Y[:,s] + K Sigma (K^T x) - mu x, out[s] = |y|.
__global__ void __launch_bounds__(kChkThreads) residual_kernel(
    int64_t n, int k, const double* __restrict__ K, unsigned long long negmask,
    const double* __restrict__ Xs, const double* __restrict__ Y, const double* __restrict__ mu,
    const int* __restrict__ cols, double* __restrict__ out) {
  __shared__ double sh[kChkThreads];
  __shared__ double kt[EIG_MAX_K];
  const int s = blockIdx.x;
  const double* x = Xs + (int64_t)s * n;
  const double* y = Y + (int64_t)s * n;
  for (int c = 0; c < k; ++c) {
    double p = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kChkThreads) p = fma(K[i + (int64_t)c * n], x[i], p);
    p = block_sum_chk(p, sh);
    if (threadIdx.x == 0) kt[c] = ((negmask >> c) & 1ull) ? -p : p;
  }
  __syncthreads();
  const double m = mu[cols[s]];
  double r2 = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += kChkThreads) {
    double v = y[i] - m * x[i];
    for (int c = 0; c < k; ++c) v = fma(K[i + (int64_t)c * n], kt[c], v);
    r2 = fma(v, v, r2);
  }
  r2 = block_sum_chk(r2, sh);
  if (threadIdx.x == 0) out[s] = sqrt(r2);
}

__global__ void __launch_bounds__(kChkThreads) gram_kernel(int64_t n, int nc,
                                                           const double* __restrict__ Xs,
                                                           double* __restrict__ out) {
  __shared__ double sh[kChkThreads];
  const int a = blockIdx.x, b = blockIdx.y;
  double p = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += kChkThreads)
    p = fma(Xs[i + (int64_t)a * n], Xs[i + (int64_t)b * n], p);
  p = block_sum_chk(p, sh);
  if (threadIdx.x == 0) out[a + b * nc] = p;
}

}  // namespace

cudaError_t launch_check_pairs(int64_t n, int k, const double* Q, const double* lam,
                               const double* K, unsigned long long negmask, const double* X,
                               const double* mu, const int* cols, int nc, double* tmp,
                               double* out, cudaStream_t s) {
  double* Xs = tmp;
  double* Z = tmp + n * nc;
  double* Y = tmp + 2 * n * nc;
  dim3 g1((unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), (unsigned)nc);
  gather_cols_kernel<<<g1, 256, 0, s>>>(n, X, cols, nc, Xs);
  cudaError_t e = launch_project_f64(n, nc, Q, Xs, Z, s);  // Z = Q^T Xs
  if (e != cudaSuccess) return e;
  scale_rows_kernel<<<1024, 256, 0, s>>>(n, nc, lam, Z);
  e = launch_gemm_f64(n, nc, n, Q, n, Z, n, Y, n, s);  // Y = Q diag(lam) Q^T Xs
  if (e != cudaSuccess) return e;
  residual_kernel<<<nc, kChkThreads, 0, s>>>(n, k, K, negmask, Xs, Y, mu, cols, out);
  gram_kernel<<<dim3(nc, nc), kChkThreads, 0, s>>>(n, nc, Xs, out + nc);
  return cudaGetLastError();
}

}  // namespace eig
