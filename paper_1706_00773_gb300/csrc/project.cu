// project.cu -- U = Q^T K (Sec. 2.1, below eq. (1)) in FP64 and the
// one-row-one-column canonicalisation of Sec. 2.2 (Steps 1-2).
#include "eig_internal.cuh"

namespace eig {
namespace {

constexpr int kProjChunk = 8;  // columns of K accumulated per pass over a Q column

// One warp per column j of Q: U[j, c] = sum_i Q[i, j] K[i, c].  Lanes stride
// over i (coalesced 256-byte reads of the column); k is processed in chunks of
// kProjChunk columns held in registers, then reduced across the warp with a
// fixed butterfly (deterministic).  Roofline: FP64 FMA (2 n^2 k flops against
// n^2 * 8 bytes of Q).
__device__ __forceinline__ void project_column(int64_t n, int k, const double* __restrict__ Q,
                                               const double* __restrict__ K,
                                               double* __restrict__ U, int64_t j, int lane) {
  const double* q = Q + j * n;
  for (int c0 = 0; c0 < k; c0 += kProjChunk) {
    double acc[kProjChunk];
#pragma unroll
    for (int c = 0; c < kProjChunk; ++c) acc[c] = 0.0;
    const int cw = min(kProjChunk, k - c0);
    for (int64_t i = lane; i < n; i += 32) {
      const double qi = q[i];
#pragma unroll
      for (int c = 0; c < kProjChunk; ++c)
        if (c < cw) acc[c] = fma(qi, __ldg(K + (int64_t)(c0 + c) * n + i), acc[c]);
    }
#pragma unroll
    for (int c = 0; c < kProjChunk; ++c) {
      double v = acc[c];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (lane == 0 && c < cw) U[(int64_t)(c0 + c) * n + j] = v;
    }
  }
}

__global__ void __launch_bounds__(256) project_f64_kernel(int64_t n, int k, const double* __restrict__ Q,
                                                          const double* __restrict__ K,
                                                          double* __restrict__ U) {
  const int lane = threadIdx.x & 31;
  const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= n) return;
  project_column(n, k, Q, K, U, j, lane);
}

// Warp w of the grid handles column (w - prefix[p]) of update p.
__global__ void __launch_bounds__(256) project_grouped_kernel(const ProbDesc* __restrict__ P, int count,
                                                              const long long* __restrict__ pre,
                                                              long long total) {
  const int lane = threadIdx.x & 31;
  const long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= total) return;
  const int p = find_owner(pre, count, w);
  const ProbDesc& d = P[p];
  project_column(d.n, d.k, d.Q, d.Km, d.U, w - pre[p], lane);
}

// K = [(e_j + a)/sqrt(2), (e_j - a)/sqrt(2)]: e_j a^T + a e_j^T = K diag(1,-1) K^T.
__global__ void make_rank2_kernel(int64_t n, int64_t j, const double* __restrict__ a,
                                  double* __restrict__ K) {
  const double r = 0.70710678118654752440;  // 1/sqrt(2), correctly rounded
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double e = (i == j) ? 1.0 : 0.0;
    K[i] = (e + a[i]) * r;
    K[n + i] = (e - a[i]) * r;
  }
}

}  // namespace

cudaError_t launch_project_f64(int64_t n, int k, const double* Q, const double* K, double* U,
                               cudaStream_t s) {
  const int warps = 8;
  const int64_t blocks = (n + warps - 1) / warps;
  project_f64_kernel<<<(unsigned)blocks, warps * 32, 0, s>>>(n, k, Q, K, U);
  return cudaGetLastError();
}

cudaError_t launch_project_grouped(const ProbDesc* P, int count, const long long* col_prefix,
                                   long long total_cols, cudaStream_t s) {
  const long long blocks = (total_cols + 7) / 8;
  project_grouped_kernel<<<(unsigned)blocks, 256, 0, s>>>(P, count, col_prefix, total_cols);
  return cudaGetLastError();
}

cudaError_t launch_make_rank2(int64_t n, int64_t j, const double* a, double* K, cudaStream_t s) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  make_rank2_kernel<<<(unsigned)blocks, 256, 0, s>>>(n, j, a, K);
  return cudaGetLastError();
}

}  // namespace eig
