// gemm_f64.cu -- C = A B in FP64 on the CUDA cores (column-major), used for
// X = Q W (Sec. 2.4, eq. (10)) in the FP64 mode and by the residual check.
//
// 64 x 64 output tile per 256-thread CTA, 4 x 4 outputs per thread, K staged
// 16 at a time in shared memory.  On GB300 the FP64 pipe issues 2 DFMA/clk/SM,
// so a tile step (16 KB of operands for 65,536 DFMA) needs ~0.5 B/clk/SM:
// the kernel is bound by the FP64 pipe, not by memory.
#include "eig_internal.cuh"

namespace eig {
namespace {

constexpr int BM = 64, BN = 64, BK = 16;

__device__ __forceinline__ void gemm_f64_tile(int64_t m, int64_t n, int64_t k,
                                              const double* __restrict__ A, int64_t lda,
                                              const double* __restrict__ B, int64_t ldb,
                                              double* __restrict__ C, int64_t ldc, int64_t row0,
                                              int64_t col0) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;  // 16 x 16 threads
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int64_t k0 = 0; k0 < k; k0 += BK) {
    // A tile: BM rows x BK cols (column-major source); 1024 doubles, 4 per thread.
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e = tid + t * 256;
      const int r = e & (BM - 1), c = e >> 6;
      const int64_t gr = row0 + r, gc = k0 + c;
      As[c][r] = (gr < m && gc < k) ? A[gr + gc * lda] : 0.0;
    }
    // B tile: BK rows x BN cols.
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e = tid + t * 256;
      const int r = e & (BK - 1), c = e >> 4;
      const int64_t gr = k0 + r, gc = col0 + c;
      Bs[r][c] = (gr < k && gc < n) ? B[gr + gc * ldb] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gr = row0 + tx + 16 * i;
    if (gr >= m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gc = col0 + ty + 16 * j;
      if (gc < n) C[gr + gc * ldc] = acc[i][j];
    }
  }
}

__global__ void __launch_bounds__(256) gemm_f64_kernel(int64_t m, int64_t n, int64_t k,
                                                       const double* __restrict__ A, int64_t lda,
                                                       const double* __restrict__ B, int64_t ldb,
                                                       double* __restrict__ C, int64_t ldc,
                                                       const DevStatus* st) {
  if (st && (st->flags & (ST_UNSORTED | ST_NONFINITE))) return;
  gemm_f64_tile(m, n, k, A, lda, B, ldb, C, ldc, (int64_t)blockIdx.x * BM, (int64_t)blockIdx.y * BN);
}

// X = Q W for every update of a table; CTA b handles tile (b - prefix[p]) of update p.
__global__ void __launch_bounds__(256) gemm_f64_grouped_kernel(const ProbDesc* __restrict__ P, int count,
                                                               const int* __restrict__ tile_prefix) {
  const int p = find_owner(tile_prefix, count, (int)blockIdx.x);
  const ProbDesc& d = P[p];
  if (d.st->flags & (ST_UNSORTED | ST_NONFINITE)) return;
  const int tm = (d.n + BM - 1) / BM;
  const int local = (int)blockIdx.x - tile_prefix[p];
  gemm_f64_tile(d.n, d.n, d.n, d.Q, d.n, d.W, d.n, d.Xout, d.n, (int64_t)(local % tm) * BM,
                (int64_t)(local / tm) * BN);
}

__global__ void copyback_grouped_kernel(const ProbDesc* __restrict__ P, int count,
                                        const long long* __restrict__ pre, long long total) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int p = find_owner(pre, count, e);
    const ProbDesc& d = P[p];
    if (!d.Qback || (d.st->flags & (ST_UNSORTED | ST_NONFINITE))) continue;
    const long long i = e - pre[p];
    d.Qback[i] = d.Xout[i];
  }
}

}  // namespace

cudaError_t launch_gemm_f64_grouped(const ProbDesc* P, int count, const int* tile_prefix, int total_tiles,
                                    cudaStream_t s) {
  gemm_f64_grouped_kernel<<<total_tiles, 256, 0, s>>>(P, count, tile_prefix);
  return cudaGetLastError();
}

cudaError_t launch_copyback_grouped(const ProbDesc* P, int count, const long long* elem_prefix,
                                    long long total, cudaStream_t s) {
  long long blocks = (total + 255) / 256;
  if (blocks > 16384) blocks = 16384;
  if (blocks < 1) blocks = 1;
  copyback_grouped_kernel<<<(unsigned)blocks, 256, 0, s>>>(P, count, elem_prefix, total);
  return cudaGetLastError();
}

cudaError_t launch_gemm_f64_guarded(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda,
                                    const double* B, int64_t ldb, double* C, int64_t ldc,
                                    const DevStatus* st, cudaStream_t s) {
  dim3 grid((unsigned)((m + BM - 1) / BM), (unsigned)((n + BN - 1) / BN));
  gemm_f64_kernel<<<grid, 256, 0, s>>>(m, n, k, A, lda, B, ldb, C, ldc, st);
  return cudaGetLastError();
}

cudaError_t launch_gemm_f64(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda,
                            const double* B, int64_t ldb, double* C, int64_t ldc, cudaStream_t s) {
  return launch_gemm_f64_guarded(m, n, k, A, lda, B, ldb, C, ldc, nullptr, s);
}

}  // namespace eig
