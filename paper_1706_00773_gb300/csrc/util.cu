// util.cu -- small device helpers of the host orchestration.
#include "eig_internal.cuh"

namespace eig {
namespace {

__global__ void copy_guarded_kernel(double* __restrict__ dst, const double* __restrict__ src,
                                    int64_t count, const DevStatus* st, bool vec) {
  if (st && (st->flags & (ST_UNSORTED | ST_NONFINITE))) return;
  if (!vec) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
      dst[i] = src[i];
    return;
  }
  const int64_t n2 = count / 2;
  const double2* s2 = reinterpret_cast<const double2*>(src);
  double2* d2 = reinterpret_cast<double2*>(dst);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2;
       i += (int64_t)gridDim.x * blockDim.x)
    d2[i] = s2[i];
  if (blockIdx.x == 0 && threadIdx.x == 0 && (count & 1)) dst[count - 1] = src[count - 1];
}

// The sub-problem without deflation (every row kept): the layout of the
// deflation kernel's output, for root counts of the problem exactly as given.
__global__ void prepare_undeflated_kernel(int64_t n, int k, int K, const double* __restrict__ lam,
                                          const double* __restrict__ U, double* __restrict__ lam_keep,
                                          double* __restrict__ Us, int ld, int* __restrict__ idx_keep,
                                          DevStatus* st) {
  const int64_t tot = (int64_t)K * ld;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / ld, i = e - c * ld;
    Us[e] = (c < k && i < n) ? U[c * n + i] : 0.0;
    if (c == 0 && i < n) {
      lam_keep[i] = lam[i];
      idx_keep[i] = (int)i;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->n_keep = (int)n;
    st->n_defl = 0;
  }
}

__device__ __forceinline__ int lb(const double* a, int n, double v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ int ub(const double* a, int n, double v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] <= v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void scatter_iters_kernel(Sub sub, int64_t n, const int* __restrict__ root_iters,
                                     const double* __restrict__ lam_defl,
                                     const double* __restrict__ mu_sec, int* __restrict__ out) {
  if (sub.st->flags & (ST_UNSORTED | ST_NONFINITE)) return;
  const int nk = *sub.n_dev;
  const int nd = sub.st->n_defl;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < nk) out[e + lb(lam_defl, nd, mu_sec[e])] = root_iters[e];
    if (e < nd) out[e + ub(mu_sec, nk, lam_defl[e])] = 0;
  }
}

// Column 2 of the per-eigenpair report: the distance of each new eigenvalue
// to its nearest neighbour (over the whole spectrum, deflated pairs included),
// relative to |A|.
__global__ void errors_gap_grouped_kernel(const ProbDesc* __restrict__ P, int count,
                                          const long long* __restrict__ colpre) {
  const long long total = colpre[count];
  for (long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x; item < total;
       item += (long long)gridDim.x * blockDim.x) {
    const int p = find_owner(colpre, count, item);
    const ProbDesc& d = P[p];
    if (!d.errors || (d.st->flags & (ST_UNSORTED | ST_NONFINITE))) continue;
    const int64_t pos = item - colpre[p];
    const double v = d.lam[pos];
    double g = INFINITY;
    if (pos > 0) g = v - d.lam[pos - 1];
    if (pos + 1 < d.n) g = fmin(g, d.lam[pos + 1] - v);
    d.errors[pos + 2 * (int64_t)d.n] = g / (d.st->lam_absmax + d.st->fro2);
  }
}

}  // namespace

cudaError_t launch_errors_gap_grouped(const ProbDesc* P, int count, const long long* colpre, long long total,
                                      cudaStream_t s) {
  long long blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  errors_gap_grouped_kernel<<<(unsigned)blocks, 256, 0, s>>>(P, count, colpre);
  return cudaGetLastError();
}

cudaError_t launch_copy_guarded(double* dst, const double* src, int64_t count, const DevStatus* st,
                                cudaStream_t s) {
  int64_t blocks = (count / 2 + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  if (blocks < 1) blocks = 1;
  const bool vec = ((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15) == 0;
  copy_guarded_kernel<<<(unsigned)blocks, 256, 0, s>>>(dst, src, count, st, vec);
  return cudaGetLastError();
}

cudaError_t launch_prepare_undeflated(int64_t n, int k, int K, const double* lam, const double* U,
                                      double* lam_keep, double* Us, int ld, int* idx_keep,
                                      DevStatus* st, cudaStream_t s) {
  int64_t blocks = ((int64_t)K * ld + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  prepare_undeflated_kernel<<<(unsigned)blocks, 256, 0, s>>>(n, k, K, lam, U, lam_keep, Us, ld,
                                                             idx_keep, st);
  return cudaGetLastError();
}

cudaError_t launch_scatter_iters(const Sub& sub, int64_t n, const int* root_iters,
                                 const double* lam_defl, const double* mu_sec, int* iters_out,
                                 cudaStream_t s) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  scatter_iters_kernel<<<(unsigned)blocks, 256, 0, s>>>(sub, n, root_iters, lam_defl, mu_sec,
                                                        iters_out);
  return cudaGetLastError();
}

}  // namespace eig
