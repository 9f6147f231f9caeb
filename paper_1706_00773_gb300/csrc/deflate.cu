// deflate.cu -- deflation and compaction of the secular sub-problem.
//
// The paper assumes distinct lam and nonzero rows of U (Sec. 2.1); it is
// silent on what to do otherwise.  Row i is dropped when
//     |u_i|_2 * |U|_F <= 8 eps (max|lam| + |U|_F^2),
// the size of the change to A' that zeroing it makes; the pair keeps mu = lam_i
// and the old eigenvector.  The kept rows form the sub-problem diag(lam') +
// U' Sigma U'^T that the secular kernels solve.
//
// One CTA does everything (reductions, flags, scan, compaction) so that every
// sum is taken in one fixed order (deterministic, no atomics).  Its cost is a
// single pass over U (n k doubles), negligible next to the secular solve.
#include <math.h>

#include "eig_internal.cuh"

namespace eig {
namespace {

constexpr int kDeflThreads = 1024;

__device__ double block_sum(double v, double* sh) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int s = kDeflThreads / 2; s > 0; s >>= 1) {
    if (t < s) sh[t] += sh[t + s];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

__device__ double block_max(double v, double* sh) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int s = kDeflThreads / 2; s > 0; s >>= 1) {
    if (t < s) sh[t] = fmax(sh[t], sh[t + s]);
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

// Exclusive prefix sum of one int per thread (Hillis-Steele in shared memory).
__device__ int block_exclusive_scan(int v, int* sh, int* total) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int off = 1; off < kDeflThreads; off <<= 1) {
    int add = (t >= off) ? sh[t - off] : 0;
    __syncthreads();
    sh[t] += add;
    __syncthreads();
  }
  int incl = sh[t];
  *total = sh[kDeflThreads - 1];
  __syncthreads();
  return incl - v;
}

__device__ __forceinline__ double row_norm2(const double* __restrict__ U, int64_t n, int k,
                                            int64_t i) {
  double s = 0.0;
  for (int c = 0; c < k; ++c) {
    double u = U[(int64_t)c * n + i];
    s = fma(u, u, s);
  }
  return s;
}

__device__ __forceinline__ void deflate_body(
    int64_t n, int k, int K, const double* __restrict__ lam, const double* __restrict__ U,
    unsigned long long negmask, double* __restrict__ lam_keep, double* __restrict__ Us, int ld,
    int* __restrict__ idx_keep, int* __restrict__ idx_defl, double* __restrict__ lam_defl,
    DevStatus* st, double* __restrict__ lam_old, float2* __restrict__ lamf = nullptr,
    float* __restrict__ Usf = nullptr, float* __restrict__ Ulo = nullptr) {
  __shared__ double shd[kDeflThreads];
  __shared__ int shi[kDeflThreads];
  __shared__ double colsq[EIG_MAX_K];
  const int t = threadIdx.x;

  // lam: finite, ascending, largest magnitude; U: finite.
  int bad = 0;
  double amax = 0.0;
  for (int64_t i = t; i < n; i += kDeflThreads) {
    const double v = lam[i];
    if (lam_old) lam_old[i] = v;
    if (!isfinite(v)) bad |= ST_NONFINITE;
    if (i > 0 && !(lam[i - 1] <= v)) bad |= ST_UNSORTED;
    amax = fmax(amax, fabs(v));
  }
  for (int c = 0; c < k; ++c) {
    double part = 0.0;
    for (int64_t i = t; i < n; i += kDeflThreads) {
      const double u = U[(int64_t)c * n + i];
      if (!isfinite(u)) bad |= ST_NONFINITE;
      part = fma(u, u, part);
    }
    const double tot = block_sum(part, shd);
    if (t == 0) colsq[c] = tot;
  }
  amax = block_max(amax, shd);
  shi[t] = bad;
  __syncthreads();
  for (int s = kDeflThreads / 2; s > 0; s >>= 1) {
    if (t < s) shi[t] |= shi[t + s];
    __syncthreads();
  }
  bad = shi[0];
  __syncthreads();

  double fro2 = 0.0, splus = 0.0, sminus = 0.0;
  for (int c = 0; c < k; ++c) {
    fro2 += colsq[c];
    if ((negmask >> c) & 1ull) sminus += colsq[c]; else splus += colsq[c];
  }
  const double fro = sqrt(fro2);
  const double tol = 8.0 * kEps * (amax + fro2);

  // Chunked compaction: thread t owns rows [beg, end).
  const int64_t chunk = (n + kDeflThreads - 1) / kDeflThreads;
  const int64_t beg = min((int64_t)t * chunk, n);
  const int64_t end = min(beg + chunk, n);
  int cnt = 0;
  for (int64_t i = beg; i < end; ++i) cnt += (sqrt(row_norm2(U, n, k, i)) * fro > tol);
  int nkeep = 0;
  const int off = block_exclusive_scan(cnt, shi, &nkeep);
  int pk = off;
  int pd = (int)beg - off;
  for (int64_t i = beg; i < end; ++i) {
    if (sqrt(row_norm2(U, n, k, i)) * fro > tol) {
      lam_keep[pk] = lam[i];
      idx_keep[pk] = (int)i;
      for (int c = 0; c < k; ++c) Us[(int64_t)c * ld + pk] = U[(int64_t)c * n + i];
      if (lamf) {
        // lam = hi + lo + O(2^-48 |lam|): the FP32 phase forms lam_i - lam_o from the pairs
        const float hi = (float)lam[i];
        lamf[pk] = make_float2(hi, (float)(lam[i] - (double)hi));
        for (int c = 0; c < k; ++c) {
          const double u = U[(int64_t)c * n + i];
          const float uh = (float)u;
          Usf[(int64_t)c * ld + pk] = uh;
          if (Ulo) Ulo[(int64_t)c * ld + pk] = (float)(u - (double)uh);
        }
      }
      ++pk;
    } else {
      idx_defl[pd] = (int)i;
      lam_defl[pd] = lam[i];
      ++pd;
    }
  }
  // Zero the tail rows and the padding columns the kernels may touch.
  for (int c = 0; c < K; ++c) {
    const int64_t from = (c < k) ? nkeep : 0;
    for (int64_t i = from + t; i < ld; i += kDeflThreads) {
      Us[(int64_t)c * ld + i] = 0.0;
      if (Usf) Usf[(int64_t)c * ld + i] = 0.0f;
      if (Ulo) Ulo[(int64_t)c * ld + i] = 0.0f;
    }
  }
  __syncthreads();
  if (t == 0) {
    st->flags |= bad;
    st->n_keep = nkeep;
    st->n_defl = (int)(n - nkeep);
    st->lam_absmax = amax;
    st->fro2 = fro2;
    if (nkeep > 0) {
      const double l0 = lam_keep[0], l1 = lam_keep[nkeep - 1];
      // Weyl: every eigenvalue of diag(lam') + U' Sigma U'^T lies in
      // [lam'_min - sum_{sigma<0} |U_c|^2, lam'_max + sum_{sigma>0} |U_c|^2].
      st->lo_sent = l0 - 2.0 * sminus - 4.0 * kEps * fabs(l0) - 1e-300;
      st->hi_sent = l1 + 2.0 * splus + 4.0 * kEps * fabs(l1) + 1e-300;
    } else {
      st->lo_sent = 0.0;
      st->hi_sent = 0.0;
    }
  }
}

__global__ void __launch_bounds__(kDeflThreads) deflate_kernel(
    int64_t n, int k, int K, const double* __restrict__ lam, const double* __restrict__ U,
    unsigned long long negmask, double* __restrict__ lam_keep, double* __restrict__ Us, int ld,
    int* __restrict__ idx_keep, int* __restrict__ idx_defl, double* __restrict__ lam_defl,
    DevStatus* st, float2* __restrict__ lamf, float* __restrict__ Usf) {
  deflate_body(n, k, K, lam, U, negmask, lam_keep, Us, ld, idx_keep, idx_defl, lam_defl, st, nullptr, lamf,
               Usf);
}

// One CTA per update of the table.
__global__ void __launch_bounds__(kDeflThreads) deflate_grouped_kernel(const ProbDesc* __restrict__ P) {
  const ProbDesc& d = P[blockIdx.x];
  deflate_body(d.n, d.k, d.K, d.lam, d.U, d.negmask, d.lam_keep, d.Us, d.ld, d.idx_keep, d.idx_defl,
               d.lam_defl, d.st, d.lam_old, d.lamf, d.Usf, d.Ulo);
}

// u_ia u_ib for every kept row i and a <= b (the upper triangle row by row),
// written as K(K+1)/2 arrays of ld doubles; one thread per row.
__global__ void products_grouped_kernel(const ProbDesc* __restrict__ P, int count,
                                        const long long* __restrict__ colpre) {
  const long long total = colpre[count];
  for (long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x; item < total;
       item += (long long)gridDim.x * blockDim.x) {
    const int q = find_owner(colpre, count, item);
    const ProbDesc& d = P[q];
    if (!d.Pp || (d.st->flags & (ST_UNSORTED | ST_NONFINITE))) continue;
    const int i = (int)(item - colpre[q]);
    if (i >= d.st->n_keep) continue;
    const int K = d.K, ld = d.ld;
    int s = 0;
    for (int a = 0; a < K; ++a) {
      const double ua = d.Us[(size_t)a * ld + i];
      for (int b = a; b < K; ++b, ++s) d.Pp[(size_t)s * ld + i] = ua * d.Us[(size_t)b * ld + i];
    }
  }
}

__global__ void products_kernel(const double* __restrict__ Us, int K, int ld, const DevStatus* st,
                                double* __restrict__ Pp) {
  if (st->flags & (ST_UNSORTED | ST_NONFINITE)) return;
  const int nk = st->n_keep;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nk; i += gridDim.x * blockDim.x) {
    int s = 0;
    for (int a = 0; a < K; ++a) {
      const double ua = Us[(size_t)a * ld + i];
      for (int b = a; b < K; ++b, ++s) Pp[(size_t)s * ld + i] = ua * Us[(size_t)b * ld + i];
    }
  }
}

}  // namespace

cudaError_t launch_products(const double* Us, int K, int ld, const DevStatus* st, double* Pp, cudaStream_t s) {
  int blocks = (ld + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  products_kernel<<<blocks, 256, 0, s>>>(Us, K, ld, st, Pp);
  return cudaGetLastError();
}

cudaError_t launch_products_grouped(const ProbDesc* P, int count, const long long* colpre, long long total,
                                    cudaStream_t s) {
  long long blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  products_grouped_kernel<<<(unsigned)blocks, 256, 0, s>>>(P, count, colpre);
  return cudaGetLastError();
}

cudaError_t launch_deflate_grouped(const ProbDesc* P, int count, cudaStream_t s) {
  deflate_grouped_kernel<<<count, kDeflThreads, 0, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_deflate(int64_t n, int k, int K, const double* lam, const double* U,
                           unsigned long long negmask, double* lam_keep, double* Us, int ld,
                           int* idx_keep, int* idx_defl, double* lam_defl, DevStatus* st,
                           cudaStream_t s, float2* lamf, float* Usf) {
  deflate_kernel<<<1, kDeflThreads, 0, s>>>(n, k, K, lam, U, negmask, lam_keep, Us, ld, idx_keep,
                                            idx_defl, lam_defl, st, lamf, Usf);
  return cudaGetLastError();
}

}  // namespace eig
