// runs.cu -- runs of exactly repeated eigenvalues.
//
// The paper assumes distinct lam (Sec. 2.1).  On a run G of m >= 2 equal lam,
// A = Q diag(lam) Q^T does not change when Q_G becomes Q_G H^T for any
// orthogonal H, and U_G = Q_G^T K then becomes H U_G.  Householder reflectors
// H = H_{r-1} ... H_0 (r = min(m - 1, k)) reduce U_G to upper-trapezoidal R:
// the run's rows past min(m, k) become zero and rows past rank(U_G) sit at
// rounding level, so the row deflation drops them and the secular problem keeps
// the pole at most min(m, k) times.  (Left alone, a run longer than k leaves
// m - k roots exactly on the pole, where no pole interval can bracket them.)
//
// The eigenvectors then come out in the rotated basis Q~ = Q B, B = diag(I,
// H^T on each run).  The FP64 GEMM paths form X = Q (B W): B is applied to W's
// rows of every run before the GEMM.  The split-BF16 path writes Q~ into the
// output buffer (its GEMM reads only the BF16 slices, so that buffer is free
// until the GEMM writes it) and slices Q~ instead of Q.
//
// Layout: reflector c of the run starting at g0 lives in V[c*n + g0 + i],
// i = c..m-1 (V[c*n + g0 + c] = 1), with tau[g0 + c]; the runs are listed as
// (g0, m) pairs in runs[], their number in DevStatus::n_runs (list order is
// arbitrary; runs are disjoint, so no result depends on it).
#include <math.h>

#include "eig_internal.cuh"

namespace eig {
namespace {

constexpr int kRunThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Householder QR of the m x k block U[g0 .. g0+m) (column stride n) by one warp:
// the block becomes R, the reflectors go to V / tau.
__device__ void run_qr(int64_t n, int k, double* __restrict__ U, double* __restrict__ V,
                       double* __restrict__ tau, int64_t g0, int64_t m, int lane) {
  const int r = (int)min(m - 1, (int64_t)k);
  for (int c = 0; c < r; ++c) {
    double* x = U + (int64_t)c * n + g0;  // column c of the run, rows c..m-1 active
    const double alpha = x[c];
    double amax = 0.0;
    for (int64_t i = c + 1 + lane; i < m; i += 32) amax = fmax(amax, fabs(x[i]));
    amax = warp_max(amax);
    double tc = 0.0, scal = 0.0, beta = alpha;
    if (amax > 0.0) {
      // |x| formed from the entries scaled by their largest magnitude
      const double sc = fmax(amax, fabs(alpha));
      const double inv = 1.0 / sc;
      double ss = 0.0;
      for (int64_t i = c + 1 + lane; i < m; i += 32) {
        const double t = x[i] * inv;
        ss = fma(t, t, ss);
      }
      ss = warp_sum(ss);
      const double a = alpha * inv;
      beta = -copysign(sc * sqrt(fma(a, a, ss)), alpha);
      tc = (beta - alpha) / beta;
      scal = 1.0 / (alpha - beta);
    }
    // H_c = I - tc v v^T with v = [1; x[c+1:] / (alpha - beta)] (tc = 0: H_c = I)
    double* v = V + (int64_t)c * n + g0;
    for (int64_t i = c + lane; i < m; i += 32) v[i] = (i == c) ? 1.0 : x[i] * scal;
    __syncwarp();
    for (int cc = c + 1; cc < k; ++cc) {
      double* y = U + (int64_t)cc * n + g0;
      double s = 0.0;
      for (int64_t i = c + lane; i < m; i += 32) s = fma(v[i], y[i], s);
      s = warp_sum(s) * tc;
      for (int64_t i = c + lane; i < m; i += 32) y[i] = fma(-s, v[i], y[i]);
    }
    __syncwarp();
    for (int64_t i = c + lane; i < m; i += 32) x[i] = (i == c) ? beta : 0.0;
    if (lane == 0) tau[g0 + c] = tc;
    __syncwarp();
  }
}

// Every warp scans 32 consecutive indices per step for run starts; a run is
// reduced by the warp that finds its first index.
__device__ void runs_body(int64_t n, int k, const double* __restrict__ lam, double* __restrict__ U,
                          double* __restrict__ V, double* __restrict__ tau, int* __restrict__ runs,
                          DevStatus* st, int64_t warp, int64_t nwarps, int lane) {
  for (int64_t base = warp * 32; base < n; base += nwarps * 32) {
    const int64_t i = base + lane;
    bool start = false;
    if (i + 1 < n) {
      const double li = lam[i];
      start = (lam[i + 1] == li) && (i == 0 || lam[i - 1] != li);
    }
    unsigned mask = __ballot_sync(0xffffffffu, start);
    while (mask) {
      const int b = __ffs(mask) - 1;
      mask &= mask - 1;
      const int64_t g0 = base + b;
      const double v0 = lam[g0];
      int64_t e = g0 + 1;  // lam[g0 + 1] == v0 by the start test
      for (;;) {
        const int64_t j = e + lane;
        const unsigned same = __ballot_sync(0xffffffffu, j < n && lam[j] == v0);
        if (same == 0xffffffffu) {
          e += 32;
          continue;
        }
        e += __ffs(~same) - 1;
        break;
      }
      run_qr(n, k, U, V, tau, g0, e - g0, lane);
      if (lane == 0) {
        const int slot = atomicAdd(&st->n_runs, 1);
        runs[2 * slot] = (int)g0;
        runs[2 * slot + 1] = (int)(e - g0);
        atomicAdd(&st->run_rows, (int)(e - g0));
      }
    }
  }
}

// Y <- B Y on the rows of every run: Y_G <- H_0 H_1 ... H_{r-1} Y_G, one warp
// per (run, column) pair.
__device__ void apply_runs_rows(int64_t n, int k, const double* __restrict__ V,
                                const double* __restrict__ tau, const int* __restrict__ runs, int nruns,
                                double* __restrict__ Y, int64_t ldy, int64_t ncols, int64_t warp,
                                int64_t nwarps, int lane) {
  const int64_t total = (int64_t)nruns * ncols;
  for (int64_t w = warp; w < total; w += nwarps) {
    const int ri = (int)(w / ncols);
    const int64_t col = w - (int64_t)ri * ncols;
    const int64_t g0 = runs[2 * ri], m = runs[2 * ri + 1];
    const int r = (int)min(m - 1, (int64_t)k);
    double* y = Y + col * ldy + g0;
    for (int c = r - 1; c >= 0; --c) {
      const double tc = tau[g0 + c];
      if (tc == 0.0) continue;
      const double* v = V + (int64_t)c * n + g0;
      double s = 0.0;
      for (int64_t i = c + lane; i < m; i += 32) s = fma(v[i], y[i], s);
      s = warp_sum(s) * tc;
      for (int64_t i = c + lane; i < m; i += 32) y[i] = fma(-s, v[i], y[i]);
      __syncwarp();
    }
  }
}

// Q~ = Q B on the columns of every run, in place in Xq (a copy of Q): row rho's
// run segment q becomes H_{r-1} ... H_0 q.  One thread per (run, row) pair;
// consecutive threads take consecutive rows, so every access is coalesced.
__device__ void rotate_runs_cols(int64_t n, int k, const double* __restrict__ V,
                                 const double* __restrict__ tau, const int* __restrict__ runs, int nruns,
                                 double* __restrict__ Xq, int64_t tid, int64_t nthreads) {
  const int64_t total = (int64_t)nruns * n;
  for (int64_t p = tid; p < total; p += nthreads) {
    const int ri = (int)(p / n);
    const int64_t row = p - (int64_t)ri * n;
    const int64_t g0 = runs[2 * ri], m = runs[2 * ri + 1];
    const int r = (int)min(m - 1, (int64_t)k);
    double* q = Xq + g0 * n + row;  // q[i * n] = Q~[row, g0 + i]
    for (int c = 0; c < r; ++c) {
      const double tc = tau[g0 + c];
      if (tc == 0.0) continue;
      const double* v = V + (int64_t)c * n + g0;
      double s = 0.0;
      for (int64_t i = c; i < m; ++i) s = fma(v[i], q[i * n], s);
      s *= tc;
      for (int64_t i = c; i < m; ++i) q[i * n] = fma(-s, v[i], q[i * n]);
    }
  }
}

__global__ void __launch_bounds__(kRunThreads) runs_qr_kernel(int64_t n, int k, const double* __restrict__ lam,
                                                              double* __restrict__ U, double* __restrict__ V,
                                                              double* __restrict__ tau, int* __restrict__ runs,
                                                              DevStatus* st) {
  const int64_t warp = ((int64_t)blockIdx.x * kRunThreads + threadIdx.x) >> 5;
  runs_body(n, k, lam, U, V, tau, runs, st, warp, (int64_t)gridDim.x * (kRunThreads / 32), threadIdx.x & 31);
}

__global__ void __launch_bounds__(kRunThreads) runs_qr_grouped_kernel(const ProbDesc* __restrict__ P) {
  const ProbDesc& d = P[blockIdx.y];
  const int64_t warp = ((int64_t)blockIdx.x * kRunThreads + threadIdx.x) >> 5;
  runs_body(d.n, d.k, d.lam, d.U, d.Vr, d.taur, d.runs, d.st, warp, (int64_t)gridDim.x * (kRunThreads / 32),
            threadIdx.x & 31);
}

__global__ void __launch_bounds__(kRunThreads) runs_apply_w_kernel(int64_t n, int k, const double* __restrict__ V,
                                                                   const double* __restrict__ tau,
                                                                   const int* __restrict__ runs,
                                                                   const DevStatus* st, double* __restrict__ W,
                                                                   int64_t ldw, int64_t ncols) {
  const int nruns = st->n_runs;
  if (nruns == 0) return;
  const int64_t warp = ((int64_t)blockIdx.x * kRunThreads + threadIdx.x) >> 5;
  apply_runs_rows(n, k, V, tau, runs, nruns, W, ldw, ncols, warp, (int64_t)gridDim.x * (kRunThreads / 32),
                  threadIdx.x & 31);
}

__global__ void __launch_bounds__(kRunThreads) runs_apply_w_grouped_kernel(const ProbDesc* __restrict__ P) {
  const ProbDesc& d = P[blockIdx.y];
  const int nruns = d.st->n_runs;
  if (nruns == 0 || (d.st->flags & (ST_UNSORTED | ST_NONFINITE))) return;
  const int64_t warp = ((int64_t)blockIdx.x * kRunThreads + threadIdx.x) >> 5;
  apply_runs_rows(d.n, d.k, d.Vr, d.taur, d.runs, nruns, d.W, d.n, d.n, warp,
                  (int64_t)gridDim.x * (kRunThreads / 32), threadIdx.x & 31);
}

// Split-BF16 path, step 1: Xout = Q (only when the update has runs).
__global__ void __launch_bounds__(kRunThreads) runs_copy_q_grouped_kernel(const ProbDesc* __restrict__ P) {
  const ProbDesc& d = P[blockIdx.y];
  if (d.st->n_runs == 0 || (d.st->flags & (ST_UNSORTED | ST_NONFINITE))) return;
  const int64_t nn = (int64_t)d.n * d.n;
  for (int64_t i = (int64_t)blockIdx.x * kRunThreads + threadIdx.x; i < nn; i += (int64_t)gridDim.x * kRunThreads)
    d.Xout[i] = d.Q[i];
}

// Split-BF16 path, step 2: rotate the run columns of Xout.
__global__ void __launch_bounds__(kRunThreads) runs_rotate_q_grouped_kernel(const ProbDesc* __restrict__ P) {
  const ProbDesc& d = P[blockIdx.y];
  const int nruns = d.st->n_runs;
  if (nruns == 0 || (d.st->flags & (ST_UNSORTED | ST_NONFINITE))) return;
  rotate_runs_cols(d.n, d.k, d.Vr, d.taur, d.runs, nruns, d.Xout, (int64_t)blockIdx.x * kRunThreads + threadIdx.x,
                   (int64_t)gridDim.x * kRunThreads);
}

int grouped_width(int count, int most) {
  int bx = 1024 / (count > 0 ? count : 1);
  return bx < 1 ? 1 : (bx > most ? most : bx);
}

}  // namespace

cudaError_t launch_runs_qr(int64_t n, int k, const double* lam, double* U, double* V, double* tau, int* runs,
                           DevStatus* st, cudaStream_t s) {
  const int64_t blocks = (n + kRunThreads - 1) / kRunThreads;
  runs_qr_kernel<<<(unsigned)(blocks < 1024 ? blocks : 1024), kRunThreads, 0, s>>>(n, k, lam, U, V, tau, runs, st);
  return cudaGetLastError();
}

cudaError_t launch_runs_qr_grouped(const ProbDesc* P, int count, int64_t max_n, cudaStream_t s) {
  const int64_t need = (max_n + kRunThreads - 1) / kRunThreads;
  const int bx = grouped_width(count, (int)(need < 256 ? (need < 1 ? 1 : need) : 256));
  runs_qr_grouped_kernel<<<dim3(bx, count), kRunThreads, 0, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_runs_apply_w(int64_t n, int k, const double* V, const double* tau, const int* runs,
                                const DevStatus* st, double* W, int64_t ldw, int64_t ncols, int num_sms,
                                cudaStream_t s) {
  runs_apply_w_kernel<<<2 * num_sms, kRunThreads, 0, s>>>(n, k, V, tau, runs, st, W, ldw, ncols);
  return cudaGetLastError();
}

cudaError_t launch_runs_apply_w_grouped(const ProbDesc* P, int count, int num_sms, cudaStream_t s) {
  runs_apply_w_grouped_kernel<<<dim3(grouped_width(count, 2 * num_sms), count), kRunThreads, 0, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_runs_rotate_q_grouped(const ProbDesc* P, int count, int num_sms, cudaStream_t s) {
  const dim3 grid(grouped_width(count, 2 * num_sms), count);
  runs_copy_q_grouped_kernel<<<grid, kRunThreads, 0, s>>>(P);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  runs_rotate_q_grouped_kernel<<<grid, kRunThreads, 0, s>>>(P);
  return cudaGetLastError();
}

}  // namespace eig
