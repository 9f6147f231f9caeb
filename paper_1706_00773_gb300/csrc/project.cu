// project.cu -- U = Q^T K (Sec. 2.1, below eq. (1)) in FP64 or, in mixed
// mode, in double-float arithmetic; and the one-row-one-column
// canonicalisation of Sec. 2.2 (Steps 1-2).
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

// ---- mixed mode: U in double-float arithmetic --------------------------------
// U enters the secular equation, so it needs FP64-level accuracy; pairs of FP32
// (48 bits) accumulated with a two-sum and renormalised after every term keep
// each entry within a few units of 2^-48 of sum_i |Q_ij K_ic| (the FP64 sum's
// bound is n 2^-53 of the same), and run on the FP32 pipe, 64 times the FP64
// pipe's rate on this part.

constexpr int kBadExp = 0x7fffffff;  // a column of K with a non-finite entry

// One CTA per column c of K (blockDim 256): the column scaled by 2^-e (e the
// exponent of its largest entry, so |K 2^-e| < 1) and cut into FP32 high and
// low parts from the bits; entries below 2^-60 of the maximum flush to zero
// (their products are below 2^-60 of the column's own).
__device__ __forceinline__ void split_k_column(int64_t n, int c, const double* __restrict__ K,
                                               float* __restrict__ Kh, float* __restrict__ Kl,
                                               int* __restrict__ Kexp) {
  const double* Kc = K + (int64_t)c * n;
  __shared__ double s_mx[8];
  __shared__ int s_bad[8];
  double mx = 0.0;
  int bad = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = Kc[i];
    bad |= !isfinite(v);
    mx = fmax(mx, fabs(v));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    bad |= __shfl_xor_sync(0xffffffffu, bad, off);
  }
  if ((threadIdx.x & 31) == 0) {
    s_mx[threadIdx.x >> 5] = mx;
    s_bad[threadIdx.x >> 5] = bad;
  }
  __syncthreads();
  mx = 0.0;
  bad = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    mx = fmax(mx, s_mx[w]);
    bad |= s_bad[w];
  }
  int e = 0;
  if (mx > 0.0) frexp(mx, &e);
  if (threadIdx.x == 0) Kexp[c] = bad ? kBadExp : e;
  if (bad) return;
  const double sc = ldexp(1.0, -e);
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    DF v;
    df_bits(Kc[i] * sc, v);  // |.| < 1: false only below 2^-60, a zero pair
    Kh[(int64_t)c * n + i] = v.h;
    Kl[(int64_t)c * n + i] = v.l;
  }
}

// One CTA per (update, column of K) of a table.
__global__ void __launch_bounds__(256) split_k_grouped_kernel(const ProbDesc* __restrict__ P) {
  const ProbDesc& d = P[blockIdx.x / 16];
  const int c = (int)(blockIdx.x % 16);
  if (c >= d.k || !d.Kh) return;  // uniform over the CTA
  split_k_column(d.n, c, d.Km, d.Kh, d.Kl, d.Kexp);
}

__global__ void __launch_bounds__(256) split_k_kernel(int64_t n, const double* __restrict__ K,
                                                      float* __restrict__ Kh, float* __restrict__ Kl,
                                                      int* __restrict__ Kexp) {
  split_k_column(n, (int)blockIdx.x, K, Kh, Kl, Kexp);
}

constexpr int kTileRows = 128;  // rows of K's split per shared-memory tile
constexpr int kRowsPerLane = kTileRows / 32;

// One CTA of eight warps: columns j0 .. j0 + ncols - 1 of Q (warp w: column
// j0 + w), one update.  K's split is staged through shared memory in 128-row
// tiles (two buffers); each lane takes four rows of its column per tile, and
// the next tile's K and Q values are loaded into registers while the current
// tile is summed: one memory latency per 128 rows, K read once per CTA.
// Returns, per warp, whether its column was formed here (false: K has a
// non-finite entry, or the column of Q an entry at or above 2^60 or not
// finite; the caller takes the FP64 path).  Entries of Q below 2^-60 flush to
// zero.  Every thread of the CTA must call it.
__device__ __forceinline__ bool project_cta_df(int64_t n, int k, const double* __restrict__ Q,
                                               const float* __restrict__ Kh, const float* __restrict__ Kl,
                                               const int* __restrict__ Kexp, double* __restrict__ U, int64_t j0,
                                               int ncols) {
  __shared__ float2 sK[2][kProjChunk][kTileRows];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const bool active = w < ncols;
  bool kbad = false;
  for (int c = 0; c < k; ++c) kbad = kbad || (Kexp[c] == kBadExp);
  if (kbad) return false;  // uniform over the CTA
  const double* q = Q + (active ? j0 + w : j0) * n;
  const int ntiles = (int)((n + kTileRows - 1) / kTileRows);
  constexpr int kPer = kProjChunk * kTileRows / 256;  // K elements staged per thread
  bool ok = true;
  for (int c0 = 0; c0 < k; c0 += kProjChunk) {
    const int cw = min(kProjChunk, k - c0);
    float sh[kProjChunk], sl[kProjChunk];
#pragma unroll
    for (int c = 0; c < kProjChunk; ++c) {
      sh[c] = 0.0f;
      sl[c] = 0.0f;
    }
    float2 kn[kPer];
    double qn[kRowsPerLane];
    auto load_tile = [&](int tile) {
      const int64_t i0 = (int64_t)tile * kTileRows;
#pragma unroll
      for (int e = 0; e < kPer; ++e) {
        const int idx = t + 256 * e;
        const int c = idx / kTileRows, r = idx - (idx / kTileRows) * kTileRows;
        const int64_t i = i0 + r;
        kn[e] = (c < cw && i < n) ? make_float2(__ldg(Kh + (int64_t)(c0 + c) * n + i),
                                                __ldg(Kl + (int64_t)(c0 + c) * n + i))
                                  : make_float2(0.0f, 0.0f);
      }
#pragma unroll
      for (int r = 0; r < kRowsPerLane; ++r) {
        const int64_t i = i0 + lane + 32 * r;
        qn[r] = (active && i < n) ? q[i] : 0.0;
      }
    };
    auto store_tile = [&](int buf) {
#pragma unroll
      for (int e = 0; e < kPer; ++e) {
        const int idx = t + 256 * e;
        sK[buf][idx / kTileRows][idx - (idx / kTileRows) * kTileRows] = kn[e];
      }
    };
    load_tile(0);
    store_tile(0);
    double qc[kRowsPerLane];
#pragma unroll
    for (int r = 0; r < kRowsPerLane; ++r) qc[r] = qn[r];
    __syncthreads();
    for (int tile = 0; tile < ntiles; ++tile) {
      const int buf = tile & 1;
      if (tile + 1 < ntiles) load_tile(tile + 1);  // in flight while this tile is summed
#pragma unroll
      for (int r = 0; r < kRowsPerLane; ++r) {
        DF qd;
        if (!df_bits(qc[r], qd)) {
          // a zero pair; only magnitudes >= 2^60, Inf and NaN need FP64
          const int ex = (int)(((unsigned)(__double_as_longlong(qc[r]) >> 32) >> 20) & 0x7ffu) - 1023;
          ok = ok && ex < -60;
        }
        const int row = lane + 32 * r;
#pragma unroll
        for (int c = 0; c < kProjChunk; ++c) {
          if (c < cw) {
            const float2 kv = sK[buf][c][row];
            const float pr = qd.h * kv.x;
            float e = fmaf(qd.h, kv.x, -pr);
            e = fmaf(qd.h, kv.y, e);
            e = fmaf(qd.l, kv.x, e);
            DF tt = df_two_sum(sh[c], pr);
            tt = df_fast(tt.h, tt.l + (sl[c] + e));
            sh[c] = tt.h;
            sl[c] = tt.l;
          }
        }
      }
      if (tile + 1 < ntiles) {
        store_tile(buf ^ 1);
#pragma unroll
        for (int r = 0; r < kRowsPerLane; ++r) qc[r] = qn[r];
      }
      __syncthreads();
    }
    const bool wok = __all_sync(0xffffffffu, ok);
#pragma unroll
    for (int c = 0; c < kProjChunk; ++c) {
      float h = sh[c], l = sl[c];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, h, off), ol = __shfl_xor_sync(0xffffffffu, l, off);
        DF tt = df_two_sum(h, oh);
        tt = df_fast(tt.h, tt.l + (l + ol));
        h = tt.h;
        l = tt.l;
      }
      if (active && wok && lane == 0 && c < cw) {
        // (h + l) 2^e: exact in FP64
        const double v = d_of_bits(h) + d_of_bits(l);
        U[(int64_t)(c0 + c) * n + j0 + w] = ldexp(v, Kexp[c0 + c]);
      }
    }
  }
  return __all_sync(0xffffffffu, ok);
}

// Mixed mode, a table: CTA b takes columns 8b .. 8b + 7 of the table's column
// numbering, update by update when they span several (a column's sums do not
// depend on which CTA or warp forms them, so a batch gives the same U as the
// updates one by one).  An update without K's split takes the FP64 path.
__global__ void __launch_bounds__(256) project_df_grouped_kernel(const ProbDesc* __restrict__ P, int count,
                                                                 const long long* __restrict__ pre,
                                                                 long long total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long c0 = (long long)blockIdx.x * 8;
  const long long c1 = min(c0 + 8, total);  // exclusive
  const int p0 = find_owner(pre, count, c0);
  const int p1 = find_owner(pre, count, c1 - 1);
  for (int p = p0; p <= p1; ++p) {  // uniform over the CTA
    const ProbDesc& d = P[p];
    const long long s0 = max(c0, pre[p]), s1 = min(c1, pre[p + 1]);
    if (s1 <= s0) continue;
    const long long j0 = s0 - pre[p];
    const int ncols = (int)(s1 - s0);
    const bool done = d.Kh ? project_cta_df(d.n, d.k, d.Q, d.Kh, d.Kl, d.Kexp, d.U, j0, ncols) : false;
    if (!done && w < ncols) project_column(d.n, d.k, d.Q, d.Km, d.U, j0 + w, lane);
  }
}

// One update: CTA b takes columns 8b .. 8b + 7.
__global__ void __launch_bounds__(256) project_df_kernel(int64_t n, int k, const double* __restrict__ Q,
                                                         const double* __restrict__ K,
                                                         const float* __restrict__ Kh,
                                                         const float* __restrict__ Kl,
                                                         const int* __restrict__ Kexp, double* __restrict__ U) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t j0 = (int64_t)blockIdx.x * 8;
  const int ncols = (int)min((int64_t)8, n - j0);
  const bool done = project_cta_df(n, k, Q, Kh, Kl, Kexp, U, j0, ncols);
  if (!done && w < ncols) project_column(n, k, Q, K, U, j0 + w, lane);
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

cudaError_t launch_project_mixed(int64_t n, int k, const double* Q, const double* K, double* U, float* Kh,
                                 float* Kl, int* Kexp, cudaStream_t s) {
  split_k_kernel<<<(unsigned)k, 256, 0, s>>>(n, K, Kh, Kl, Kexp);
  const int warps = 8;
  const int64_t blocks = (n + warps - 1) / warps;
  project_df_kernel<<<(unsigned)blocks, warps * 32, 0, s>>>(n, k, Q, K, Kh, Kl, Kexp, U);
  return cudaGetLastError();
}

cudaError_t launch_project_grouped(const ProbDesc* P, int count, const long long* col_prefix,
                                   long long total_cols, cudaStream_t s, bool mixed) {
  const long long blocks = (total_cols + 7) / 8;
  if (mixed) {
    split_k_grouped_kernel<<<(unsigned)count * 16u, 256, 0, s>>>(P);
    project_df_grouped_kernel<<<(unsigned)blocks, 256, 0, s>>>(P, count, col_prefix, total_cols);
  } else {
    project_grouped_kernel<<<(unsigned)blocks, 256, 0, s>>>(P, count, col_prefix, total_cols);
  }
  return cudaGetLastError();
}

cudaError_t launch_make_rank2(int64_t n, int64_t j, const double* a, double* K, cudaStream_t s) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  make_rank2_kernel<<<(unsigned)blocks, 256, 0, s>>>(n, j, a, K);
  return cudaGetLastError();
}

}  // namespace eig
