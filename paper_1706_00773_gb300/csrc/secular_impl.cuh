// secular_impl.cuh -- the FP64 secular stage of the rank-k update: kernels and
// per-rank launch templates.  Included by secular.cu (dispatch and the
// rank-independent kernels) and by secular_perk.cu, which the build compiles
// once per padded rank K (-DEIG_SECULAR_K=K) so that the ranks compile in
// parallel; each rank's entry points are instantiated there only.
//
//
//   count(x) = #{mu < x} = #{lam_i < x} + neg(M(x) - Sigma) - k_plus        (1)
//   M(x) = sum_i u_i u_i^T / (x - lam_i),  N(x) = sum_i u_i u_i^T / (x - lam_i)^2
//
// (1) is the integer the modified Sturm chain of Sec. 2.2 (eqs. 4-6) delivers:
// the number of roots of f(x) = det(I - Sigma U^T (xI - Lambda)^{-1} U) (eq. 1)
// below x.  It follows from Sylvester's law of inertia applied to the bordered
// matrix [[Lambda - xI, U], [U^T, -Sigma]], whose two Schur complements are
// A' - xI and M(x) - Sigma.  It is exact in exact arithmetic, needs no chain
// construction (the long division of Sec. 2.2 is unstable), and costs one
// O(n k^2) reduction plus a k x k eigen-decomposition.
//
// Kernels
//   counts_kernel  count at every pole (limit from the left) or at given x:
//                  the location sub-problem of Sec. 2.1/2.2.
//   roots_kernel   the root-value sub-problem (Sec. 2.3).  Each root m is first
//                  placed in the pole interval that holds it (from the pole
//                  counts), measured from its nearest pole (x = lam_o + tau, so
//                  that every x - lam_i keeps full relative accuracy), then
//                  refined by Newton on p(x) = (x - lam_a)(x - lam_b) det(Sigma - M(x))
//                  (lam_a, lam_b the interval's poles, so p is smooth there),
//                  safeguarded by bisection on (1) -- the one-point case of the
//                  paper's divide-and-conquer zero finder.
//   assemble_*     eq. (10): w_i = (u_i^T alpha_0) / (lam_i - mu), normalised,
//                  scattered into W; new eigenvalues merged with deflated ones.
//
// Work layout.  FP64 runs at 2 DFMA/clk/SM on GB300, so a term (8(k+1) bytes
// of U and lam) feeds ~k^2 DFMAs: operand traffic is far below L1/L2
// bandwidth and the kernels read terms straight from global memory (L2
// resident).  One warp (K <= 8) or a group of 2 or 4 warps (K <= 16) owns a
// root; lanes split the terms, the warps of a group split the k(k+1)/2 matrix
// entries (rows a and K-1-a paired, pairs dealt round-robin), and each lane
// keeps its partial sums in registers.  The k x k eigen-decomposition is a
// warp-parallel cyclic Jacobi in shared memory.
#pragma once
#include <math.h>

#include "eig_internal.cuh"

namespace eig {
namespace {

// ----------------------------------------------------------------------------
// Compile-time partition of the upper triangle of a K x K matrix.
// ----------------------------------------------------------------------------
template <int K, int E>
__host__ __device__ constexpr int owner_of(int a) {
  return (a < K - 1 - a ? a : K - 1 - a) % E;
}
template <int K, int E, int e>
__host__ __device__ constexpr int nslots() {
  int s = 0;
  for (int a = 0; a < K; ++a)
    if (owner_of<K, E>(a) == e) s += K - a;
  return s;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// FP32 butterfly: the sums taken in FP32 are also reduced across the warp in
// FP32 (five more roundings per sum, in the error bounds' L + 16; every lane
// ends with the same value).
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

template <int E>
__device__ __forceinline__ void group_sync(int g) {
  if (E == 1) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(32 * E) : "memory");
  }
}

// ACC_MN: M and N in FP64 (the zero finder, FP64 mode); ACC_MN32: M in FP64,
// N (used only for Newton derivatives and first-order updates, which tolerate
// FP32 relative error) in FP32 from the FP32 copy of U'; ACC_MG: M and the
// terms on the point (the counts).  Only ACC_MG counts #{lam_i < x}: inside a
// root's bracket that number is the pole index.
enum { ACC_M = 0, ACC_MN = 1, ACC_MG = 2, ACC_MN32 = 3 };

template <bool C, typename T, typename F>
struct pick_type {
  using type = T;
};
template <typename T, typename F>
struct pick_type<false, T, F> {
  using type = F;
};

// Sum over the kept terms of u_i u_i^T * r_i (r_i = 1/(x - lam_i)) into A and,
// per MODE, of u_i u_i^T r_i^2 into B (ACC_MN) or, for terms sitting exactly on
// the point (x == lam_i), u_i u_i^T into B (ACC_MG).  x = tau when absolute,
// else lam_o + tau with x - lam_i formed as tau - (lam_i - lam_o).  Lane 0
// writes the owned entries of the reduced sums into the symmetric K x K
// shared-memory matrices sA, sB (row stride K+1).  Returns #{lam_i < x}.
template <int K, int E, int e, int MODE>
__device__ __forceinline__ int accumulate(const double* __restrict__ lam,
                                          const double* __restrict__ Us, int ld, int n,
                                          double lam_o, bool absolute, double tau, int skip_a,
                                          int skip_b, double* sA, double* sB, int lane,
                                          const float* __restrict__ Usf = nullptr) {
  constexpr int NS = nslots<K, E, e>();
  constexpr int KP = K + 1;
  using BT = typename pick_type<MODE == ACC_MN32, float, double>::type;
  double A[NS];
  BT B[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    A[s] = 0.0;
    B[s] = (BT)0;
  }
  int below = 0;
  for (int i = lane; i < n; i += 32) {
    const double li = __ldg(lam + i);
    const double d = absolute ? (tau - li) : (tau - (li - lam_o));
    if (MODE == ACC_MG) below += (d > 0.0) ? 1 : 0;
    double u[K];
#pragma unroll
    for (int c = 0; c < K; ++c) u[c] = __ldg(Us + (size_t)c * ld + i);
    if (MODE == ACC_MG && d == 0.0) {
      int s = 0;
#pragma unroll
      for (int a = 0; a < K; ++a) {
        if (owner_of<K, E>(a) == e) {
#pragma unroll
          for (int b = a; b < K; ++b) {
            B[s] = (BT)fma(u[a], u[b], (double)B[s]);
            ++s;
          }
        }
      }
    } else {
      // Terms skip_a / skip_b (the poles bracketing a root) are left out of the
      // sums; the caller carries them exactly in a bordered matrix.
      const double r = (i == skip_a || i == skip_b) ? 0.0 : rcp_nr(d);
      // t = r u: M += t u^T, N += t t^T (= r^2 u u^T).
      double t[K];
#pragma unroll
      for (int c = 0; c < K; ++c) t[c] = u[c] * r;
      float tf[K];
      if (MODE == ACC_MN32) {
        const float rf = (float)r;
#pragma unroll
        for (int c = 0; c < K; ++c) tf[c] = __ldg(Usf + (size_t)c * ld + i) * rf;
      }
      int s = 0;
#pragma unroll
      for (int a = 0; a < K; ++a) {
        if (owner_of<K, E>(a) == e) {
#pragma unroll
          for (int b = a; b < K; ++b) {
            A[s] = fma(t[a], u[b], A[s]);
            if (MODE == ACC_MN) B[s] = (BT)fma(t[a], t[b], (double)B[s]);
            if (MODE == ACC_MN32) B[s] = (BT)fmaf(tf[a], tf[b], (float)B[s]);
            ++s;
          }
        }
      }
    }
  }
  double B64[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    A[s] = warp_sum(A[s]);
    if (MODE == ACC_MN32) B64[s] = (double)warp_sum_f((float)B[s]);
    else B64[s] = (MODE != ACC_M) ? warp_sum((double)B[s]) : 0.0;
  }
  if (MODE == ACC_MG) below = __reduce_add_sync(0xffffffffu, below);
  if (lane == 0) {
    int s = 0;
#pragma unroll
    for (int a = 0; a < K; ++a) {
      if (owner_of<K, E>(a) == e) {
#pragma unroll
        for (int b = a; b < K; ++b) {
          sA[a * KP + b] = A[s];
          sA[b * KP + a] = A[s];
          if (MODE != ACC_M) {
            sB[a * KP + b] = B64[s];
            sB[b * KP + a] = B64[s];
          }
          ++s;
        }
      }
    }
  }
  return below;
}

template <int K, int E, int MODE>
__device__ __forceinline__ int accumulate_group(int e, const double* __restrict__ lam,
                                                const double* __restrict__ Us, int ld, int n,
                                                double lam_o, bool absolute, double tau,
                                                int skip_a, int skip_b, double* sA, double* sB,
                                                int lane, const float* __restrict__ Usf = nullptr) {
  // e is warp-uniform: each warp of a group runs the code for its own rows.
  if (E == 1 || e == 0)
    return accumulate<K, E, 0, MODE>(lam, Us, ld, n, lam_o, absolute, tau, skip_a, skip_b, sA, sB,
                                     lane, Usf);
  if (E > 1 && e == 1)
    return accumulate<K, E, (E > 1 ? 1 : 0), MODE>(lam, Us, ld, n, lam_o, absolute, tau, skip_a,
                                                   skip_b, sA, sB, lane, Usf);
  if (E > 2 && e == 2)
    return accumulate<K, E, (E > 2 ? 2 : 0), MODE>(lam, Us, ld, n, lam_o, absolute, tau, skip_a,
                                                   skip_b, sA, sB, lane, Usf);
  return accumulate<K, E, (E > 3 ? 3 : 0), MODE>(lam, Us, ld, n, lam_o, absolute, tau, skip_a,
                                                 skip_b, sA, sB, lane, Usf);
}

// The zero finder's FP64 sums from the products p_i,ab = u_ia u_ib of the
// kept rows (Sub::Pp): M^_ab += r_i p_i,ab, one FMA per entry and no t = r u
// multiplications.  N^ as in accumulate: FP64 N^_ab += r_i^2 p_i,ab (ACC_MN) or
// FP32 from the FP32 copy of U' (ACC_MN32).  Same terms in the same order per
// lane as accumulate; the products themselves are rounded once, so M^ differs
// from accumulate's by rounding only.
template <int K, int E, int e, int MODE>
__device__ __forceinline__ void accumulate_p(const double* __restrict__ lam, const double* __restrict__ Pp,
                                             int ld, int n, double lam_o, double tau, int skip_a, int skip_b,
                                             double* sA, double* sB, int lane, const float* __restrict__ Usf) {
  static_assert(MODE == ACC_MN || MODE == ACC_MN32, "zero-finder sums only");
  constexpr int NS = nslots<K, E, e>();
  constexpr int KP = K + 1;
  using BT = typename pick_type<MODE == ACC_MN32, float, double>::type;
  double A[NS];
  BT B[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    A[s] = 0.0;
    B[s] = (BT)0;
  }
  for (int i = lane; i < n; i += 32) {
    const double d = tau - (__ldg(lam + i) - lam_o);
    const double r = (i == skip_a || i == skip_b) ? 0.0 : rcp_nr(d);
    float tf[K];
    if (MODE == ACC_MN32) {
      const float rf = (float)r;
#pragma unroll
      for (int c = 0; c < K; ++c) tf[c] = __ldg(Usf + (size_t)c * ld + i) * rf;
    }
    const double r2 = (MODE == ACC_MN) ? r * r : 0.0;
    int s = 0, g = 0;  // s: this warp's slot, g: slot of the full upper triangle
#pragma unroll
    for (int a = 0; a < K; ++a) {
#pragma unroll
      for (int b = a; b < K; ++b, ++g) {
        if (owner_of<K, E>(a) == e) {
          const double pv = __ldg(Pp + (size_t)g * ld + i);
          A[s] = fma(r, pv, A[s]);
          if (MODE == ACC_MN) B[s] = (BT)fma(r2, pv, (double)B[s]);
          if (MODE == ACC_MN32) B[s] = (BT)fmaf(tf[a], tf[b], (float)B[s]);
          ++s;
        }
      }
    }
  }
  double B64[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    A[s] = warp_sum(A[s]);
    B64[s] = (MODE == ACC_MN32) ? (double)warp_sum_f((float)B[s]) : warp_sum((double)B[s]);
  }
  if (lane == 0) {
    int s = 0;
#pragma unroll
    for (int a = 0; a < K; ++a) {
      if (owner_of<K, E>(a) == e) {
#pragma unroll
        for (int b = a; b < K; ++b) {
          sA[a * KP + b] = A[s];
          sA[b * KP + a] = A[s];
          sB[a * KP + b] = B64[s];
          sB[b * KP + a] = B64[s];
          ++s;
        }
      }
    }
  }
}

template <int K, int E, int MODE>
__device__ __forceinline__ void accumulate_p_group(int e, const double* __restrict__ lam,
                                                   const double* __restrict__ Pp, int ld, int n, double lam_o,
                                                   double tau, int skip_a, int skip_b, double* sA, double* sB,
                                                   int lane, const float* __restrict__ Usf) {
  if (E == 1 || e == 0)
    accumulate_p<K, E, 0, MODE>(lam, Pp, ld, n, lam_o, tau, skip_a, skip_b, sA, sB, lane, Usf);
  else if (E > 1 && e == 1)
    accumulate_p<K, E, (E > 1 ? 1 : 0), MODE>(lam, Pp, ld, n, lam_o, tau, skip_a, skip_b, sA, sB, lane, Usf);
  else if (E > 2 && e == 2)
    accumulate_p<K, E, (E > 2 ? 2 : 0), MODE>(lam, Pp, ld, n, lam_o, tau, skip_a, skip_b, sA, sB, lane, Usf);
  else
    accumulate_p<K, E, (E > 3 ? 3 : 0), MODE>(lam, Pp, ld, n, lam_o, tau, skip_a, skip_b, sA, sB, lane, Usf);
}

// ----------------------------------------------------------------------------
// FP32 accumulation for the coarse phase of the zero finder (mixed mode).
// The same sums as ACC_MN with x - lam_i formed from (hi, lo) float pairs as
// (th - (hi_i - hi_o)) + (tl - (lo_i - lo_o)), tau = th + tl.  Measured from the
// nearer bracketing pole (|tau| <= half the bracket), every other pole has
// |x - lam_i| >= |lam_i - lam_o| / 2, so each term keeps ~2^-23 relative
// accuracy; the pair representation adds an absolute error of 2^-48 |lam| per
// difference.  Returns the two bound sums of the a-posteriori error of M^,
//   S1 = sum_i |r_i| |u_i|^2   (relative rounding of the terms and the sums),
//   S2 = sum_i r_i^2 |u_i|^2   (times the absolute error of x - lam_i),
// through out2[0], out2[1] (lane 0 of every warp writes the same values).
// ----------------------------------------------------------------------------
template <int K, int E, int e, bool WN>
__device__ __forceinline__ void accumulate32(const float2* __restrict__ lamf, const float* __restrict__ Usf,
                                             int ld, int n, float ho, float lo_o, float th, float tl,
                                             int skip_a, int skip_b, double* sA, double* sB, double* out2,
                                             int lane) {
  constexpr int NS = nslots<K, E, e>();
  constexpr int KP = K + 1;
  float A[NS], B[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    A[s] = 0.0f;
    B[s] = 0.0f;
  }
  float s1 = 0.0f, s2 = 0.0f;
  for (int i = lane; i < n; i += 32) {
    const float2 l = __ldg(lamf + i);
    const float d = (th - (l.x - ho)) + (tl - (l.y - lo_o));
    float u[K];
    float nu = 0.0f;
#pragma unroll
    for (int c = 0; c < K; ++c) {
      u[c] = __ldg(Usf + (size_t)c * ld + i);
      nu = fmaf(u[c], u[c], nu);
    }
    const float r = (i == skip_a || i == skip_b) ? 0.0f : __frcp_rn(d);
    s1 = fmaf(fabsf(r), nu, s1);
    s2 = fmaf(r * r, nu, s2);
    float t[K];
#pragma unroll
    for (int c = 0; c < K; ++c) t[c] = u[c] * r;
    int s = 0;
#pragma unroll
    for (int a = 0; a < K; ++a) {
      if (owner_of<K, E>(a) == e) {
#pragma unroll
        for (int b = a; b < K; ++b) {
          A[s] = fmaf(t[a], u[b], A[s]);
          if (WN) B[s] = fmaf(t[a], t[b], B[s]);
          ++s;
        }
      }
    }
  }
  double A64[NS], B64[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    A64[s] = (double)warp_sum_f(A[s]);
    B64[s] = WN ? (double)warp_sum_f(B[s]) : 0.0;
  }
  const double S1 = (double)warp_sum_f(s1), S2 = (double)warp_sum_f(s2);
  if (lane == 0) {
    int s = 0;
#pragma unroll
    for (int a = 0; a < K; ++a) {
      if (owner_of<K, E>(a) == e) {
#pragma unroll
        for (int b = a; b < K; ++b) {
          sA[a * KP + b] = A64[s];
          sA[b * KP + a] = A64[s];
          if (WN) {
            sB[a * KP + b] = B64[s];
            sB[b * KP + a] = B64[s];
          }
          ++s;
        }
      }
    }
    if (e == 0) {
      out2[0] = S1;
      out2[1] = S2;
    }
  }
}

template <int K, int E, bool WN>
__device__ __forceinline__ void accumulate32_group(int e, const float2* __restrict__ lamf,
                                                   const float* __restrict__ Usf, int ld, int n, float ho,
                                                   float lo_o, float th, float tl, int skip_a, int skip_b,
                                                   double* sA, double* sB, double* out2, int lane) {
  if (E == 1 || e == 0) {
    accumulate32<K, E, 0, WN>(lamf, Usf, ld, n, ho, lo_o, th, tl, skip_a, skip_b, sA, sB, out2, lane);
  } else if (E > 1 && e == 1) {
    accumulate32<K, E, (E > 1 ? 1 : 0), WN>(lamf, Usf, ld, n, ho, lo_o, th, tl, skip_a, skip_b, sA, sB, out2,
                                            lane);
  } else if (E > 2 && e == 2) {
    accumulate32<K, E, (E > 2 ? 2 : 0), WN>(lamf, Usf, ld, n, ho, lo_o, th, tl, skip_a, skip_b, sA, sB, out2,
                                            lane);
  } else {
    accumulate32<K, E, (E > 3 ? 3 : 0), WN>(lamf, Usf, ld, n, ho, lo_o, th, tl, skip_a, skip_b, sA, sB, out2,
                                            lane);
  }
}

// ----------------------------------------------------------------------------
// Warp-parallel Jacobi on a symmetric K x K matrix in shared memory (row
// stride K+1).  On exit the diagonal of A holds the eigenvalues and, if V is
// given, V's columns the orthonormal eigenvectors (accumulated onto V when
// init_v is false).
//
// Round-robin (parallel) ordering: each round rotates ceil(K/2) disjoint index
// pairs at once, one lane per pair computing its angle, then every lane applies
// the rotations to its share of columns, rows and V.  The angle is taken in
// FP32 (t = tan of the rotation): any angle near the annihilating one gives an
// exactly orthogonal rotation when c and s are formed from t in FP64, here
// c = 1/sqrt(1 + t^2) by two Newton steps of the inverse-square-root iteration
// y <- y (3 - x y^2)/2 from an FP32 start, s = t c.  The rotated matrix is
// formed by the rotation itself (no diagonal shortcut), so A stays an exact
// similarity of the input up to rounding; the off-diagonal residual an
// inexact angle leaves is removed by later rounds.
// ----------------------------------------------------------------------------
template <int K>
__device__ void warp_jacobi(double* A, double* V, int lane, bool init_v = true) {
  constexpr int KP = K + 1;
  if (V && init_v) {
    for (int idx = lane; idx < K * K; idx += 32) {
      const int r = idx / K, c = idx - (idx / K) * K;
      V[r * KP + c] = (r == c) ? 1.0 : 0.0;
    }
  }
  __syncwarp();
  if constexpr (K == 1) return;
  constexpr int M = (K + 1) / 2 * 2;  // even number of players (K odd: one idle)
  constexpr int P = M / 2;            // pairs per round
  constexpr int ITEMS = P * K;        // (pair, row) updates per pass
  for (int sweep = 0; sweep < 16; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int idx = lane; idx < K * K; idx += 32) {
      const int r = idx / K, c = idx - (idx / K) * K;
      const double v = A[r * KP + c];
      if (r != c) off = fma(v, v, off); else dia = fma(v, v, dia);
    }
    off = warp_sum(off);
    dia = warp_sum(dia);
    // Converged when the off-diagonal part is 1e-18 of the diagonal (Frobenius).
    // The eigenvalues would be settled at 1e-16 already; the margin is for the
    // eigenvectors of the small eigenvalues (the null vector of Z), which an
    // off-diagonal residual F moves by F / (eigenvalue gap).
    if (off == 0.0 || off <= 1e-36 * dia) break;
    for (int rnd = 0; rnd < M - 1; ++rnd) {
      int pj = 0, qj = 0;
      double cj = 1.0, sj = 0.0;
      bool act = false;
      if (lane < P) {
        int a, b;
        if (lane == 0) {
          a = rnd;
          b = M - 1;
        } else {
          a = (rnd + lane) % (M - 1);
          b = (rnd - lane + (M - 1)) % (M - 1);
        }
        pj = a < b ? a : b;
        qj = a < b ? b : a;
        if (qj < K) {
          const double apq = A[pj * KP + qj], app = A[pj * KP + pj], aqq = A[qj * KP + qj];
          if (apq != 0.0) {
            if (fabs(apq) * 1e18 < fabs(app) && fabs(apq) * 1e18 < fabs(aqq)) {
              A[pj * KP + qj] = 0.0;  // negligible against both diagonal entries
              A[qj * KP + pj] = 0.0;
            } else {
              const float fa = (float)apq;
              if (fa != 0.0f) {
                const float th = (float)(aqq - app) / (2.0f * fa);
                float t;
                if (!(fabsf(th) <= 1e18f)) {
                  t = 0.5f / th;  // also th = +-inf: t = 0
                } else {
                  t = 1.0f / (fabsf(th) + sqrtf(fmaf(th, th, 1.0f)));
                  if (th < 0.0f) t = -t;
                }
                const double td = (double)t;
                const double x = fma(td, td, 1.0);
                double y = (double)rsqrtf((float)x);
                y = y * fma(-0.5 * x * y, y, 1.5);
                y = y * fma(-0.5 * x * y, y, 1.5);
                cj = y;
                sj = td * y;
                act = true;
              }
            }
          }
        }
      }
      __syncwarp();
      // A round whose pairs all need no rotation (warm starts converge to
      // that within a sweep or two) skips the column and row passes.
      if (__ballot_sync(0xffffffffu, act) == 0u) continue;
      // columns: A <- A J
#pragma unroll
      for (int base = 0; base < ITEMS; base += 32) {
        const int idx = base + lane;
        const int jj = idx < ITEMS ? idx / K : 0;
        const int r = idx - jj * K;
        const int p = __shfl_sync(0xffffffffu, pj, jj), q = __shfl_sync(0xffffffffu, qj, jj);
        const double c = __shfl_sync(0xffffffffu, cj, jj), sn = __shfl_sync(0xffffffffu, sj, jj);
        const bool go = __shfl_sync(0xffffffffu, act ? 1 : 0, jj) != 0;
        if (idx < ITEMS && go) {
          const double arp = A[r * KP + p], arq = A[r * KP + q];
          A[r * KP + p] = c * arp - sn * arq;
          A[r * KP + q] = sn * arp + c * arq;
        }
      }
      __syncwarp();
      // rows: A <- J^T A, and V <- V J
#pragma unroll
      for (int base = 0; base < ITEMS; base += 32) {
        const int idx = base + lane;
        const int jj = idx < ITEMS ? idx / K : 0;
        const int r = idx - jj * K;
        const int p = __shfl_sync(0xffffffffu, pj, jj), q = __shfl_sync(0xffffffffu, qj, jj);
        const double c = __shfl_sync(0xffffffffu, cj, jj), sn = __shfl_sync(0xffffffffu, sj, jj);
        const bool go = __shfl_sync(0xffffffffu, act ? 1 : 0, jj) != 0;
        if (idx < ITEMS && go) {
          const double apr = A[p * KP + r], aqr = A[q * KP + r];
          A[p * KP + r] = c * apr - sn * aqr;
          A[q * KP + r] = sn * apr + c * aqr;
          if (V) {
            const double vrp = V[r * KP + p], vrq = V[r * KP + q];
            V[r * KP + p] = c * vrp - sn * vrq;
            V[r * KP + q] = sn * vrp + c * vrq;
          }
        }
      }
      __syncwarp();
    }
  }
}

// The same round-robin Jacobi in FP32, for the k x k work of a count whose
// FP32 result is certified by an error bound (the rotations run on the FP32
// pipe; GB300 issues FP64 at 1/64 of the FP32 rate).  Stops once the
// off-diagonal mass is below 1e-14 of the diagonal's (FP32 resolution).
template <int K>
__device__ void warp_jacobi_f32(float* A, float* V, int lane) {
  constexpr int KP = K + 1;
  if (V) {
    for (int idx = lane; idx < K * K; idx += 32) {
      const int r = idx / K, c = idx - (idx / K) * K;
      V[r * KP + c] = (r == c) ? 1.0f : 0.0f;
    }
  }
  __syncwarp();
  if constexpr (K == 1) return;
  constexpr int M = (K + 1) / 2 * 2;
  constexpr int P = M / 2;
  constexpr int ITEMS = P * K;
  for (int sweep = 0; sweep < 16; ++sweep) {
    float off = 0.0f, dia = 0.0f;
    for (int idx = lane; idx < K * K; idx += 32) {
      const int r = idx / K, c = idx - (idx / K) * K;
      const float v = A[r * KP + c];
      if (r != c) off = fmaf(v, v, off); else dia = fmaf(v, v, dia);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      dia += __shfl_xor_sync(0xffffffffu, dia, o);
    }
    if (off == 0.0f || off <= 1e-14f * dia) break;
    for (int rnd = 0; rnd < M - 1; ++rnd) {
      int pj = 0, qj = 0;
      float cj = 1.0f, sj = 0.0f;
      bool act = false;
      if (lane < P) {
        int a, b;
        if (lane == 0) {
          a = rnd;
          b = M - 1;
        } else {
          a = (rnd + lane) % (M - 1);
          b = (rnd - lane + (M - 1)) % (M - 1);
        }
        pj = a < b ? a : b;
        qj = a < b ? b : a;
        if (qj < K) {
          const float apq = A[pj * KP + qj], app = A[pj * KP + pj], aqq = A[qj * KP + qj];
          if (apq != 0.0f) {
            const float th = (aqq - app) / (2.0f * apq);
            float t;
            if (!(fabsf(th) <= 1e18f)) {
              t = 0.5f / th;
            } else {
              t = 1.0f / (fabsf(th) + sqrtf(fmaf(th, th, 1.0f)));
              if (th < 0.0f) t = -t;
            }
            cj = rsqrtf(fmaf(t, t, 1.0f));
            sj = t * cj;
            act = true;
          }
        }
      }
      __syncwarp();
#pragma unroll
      for (int base = 0; base < ITEMS; base += 32) {
        const int idx = base + lane;
        const int jj = idx < ITEMS ? idx / K : 0;
        const int r = idx - jj * K;
        const int p = __shfl_sync(0xffffffffu, pj, jj), q = __shfl_sync(0xffffffffu, qj, jj);
        const float c = __shfl_sync(0xffffffffu, cj, jj), sn = __shfl_sync(0xffffffffu, sj, jj);
        const bool go = __shfl_sync(0xffffffffu, act ? 1 : 0, jj) != 0;
        if (idx < ITEMS && go) {
          const float arp = A[r * KP + p], arq = A[r * KP + q];
          A[r * KP + p] = c * arp - sn * arq;
          A[r * KP + q] = sn * arp + c * arq;
        }
      }
      __syncwarp();
#pragma unroll
      for (int base = 0; base < ITEMS; base += 32) {
        const int idx = base + lane;
        const int jj = idx < ITEMS ? idx / K : 0;
        const int r = idx - jj * K;
        const int p = __shfl_sync(0xffffffffu, pj, jj), q = __shfl_sync(0xffffffffu, qj, jj);
        const float c = __shfl_sync(0xffffffffu, cj, jj), sn = __shfl_sync(0xffffffffu, sj, jj);
        const bool go = __shfl_sync(0xffffffffu, act ? 1 : 0, jj) != 0;
        if (idx < ITEMS && go) {
          const float apr = A[p * KP + r], aqr = A[q * KP + r];
          A[p * KP + r] = c * apr - sn * aqr;
          A[q * KP + r] = sn * apr + c * aqr;
          if (V) {
            const float vrp = V[r * KP + p], vrq = V[r * KP + q];
            V[r * KP + p] = c * vrp - sn * vrq;
            V[r * KP + q] = sn * vrp + c * vrq;
          }
        }
      }
      __syncwarp();
    }
  }
}

// ----------------------------------------------------------------------------
// Inverse of an N x N matrix Z (row stride N+1, shared memory, left intact) by
// Gauss-Jordan elimination with partial pivoting, one warp: A is the working
// copy, B receives Z^{-1}.  Lane c owns column c of A and of B (N <= 32);
// each step first copies the rows' elimination factors (column j) into the
// spare column N of the row stride, so no factor is overwritten before use.
// Returns false (B invalid) if a pivot is zero or not finite.  *detneg = 1
// when det Z < 0 (pivot signs and row swaps); *zf = |Z|_F, *bf = |Z^{-1}|_F,
// *bkf = |(Z^{-1})_{KK}|_F (the leading KB x KB block).
// ----------------------------------------------------------------------------
template <int N>
__device__ bool warp_gj_inverse(const double* Z, double* A, double* B, int lane, int KB, int* detneg,
                                double* zf, double* bf, double* bkf) {
  constexpr int P = N + 1;
  double z2 = 0.0;
  for (int idx = lane; idx < N * N; idx += 32) {
    const int r = idx / N, c = idx - (idx / N) * N;
    const double v = Z[r * P + c];
    A[r * P + c] = v;
    B[r * P + c] = (r == c) ? 1.0 : 0.0;
    z2 = fma(v, v, z2);
  }
  z2 = warp_sum(z2);
  __syncwarp();
  int neg = 0;
  for (int j = 0; j < N; ++j) {
    double v = (lane >= j && lane < N) ? fabs(A[lane * P + j]) : -1.0;
    int ir = lane;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, v, off);
      const int oi = __shfl_xor_sync(0xffffffffu, ir, off);
      if (ov > v || (ov == v && oi < ir)) {
        v = ov;
        ir = oi;
      }
    }
    if (!(v > 0.0) || !(v < INFINITY)) return false;  // warp-uniform
    if (ir != j) {
      if (lane < N) {
        const double a0 = A[j * P + lane], a1 = A[ir * P + lane];
        A[j * P + lane] = a1;
        A[ir * P + lane] = a0;
        const double b0 = B[j * P + lane], b1 = B[ir * P + lane];
        B[j * P + lane] = b1;
        B[ir * P + lane] = b0;
      }
      neg ^= 1;
      __syncwarp();
    }
    const double pv = A[j * P + j];
    if (pv < 0.0) neg ^= 1;
    const double rp = 1.0 / pv;
    // Row factors (column j) go to the spare column N before any row changes.
    if (lane < N) A[lane * P + N] = A[lane * P + j];
    __syncwarp();
    if (lane < N) {
      A[j * P + lane] *= rp;
      B[j * P + lane] *= rp;
    }
    __syncwarp();
    if (lane < N) {
      const double aj0 = A[j * P + lane];
      const double bj0 = B[j * P + lane];
#pragma unroll 4
      for (int r = 0; r < N; ++r) {
        if (r == j) continue;
        const double fr = A[r * P + N];
        A[r * P + lane] = fma(-fr, aj0, A[r * P + lane]);
        B[r * P + lane] = fma(-fr, bj0, B[r * P + lane]);
      }
    }
    __syncwarp();
  }
  double i2 = 0.0, ik2 = 0.0;
  for (int idx = lane; idx < N * N; idx += 32) {
    const int r = idx / N, c = idx - (idx / N) * N;
    const double b = B[r * P + c];
    i2 = fma(b, b, i2);
    if (r < KB && c < KB) ik2 = fma(b, b, ik2);
  }
  i2 = warp_sum(i2);
  ik2 = warp_sum(ik2);
  *detneg = neg;
  *zf = sqrt(z2);
  *bf = sqrt(i2);
  *bkf = sqrt(ik2);
  return isfinite(i2);
}

__device__ __forceinline__ bool input_invalid(const DevStatus* st) {
  return (st->flags & (ST_UNSORTED | ST_NONFINITE)) != 0;
}

__device__ __forceinline__ double sigma_of(unsigned long long negmask, int a) {
  return ((negmask >> a) & 1ull) ? -1.0 : 1.0;
}

// ----------------------------------------------------------------------------
// counts_kernel: #{mu < x} at the poles (x == nullptr) or at absolute points.
// At a point that coincides with poles, the terms on it blow up along
// R = span{u_i : lam_i = x}; the limit from the left is
//   #{lam_i < x} + dim R + #{positive eigenvalues of (Sigma - M~(x)) on R^perp} - k_plus
// with M~ the sum over the other terms.  Away from poles G = 0 and this is (1).
// ----------------------------------------------------------------------------
// The k x k part of a count at pole q from FP32 sums (M~ in M, S1 and S2 in
// s_err), on the FP32 pipe: the range R of G = u_q u_q^T (FP32 Jacobi on G
// scaled by 1/max|u_q|^2), T = V^T (Sigma - M~) V with R decoupled, and T's
// eigenvalues.  The count is kept only when every eigenvalue on R^perp clears
//   E = 1.25 ((L + 16) 2^-24 S1 + 2^-46 max|lam| S2) + 64 K 2^-24 |B|_F,
// the FP32 error of the sums plus that of the FP32 k x k work (B's rounding,
// the products V^T B V, R's leakage into R^perp, the Jacobi's rotations);
// otherwise *s_redo asks for the FP64 pass.
template <int K>
__device__ void count_tail_f32(const Sub& sub, int n, int pole, const double* M, double* Gm, double* Vg,
                               double* Ev, const double* s_err, int* out, int* s_redo, int lane) {
  constexpr int KP = K + 1;
  float* Gf = reinterpret_cast<float*>(Gm);   // K x KP
  float* Bf = Gf + K * KP;                    // K x KP (Gm holds 2 K KP floats)
  float* Vf = reinterpret_cast<float*>(Vg);   // K x KP
  float* Evf = reinterpret_cast<float*>(Ev);  // K
  const double S1 = s_err[0], S2 = s_err[1];
  float umax = 0.0f;
  for (int r = 0; r < K; ++r) umax = fmaxf(umax, fabsf(sub.Usf[(size_t)r * sub.ld + pole]));
  // 1/0 in FP32 (a repeated pole) or a row below FP32's normal range: FP64 pass.
  if (!(S1 < INFINITY) || !(S2 < INFINITY) || !(umax >= 0x1p-60f)) {
    if (lane == 0) *s_redo = 1;
    __syncwarp();
    return;
  }
  const float us = 1.0f / umax;
  float bsq = 0.0f;
  for (int idx = lane; idx < K * K; idx += 32) {
    const int r = idx / K, c = idx - (idx / K) * K;
    const float b = (float)((r == c ? sigma_of(sub.negmask, r) : 0.0) - M[r * KP + c]);
    Bf[r * KP + c] = b;
    bsq = fmaf(b, b, bsq);
    Gf[r * KP + c] = (sub.Usf[(size_t)r * sub.ld + pole] * us) * (sub.Usf[(size_t)c * sub.ld + pole] * us);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) bsq += __shfl_xor_sync(0xffffffffu, bsq, o);
  __syncwarp();
  warp_jacobi_f32<K>(Gf, Vf, lane);
  if (lane < K) Evf[lane] = Gf[lane * KP + lane];
  __syncwarp();
  float emax = 0.0f;
  for (int j = 0; j < K; ++j) emax = fmaxf(emax, Evf[j]);
  const float tol = 64.0f * 0x1p-24f * (float)K * emax;
  int dimR = 0;
  for (int j = 0; j < K; ++j) dimR += (Evf[j] > tol) ? 1 : 0;
  // T = V^T B V into Gf: lane j forms column j.
  float bv[K];
  if (lane < K) {
#pragma unroll
    for (int r = 0; r < K; ++r) {
      float acc = 0.0f;
      for (int q = 0; q < K; ++q) acc = fmaf(Bf[r * KP + q], Vf[q * KP + lane], acc);
      bv[r] = acc;
    }
  }
  __syncwarp();
  if (lane < K) {
    for (int i = 0; i < K; ++i) {
      float acc = 0.0f;
#pragma unroll
      for (int r = 0; r < K; ++r) acc = fmaf(Vf[r * KP + i], bv[r], acc);
      Gf[i * KP + lane] = acc;
    }
  }
  __syncwarp();
  const bool rng = lane < K && Evf[lane] > tol;  // range directions: diagonal -1, never counted
  if (rng) {
    for (int i = 0; i < K; ++i) {
      Gf[lane * KP + i] = 0.0f;
      Gf[i * KP + lane] = 0.0f;
    }
  }
  __syncwarp();
  if (rng) Gf[lane * KP + lane] = -1.0f;
  __syncwarp();
  warp_jacobi_f32<K>(Gf, nullptr, lane);
  const float v = (lane < K) ? Gf[lane * KP + lane] : 0.0f;
  const unsigned pos = __ballot_sync(0xffffffffu, lane < K && v > 0.0f);
  const int cnt = pole + dimR + __popc(pos) - sub.kplus;
  const double L = (double)((n + 31) / 32);
  const double Eb = 1.25 * ((L + 16.0) * 0x1p-24 * S1 + 0x1p-46 * sub.st->lam_absmax * S2) +
                    64.0 * K * 0x1p-24 * sqrt((double)bsq);
  const bool okj = lane >= K || rng || fabs((double)v) > 2.0 * Eb;
  const bool ok = __all_sync(0xffffffffu, okj) && (Eb < INFINITY);
  if (lane == 0) {
    if (ok) *out = cnt;
    *s_redo = ok ? 0 : 1;
  }
  __syncwarp();
}

// CM selects the passes: 0 = FP32 then, if uncertified, FP64 (one kernel);
// 1 = the FP32 pass only, an uncertified count written as -1; 2 = the FP64
// pass only (the recount launch after a CM = 1 launch).  Split in two launches
// the FP32 pass needs half the registers, so twice the warps stay resident.
template <int K, int CM = 0, int EP = 0>
__device__ __forceinline__ void count_point(const Sub& sub, int n, bool active, bool absolute,
                                            double tau, double lam_o, int pole, int* out, double* M0,
                                            double* Gm, double* Vg, double* Ev, double* s_err, int* s_redo,
                                            int g, int e, int lane) {
  constexpr int E = EP ? EP : warps_per_root(K);  // warps per point
  constexpr int KP = K + 1;
  // At a pole with FP32 copies present, a first pass sums M~ in FP32 and does
  // the k x k work in FP32 too (count_tail_f32, #{lam_i < lam_q} = q); a count
  // that the error bound cannot certify is taken again in FP64.  A repeated
  // or nearly repeated pole gives 1/0 in FP32, an infinite bound, and so the
  // FP64 pass.
  const bool try32 = !absolute && sub.lamf != nullptr && CM != 2;
  constexpr int kLast = (CM == 1) ? 0 : 1;  // CM = 1 never compiles the FP64 pass
  for (int pass = try32 ? 0 : 1; pass <= kLast; ++pass) {
    const bool p32 = (CM == 1) ? true : (CM == 2) ? false : (pass == 0);
    double* M = M0;
    int below = 0;
    if (active) {
      if (p32) {
        const float ho = (float)lam_o;
        accumulate32_group<K, E, false>(e, sub.lamf, sub.Usf, sub.ld, n, ho, (float)(lam_o - (double)ho), 0.0f,
                                        0.0f, pole, -1, M, Gm, s_err, lane);
      } else {
        below = accumulate_group<K, E, ACC_MG>(e, sub.lam, sub.Us, sub.ld, n, lam_o, absolute, tau, -1, -1, M,
                                               Gm, lane);
      }
    }
    group_sync<E>(g);
    if (active && e == 0 && p32) {
      count_tail_f32<K>(sub, n, pole, M, Gm, Vg, Ev, s_err, out, s_redo, lane);
    } else if (active && e == 0) {
      for (int idx = lane; idx < K * K; idx += 32) {
        const int r = idx / K, c = idx - (idx / K) * K;
        const double v = -M[r * KP + c];
        M[r * KP + c] = (r == c) ? v + sigma_of(sub.negmask, r) : v;
      }
      double gmax = 0.0;
      for (int idx = lane; idx < K * K; idx += 32) {
        const int r = idx / K, c = idx - (idx / K) * K;
        gmax = fmax(gmax, fabs(Gm[r * KP + c]));
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1)
        gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, off));
      __syncwarp();
      int dimR = 0;
      if (gmax > 0.0) {
        double* V = Vg;
        warp_jacobi<K>(Gm, V, lane);
        if (lane < K) Ev[lane] = Gm[lane * KP + lane];
        __syncwarp();
        double emax = 0.0;
        for (int j = 0; j < K; ++j) emax = fmax(emax, Ev[j]);
        const double tol = 64.0 * kEps * K * emax;
        for (int j = 0; j < K; ++j) dimR += (Ev[j] > tol) ? 1 : 0;
        // T = V^T B V into Gm: lane j forms column j.
        double bv[K];
        if (lane < K) {
#pragma unroll
          for (int r = 0; r < K; ++r) {
            double acc = 0.0;
            for (int q = 0; q < K; ++q) acc = fma(M[r * KP + q], V[q * KP + lane], acc);
            bv[r] = acc;
          }
        }
        __syncwarp();
        if (lane < K) {
          for (int i = 0; i < K; ++i) {
            double acc = 0.0;
#pragma unroll
            for (int r = 0; r < K; ++r) acc = fma(V[r * KP + i], bv[r], acc);
            Gm[i * KP + lane] = acc;
          }
        }
        __syncwarp();
        // Range directions: decouple them with diagonal -1 (never counted).
        if (lane < K && Ev[lane] > tol) {
          for (int i = 0; i < K; ++i) {
            Gm[lane * KP + i] = 0.0;
            Gm[i * KP + lane] = 0.0;
          }
        }
        __syncwarp();
        if (lane < K && Ev[lane] > tol) Gm[lane * KP + lane] = -1.0;
        __syncwarp();
        warp_jacobi<K>(Gm, nullptr, lane);
        M = Gm;
      } else {
        warp_jacobi<K>(M, nullptr, lane);
      }
      const unsigned pos = __ballot_sync(0xffffffffu, lane < K && M[(lane < K ? lane : 0) * KP + (lane < K ? lane : 0)] > 0.0);
      const int cnt = below + dimR + __popc(pos) - sub.kplus;
      if (lane == 0) {
        *out = cnt;
        *s_redo = 0;
      }
      __syncwarp();
        }
    group_sync<E>(g);
    if (!p32 || !active || (*s_redo) == 0) break;
  }
  if (CM == 1 && active && e == 0 && lane == 0 && (!try32 || (*s_redo) != 0)) *out = -1;  // recount in FP64
  __syncwarp();
}

template <int K>
__global__ void __launch_bounds__(128) counts_kernel(Sub sub, const double* __restrict__ xs,
                                                     int npts, int* __restrict__ counts, int pt0,
                                                     int pt_end) {
  constexpr int E = warps_per_root(K);
  constexpr int G = 4 / E;
  constexpr int KP = K + 1;
  __shared__ double sM[G][K * KP], sG[G][K * KP], sV[G][K * KP];
  __shared__ double sEv[G][K], s_err[G][2];
  __shared__ int s_redo[G];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = warp / E, e = warp - (warp / E) * E;
  if (input_invalid(sub.st)) return;
  const int n = *sub.n_dev;
  const bool absolute = (xs != nullptr);
  // Pole mode covers the poles [pt0, min(n, pt_end)).
  const int first = absolute ? 0 : pt0;
  const int limit = absolute ? npts : min(n, pt_end);
  // Every group runs the same number of trips so that the named barriers match.
  for (int base = first + blockIdx.x * G; base < limit; base += gridDim.x * G) {
    const int pt = base + g;
    const bool active = pt < limit;
    const double tau = (active && absolute) ? xs[pt] : 0.0;
    const double lam_o = (active && !absolute) ? sub.lam[pt] : 0.0;
    count_point<K>(sub, n, active, absolute, tau, lam_o, pt, active ? counts + pt : nullptr, sM[g],
                   sG[g], sV[g], sEv[g], s_err[g], &s_redo[g], g, e, lane);
  }
}

// Pole counts of every update of a class (items numbered across the class).
// The recount (CM = 2) gives each point up to four warps, each owning a share
// of the k x k accumulators: a recount is one FP64 pass over all n' terms, and
// the launch lasts as long as its slowest recount.
template <int K, int CM>
__global__ void __launch_bounds__(128) counts_grouped_kernel(const ProbDesc* __restrict__ P,
                                                             ClassDesc c) {
  // (warp e owns rows e and K-1-e, so E <= ceil(K/2))
  constexpr int E = (CM == 2) ? (K >= 7 ? 4 : K >= 3 ? 2 : 1) : warps_per_root(K);
  constexpr int G = 4 / E;
  constexpr int KP = K + 1;
  __shared__ double sM[G][K * KP], sG[G][K * KP], sV[G][K * KP];
  __shared__ double sEv[G][K], s_err[G][2];
  __shared__ int s_redo[G];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = warp / E, e = warp - (warp / E) * E;
  const int total = c.pk[c.count];
  for (int base = blockIdx.x * G; base < total; base += gridDim.x * G) {
    const int item = base + g;
    bool active = item < total;
    Sub sub;
    int n = 0, pt = 0;
    int* out = nullptr;
    double lam_o = 0.0;
    if (active) {
      const int p = find_owner(c.pk, c.count, item);
      const ProbDesc& d = P[c.ids[p]];
      sub = sub_of(d);
      if (input_invalid(d.st)) {
        active = false;
      } else {
        n = *sub.n_dev;
        pt = item - c.pk[p];
        lam_o = sub.lam[pt];
        out = d.pole_cnt + pt;
        if (CM == 2 && *out >= 0) active = false;  // certified by the FP32 launch
      }
    }
    count_point<K, CM, E>(sub, n, active, false, 0.0, lam_o, pt, out, sM[g], sG[g], sV[g], sEv[g], s_err[g],
                          &s_redo[g], g, e, lane);
  }
}

// ----------------------------------------------------------------------------
// roots_kernel: persistent; each root group takes root indices m from a
// global counter and runs the safeguarded Newton / bisection to convergence.
//
// Root m lies in the pole interval (lam_a, lam_b) (a = p-1, b = p; a missing
// end is a Weyl sentinel).  The two bracketing terms are kept out of the sums
// and carried exactly in the bordered (K+2) x (K+2) matrix
//     Z(x) = [[Sigma - M^(x), -u_a, -u_b], [-u_a^T, x - lam_a, 0], [-u_b^T, 0, x - lam_b]]
// (M^ = M without terms a, b).  Eliminating the last two rows gives back
// Sigma - M(x), so
//   det Z = (x - lam_a)(x - lam_b) det(Sigma - M(x)) =: p(x), smooth on the interval,
//   pos(Sigma - M) = pos(Z) - pos(diag(x - lam_a, x - lam_b))   (inertia), and
//   Z [c; beta] = 0  <=>  (Sigma - M) c = 0 with beta_i = u_i^T c / (x - lam_i).
// Z has no entry that blows up near a pole, so the count, the Newton step
// p'/p = tr(Z^{-1} Z') with Z' = diag(N^, 1, 1), and the null vector keep their
// accuracy when the root sits next to a pole; eq. (10) then takes
// w_a = -beta_a, w_b = -beta_b directly instead of u^T c / (lam - mu), which
// cancels there.  A missing pole is a decoupled entry 1.
// ----------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void root_solve(const Sub& sub, const int* __restrict__ pole_cnt,
                                           int max_iter, const RootOut& out, DevStatus* st, int n,
                                           int m, double* sMg, double* sNg, double* sZg,
                                           double* sVg, double* sAg, double* sIg, double* s_tau, double* s_lamo,
                                           int* s_done, int* s_ia, int* s_ib, int* s_ph,
                                           double* s_err, int* s_tay, double* s_step, int g, int e,
                                           int lane) {
  constexpr int E = warps_per_root(K);
  constexpr int KP = K + 1;
  constexpr int Z2 = K + 2;
  constexpr int ZP = K + 3;
  const int ld = sub.ld;
  const double* __restrict__ lam = sub.lam;
  const double* __restrict__ Us = sub.Us;
  // ---- placement (warp 0 of the group; every lane holds the same state) ----
  int o = 0, p = 0, c_lo = 0, c_hi = 0, it = 0, it32 = 0, itay = 0, itgj = 0, slow = 0, ia = -1, ib = -1;
  // Coarse phase in FP32 (mixed mode): steps from FP32 sums, the bracket moved
  // only by counts that the error bound certifies; then FP64 to the end.
  bool phase32 = (sub.lamf != nullptr);
  bool has_a = false, has_b = false, first = false, notconv = false;
  double tl = 0.0, th = 0.0, tau = 0.0, da = 0.0, db = 0.0, prev_step = INFINITY;
  bool last_model = false;  // the current point came from a two-pole model step
  bool vvalid = false;      // V holds eigenvectors of an earlier Z (Jacobi warm start)
  if (e == 0) {
    int lo = 0, hi = n;  // p = #{q : pole_cnt[q] <= m}
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (pole_cnt[mid] <= m) lo = mid + 1; else hi = mid;
    }
    p = lo;
    has_a = p > 0;
    has_b = p < n;
    ia = has_a ? p - 1 : -1;
    ib = has_b ? p : -1;
    c_lo = has_a ? pole_cnt[p - 1] : 0;
    c_hi = has_b ? pole_cnt[p] : n;
    if (c_lo > m) c_lo = m;
    if (c_hi <= m) c_hi = m + 1;
    if (has_a && has_b) {
      o = p - 1;
      db = lam[p] - lam[p - 1];
      tl = 0.0;
      th = db;
      tau = 0.5 * db;
      first = true;
    } else if (has_a) {
      o = p - 1;
      tl = 0.0;
      th = sub.st->hi_sent - lam[o];
      tau = 0.5 * th;
    } else {
      o = 0;
      tl = sub.st->lo_sent - lam[0];
      th = 0.0;
      tau = 0.5 * tl;
    }
    if (lane == 0) {
      (*s_tau) = tau;
      (*s_lamo) = lam[o];
      (*s_ia) = ia;
      (*s_ib) = ib;
      (*s_ph) = phase32 ? 1 : 0;
      (*s_tay) = 0;
    }
  }
  group_sync<E>(g);
  const int skip_a = (*s_ia), skip_b = (*s_ib);
  for (;;) {
    const double tau_c = (*s_tau);
    const double lam_o = (*s_lamo);
    const bool ph32 = (*s_ph) != 0;
    // After a small Newton step (|s| <= 1e-8 of the distance to every pole in
    // the sums) the sums move to first order: M^(x+s) = M^(x) - s N^(x), with
    // an error below s^2 tr(N^)/d_min <= 1e-16 of their own scale, and N^ is
    // kept.  No pass over the terms.
    const bool tay = (*s_tay) != 0;
    int below = 0;
    if (tay) {
      if (e == 0) {
        const double sstep = (*s_step);
        for (int idx = lane; idx < K * K; idx += 32) {
          const int r = idx / K, c = idx - (idx / K) * K;
          sMg[r * KP + c] = fma(-sstep, sNg[r * KP + c], sMg[r * KP + c]);
        }
        __syncwarp();
      }
    } else if (ph32) {
      const float ho = (float)lam_o, th32 = (float)tau_c;
      accumulate32_group<K, E, true>(e, sub.lamf, sub.Usf, ld, n, ho, (float)(lam_o - (double)ho), th32,
                               (float)(tau_c - (double)th32), skip_a, skip_b, sMg, sNg, s_err, lane);
    } else if (sub.Pp) {
      if (sub.Usf)
        accumulate_p_group<K, E, ACC_MN32>(e, lam, sub.Pp, ld, n, lam_o, tau_c, skip_a, skip_b, sMg, sNg, lane,
                                           sub.Usf);
      else
        accumulate_p_group<K, E, ACC_MN>(e, lam, sub.Pp, ld, n, lam_o, tau_c, skip_a, skip_b, sMg, sNg, lane,
                                         nullptr);
    } else if (sub.Usf) {
      accumulate_group<K, E, ACC_MN32>(e, lam, Us, ld, n, lam_o, false, tau_c, skip_a, skip_b, sMg, sNg,
                                       lane, sub.Usf);
    } else {
      accumulate_group<K, E, ACC_MN>(e, lam, Us, ld, n, lam_o, false, tau_c, skip_a, skip_b, sMg, sNg,
                                     lane);
    }
    group_sync<E>(g);
    if (e == 0) {
      const double* M = sMg;
      const double* Nm = sNg;
      double* Z = sZg;
      double* V = sVg;
      const double Da = has_a ? tau - da : 1.0;
      const double Db = has_b ? tau - db : 1.0;
      for (int idx = lane; idx < Z2 * Z2; idx += 32) {
        const int r = idx / Z2, c = idx - (idx / Z2) * Z2;
        double v;
        if (r < K && c < K) {
          v = ((r == c) ? sigma_of(sub.negmask, r) : 0.0) - M[r * KP + c];
        } else if (r < K || c < K) {
          const int row = r < K ? r : c;  // component of u
          const int which = r < K ? c : r;  // K -> pole a, K+1 -> pole b
          const int pi = (which == K) ? ia : ib;
          v = (pi >= 0) ? -Us[(size_t)row * ld + pi] : 0.0;
        } else {
          v = (r != c) ? 0.0 : (r == K ? Da : Db);
        }
        Z[r * ZP + c] = v;
      }
      __syncwarp();
      // Eigen-decomposition of Z (parallel Jacobi, warm-started from the last
      // one's eigenvectors when there is one); Z's diagonal then holds the
      // eigenvalues and V the eigenvectors.
      auto diag_Z = [&]() {
        if (vvalid) {
          // Warm start: rotate Z into the previous eigenbasis (nearly diagonal),
          // then let Jacobi finish and accumulate onto V.  T = Z V, then V^T T,
          // each entry by one lane (all 32 lanes busy), T kept in Z's storage.
          constexpr int ZE = Z2 * Z2;
          constexpr int NB = (ZE + 31) / 32;
          double tv[NB];
  #pragma unroll
          for (int b = 0; b < NB; ++b) {
            const int idx = b * 32 + lane;
            double acc = 0.0;
            if (idx < ZE) {
              const int r = idx / Z2, c = idx - (idx / Z2) * Z2;
              for (int q = 0; q < Z2; ++q) acc = fma(Z[r * ZP + q], V[q * ZP + c], acc);
            }
            tv[b] = acc;
          }
          __syncwarp();
  #pragma unroll
          for (int b = 0; b < NB; ++b) {
            const int idx = b * 32 + lane;
            if (idx < ZE) Z[(idx / Z2) * ZP + (idx - (idx / Z2) * Z2)] = tv[b];
          }
          __syncwarp();
  #pragma unroll
          for (int b = 0; b < NB; ++b) {
            const int idx = b * 32 + lane;
            double acc = 0.0;
            if (idx < ZE) {
              const int i = idx / Z2, c = idx - (idx / Z2) * Z2;
              for (int r = 0; r < Z2; ++r) acc = fma(V[r * ZP + i], Z[r * ZP + c], acc);
            }
            tv[b] = acc;
          }
          __syncwarp();
  #pragma unroll
          for (int b = 0; b < NB; ++b) {
            const int idx = b * 32 + lane;
            if (idx < ZE) Z[(idx / Z2) * ZP + (idx - (idx / Z2) * Z2)] = tv[b];
          }
          __syncwarp();
          if (lane < Z2) {  // exact symmetry
            for (int i = lane + 1; i < Z2; ++i) Z[i * ZP + lane] = Z[lane * ZP + i];
          }
          __syncwarp();
          warp_jacobi<Z2>(Z, V, lane, false);
        } else {
          warp_jacobi<Z2>(Z, V, lane, true);
        }
        vvalid = true;
      };
      const int posD = (Da > 0.0 ? 1 : 0) + (Db > 0.0 ? 1 : 0);
      // Inside the bracket #{lam_i < x} is the pole index p.
      below = has_a ? p : 0;
      double tsum = 0.0, g11 = 0.0, g12 = 0.0, g22 = 0.0;
      int count = 0;
      bool redo = false, conv = false;
      // FP32 phase, one root in the bracket (the common case): the count is c_lo or c_hi,
      // and it follows from the sign of det Z alone -- neg(Z) has the parity of
      // [det Z < 0], so count = below + (Z2 - neg(Z)) - posD - k_plus is known
      // mod 2.  Z^{-1} (Gauss-Jordan, no eigen-decomposition) gives the Newton
      // step p'/p = tr(Z^{-1} Z'), Z' = diag(N^, [a], [b]), and the model's
      // G = (Z^{-1})_SS.  FP32 phase: the FP32 sums' error Delta sits in the
      // K x K block (|Delta|_2 <= E); Z + t Delta = Z (I + t Z^{-1} Delta) stays
      // nonsingular for t in [0, 1] when E |(Z^{-1})_KK|_2 < 1, so det Z keeps
      // its sign and the count is certified; with the Gauss-Jordan rounding
      // (64 Z2 eps |Z|_F |Z^{-1}|_F) the test below keeps a factor-2 margin.
      // The FP64 phase keeps the eigen-decomposition at every evaluation: the
      // null vector at the accepted root comes from Z's eigenvectors, and a
      // decomposition warm-started from the previous evaluation's is the one
      // that keeps neighbouring vectors orthogonal to rounding (with stale
      // eigenvectors |w_r^T w_r+1| rose from 4e-14 to 6e-11 on the
      // log-spectrum workload).
      bool gj = false;
      if (ph32 && c_hi - c_lo == 1) {
        int detneg = 0;
        double zf = 0.0, invf = 0.0, invkf = 0.0;
        gj = warp_gj_inverse<Z2>(Z, sAg, sIg, lane, K, &detneg, &zf, &invf, &invkf);
        if (gj) {
          const double* Inv = sIg;
          double q = 0.0;
          for (int idx = lane; idx < K * K; idx += 32) {
            const int r = idx / K, c = idx - (idx / K) * K;
            q = fma(Inv[r * ZP + c], Nm[c * KP + r], q);
          }
          q = warp_sum(q);
          g11 = Inv[K * ZP + K];
          g12 = Inv[K * ZP + K + 1];
          g22 = Inv[(K + 1) * ZP + K + 1];
          tsum = q + (has_a ? g11 : 0.0) + (has_b ? g22 : 0.0);
          const int par = (below + Z2 - detneg - posD - sub.kplus) & 1;
          count = ((c_lo & 1) == par) ? c_lo : c_hi;
          if (ph32) {
            const double L = (double)((n + 31) / 32);
            const double Es = 1.25 * ((L + 16.0) * 0x1p-24 * s_err[0] + 0x1p-46 * sub.st->lam_absmax * s_err[1]);
            redo = !(Es * invkf + 64.0 * Z2 * kEps * zf * invf < 0.5) || !isfinite(tsum);
          }
        }
      }
      if (!gj) {
        diag_Z();
        // p'/p = sum_j z_j^T Z' z_j / zeta_j,  Z' = diag(N^, [a real], [b real]);
        // G = (Z^{-1})_{SS} for the two-pole model below.
        double zj = 0.0, contrib = 0.0;
        if (lane < Z2) {
          zj = Z[lane * ZP + lane];
          double q = 0.0;
          for (int a = 0; a < K; ++a) {
            double na = 0.0;
            for (int b = 0; b < K; ++b) na = fma(Nm[a * KP + b], V[b * ZP + lane], na);
            q = fma(V[a * ZP + lane], na, q);
          }
          const double za = V[K * ZP + lane], zb = V[(K + 1) * ZP + lane];
          if (has_a) q = fma(za, za, q);
          if (has_b) q = fma(zb, zb, q);
          const double rz = 1.0 / zj;
          contrib = q * rz;
          g11 = za * za * rz;
          g12 = za * zb * rz;
          g22 = zb * zb * rz;
        }
        const unsigned posmask = __ballot_sync(0xffffffffu, lane < Z2 && zj > 0.0);
        tsum = warp_sum(contrib);
        g11 = warp_sum(g11);
        g12 = warp_sum(g12);
        g22 = warp_sum(g22);
        count = below + __popc(posmask) - posD - sub.kplus;
        // FP32 phase: the count is exact when no eigenvalue of Z can change sign
        // under the error of the FP32 sums, which only enters the K x K block:
        //   E = |dM^|_2 <= (L + 16) 2^-24 S1 + 2^-46 max|lam| S2   (L terms per lane,
        //   three roundings per term, five in the warp's FP32 butterfly, slack),
        // plus the Jacobi's own rounding.  Eigenvalues with |z_j| > 2E keep their
        // sign (Weyl).  The small ones belong to eigenvectors that live almost
        // entirely in the two bordered rows; with s the small set, W = |V_{K,s}|_F^2
        // (their weight in the K block) and g the distance of the large ones from
        // zero, each small eigenvalue moves by at most E W + E^2 W / g (a
        // Hermitian block perturbation with the large block eliminated).  If any
        // sign is not certain this point is evaluated again in FP64 and the FP64
        // phase takes over.
        if (ph32) {
          const bool nonfin = __any_sync(0xffffffffu, lane < Z2 && !isfinite(zj));
          double zmax = (lane < Z2) ? fabs(zj) : 0.0;
  #pragma unroll
          for (int off = 16; off > 0; off >>= 1) zmax = fmax(zmax, __shfl_xor_sync(0xffffffffu, zmax, off));
          const double L = (double)((n + 31) / 32);
          const double E = 1.25 * ((L + 16.0) * 0x1p-24 * s_err[0] + 0x1p-46 * sub.st->lam_absmax * s_err[1]) +
                           64.0 * kEps * zmax;
          const bool small = lane < Z2 && !(fabs(zj) > 2.0 * E);
          double wk = 0.0;
          if (small) {
            for (int c = 0; c < K; ++c) wk = fma(V[c * ZP + lane], V[c * ZP + lane], wk);
          }
          double zs = small ? fabs(zj) : INFINITY;
          double zb = (lane < Z2 && !small) ? fabs(zj) : INFINITY;
  #pragma unroll
          for (int off = 16; off > 0; off >>= 1) {
            wk += __shfl_xor_sync(0xffffffffu, wk, off);
            zs = fmin(zs, __shfl_xor_sync(0xffffffffu, zs, off));
            zb = fmin(zb, __shfl_xor_sync(0xffffffffu, zb, off));
          }
          const double g = zb - E;
          const double shift = E * wk + E * E * wk / g;
          const bool any_small = zs < INFINITY;
          redo = nonfin || !(E < INFINITY) ||
                 (any_small && !(g > 0.0 && zs > 2.0 * shift + 64.0 * kEps * zmax));
        }
      }
      if (redo) {
        // The count is uncertain but the FP32 Newton step is still good: with
        // one root in the bracket and the step inside it, the FP64 phase
        // starts at the stepped point (the bracket is left as it was).
        phase32 = false;
        prev_step = INFINITY;
        slow = 0;
        last_model = false;
        if (lane == 0) atomicAdd((unsigned long long*)&st->redo32_total, 1ull);
        const double tn0 = tau - 1.0 / tsum;
        if (c_hi - c_lo == 1 && isfinite(tn0) && tn0 > tl && tn0 < th) {
          tau = tn0;
          ++it;
          ++it32;
        }
      } else {
      ++it;
      if (ph32) ++it32;
      if (tay) ++itay;
      if (gj) ++itgj;
      const double wprev = th - tl;
      if (count <= m) {
        tl = tau;
        c_lo = count;
      } else {
        th = tau;
        c_hi = count;
      }
      // A model step that did not halve the bracket is not trusted again (it
      // can keep aiming at a neighbouring root): bisect instead.
      const bool stalled = last_model && (th - tl) > 0.5 * wprev;
      if (first) {
        first = false;
        if (count <= m) {  // root above the midpoint: measure it from pole b
          const double sh = -db;
          tl += sh;
          th = 0.0;
          tau += sh;
          da = sh;
          db = 0.0;
          o = p;
        }
      }
      // Two-pole model: freeze B^ (Sigma - M without the bracketing terms); then
      // det Z = 0 becomes det(diag(x - lam_a, x - lam_b) - C) = 0 with
      // C = U_S^T B^{-1} U_S = D_S - G^{-1}: the roots are the eigenvalues of
      // diag(lam_a, lam_b) + C, exact in both poles.
      double cand0 = NAN, cand1 = NAN;  // model roots inside the bracket, ascending
      int ncand = 0;
      {
        const double det = g11 * g22 - g12 * g12;
        if (isfinite(det) && det != 0.0) {
          const double c11 = Da - g22 / det, c22 = Db - g11 / det, c12 = g12 / det;
          if (has_a && has_b) {
            const double t11 = da + c11, t22 = db + c22;
            const double mid2 = 0.5 * (t11 + t22), hd = 0.5 * (t11 - t22);
            const double rad = sqrt(hd * hd + c12 * c12);
            const double lo2 = mid2 - rad, hi2 = mid2 + rad;
            if (lo2 > tl && lo2 < th) {
              cand0 = lo2;
              ncand = 1;
            }
            if (hi2 > tl && hi2 < th && hi2 != lo2) {
              if (ncand == 0) cand0 = hi2; else cand1 = hi2;
              ++ncand;
            }
          } else {
            const double t1 = has_a ? da + c11 : db + c22;
            if (t1 > tl && t1 < th) {
              cand0 = t1;
              ncand = 1;
            }
          }
        }
      }
      bool newton = false;
      double tn = tau;
      const int inb = c_hi - c_lo;  // roots in the bracket
      const int r_in = m - c_lo;    // our root's rank among them
      double model = NAN;
      if (ncand > 0 && !stalled) {
        if (inb == ncand) model = (r_in >= 1 && ncand == 2) ? cand1 : cand0;
        else if (inb == 1) model = cand0;
      }
      if (inb == 1) {
        const double step = -1.0 / tsum;
        tn = tau + step;
        // A step below half an ulp of tau leaves tau where it is.  tau is the
        // bracket end the count just moved; if the step points into the bracket
        // the root is within rounding of tau (an outward step means another
        // root sits just outside: keep bisecting).
        if (step == 0.0 || (tn == tau && ((tau == tl && step > 0.0) || (tau == th && step < 0.0)))) {
          conv = true;
          tn = tau;
        } else if (it <= 2 && isfinite(model)) {
          tn = model;  // early steps: the model captures both poles globally
        } else if (isfinite(tn) && tn > tl && tn < th) {
          newton = true;
          if (fabs(step) <= 2.0 * kEps * fabs(tn)) conv = true;
          // Quadratic regime confirmed (step far below the previous one): the
          // next error is ~ step^2, below rounding, so accept without
          // another evaluation.
          if (fabs(step) <= 1e-10 * fabs(tn) && fabs(step) <= 1e-2 * fabs(prev_step)) conv = true;
          if (fabs(step) > 0.5 * fabs(prev_step)) ++slow; else slow = 0;
          prev_step = step;
          if (slow >= 3 && !conv) {
            newton = false;
            slow = 0;
            tn = NAN;  // fall through to bisection
          }
        } else if (isfinite(model)) {
          tn = model;
        } else {
          tn = NAN;
        }
      } else {
        tn = isfinite(model) ? model : NAN;
      }
      last_model = !newton && !conv && isfinite(model) && tn == model;
      if (!conv && !newton && !(tn > tl && tn < th)) {
        tn = tl + 0.5 * (th - tl);
        if (tl > 0.0 && th > 64.0 * tl) tn = sqrt(tl) * sqrt(th);
        else if (th < 0.0 && tl < 64.0 * th) tn = -(sqrt(-tl) * sqrt(-th));
        if (!(tn > tl && tn < th)) {
          conv = true;
          tn = tl + 0.5 * (th - tl);
        }
        prev_step = INFINITY;
      }
      if (!conv && (th - tl) <= 4.0 * kEps * fmax(fabs(tl), fabs(th))) conv = true;
      if (!conv && it >= max_iter) {
        conv = true;
        notconv = true;
      }
      if (ph32) {
        // A root is never finished on FP32 sums; near FP32 resolution (a small
        // Newton step or bracket) the FP64 phase takes over at the next point.
        if (conv) {
          conv = false;
          notconv = false;
          phase32 = false;
        } else if ((newton && fabs(tn - tau) <= 1e-5 * fabs(tn)) || it32 >= 16 ||
                   (th - tl) <= 1e-5 * fmax(fabs(tl), fabs(th))) {
          phase32 = false;
        }
        if (!phase32) {
          prev_step = INFINITY;
          slow = 0;
          last_model = false;
        }
      }
      const double delta = tn - tau;  // the accepted point minus the evaluated one
      // Next evaluation by the first-order update when the Newton step is tiny
      // against the nearest pole inside the sums (the neighbours of the bracket).
      bool tay_next = false;
      if (!ph32 && !phase32 && newton && !conv) {
        double dmin = INFINITY;
        const int lo_nb = (ia >= 1) ? ia - 1 : -1;
        const int hi_nb = (ib >= 0 && ib + 1 < n) ? ib + 1 : -1;
        if (lo_nb >= 0) dmin = fmin(dmin, fabs(tau - (lam[lo_nb] - lam[o])));
        if (hi_nb >= 0) dmin = fmin(dmin, fabs(tau - (lam[hi_nb] - lam[o])));
        tay_next = fabs(delta) <= 1e-8 * dmin;
      }
      tau = tn;
      if (conv) {
        // The null vector comes from Z's eigenpairs at the evaluated point.
        if (gj) diag_Z();
        // [alpha_0; beta]: eigenvector of Z for the eigenvalue nearest zero.
        int jmin = 0;
        double amin = fabs(Z[0]);
        for (int j = 1; j < Z2; ++j) {
          const double v = fabs(Z[j * ZP + j]);
          if (v < amin) {
            amin = v;
            jmin = j;
          }
        }
        // Z was diagonalised at the evaluated point; the root is delta away
        // (an accepted Newton step or a bisection midpoint).  Move the null
        // vector there to first order: v += delta sum_j (v_j^T Z' v)/(z_min - z_j) v_j
        // with Z' = diag(N^, 1, 1).  A term that is not small (a nearly
        // repeated zero eigenvalue) is left out.
        double comp = (lane < Z2) ? V[lane * ZP + jmin] : 0.0;
        if (delta != 0.0) {
          double gam = 0.0;
          if (lane < Z2 && lane != jmin) {
            double q = 0.0;
            for (int a = 0; a < K; ++a) {
              double na = 0.0;
              for (int b = 0; b < K; ++b) na = fma(Nm[a * KP + b], V[b * ZP + jmin], na);
              q = fma(V[a * ZP + lane], na, q);
            }
            if (has_a) q = fma(V[K * ZP + lane], V[K * ZP + jmin], q);
            if (has_b) q = fma(V[(K + 1) * ZP + lane], V[(K + 1) * ZP + jmin], q);
            gam = delta * q / (Z[jmin * ZP + jmin] - Z[lane * ZP + lane]);
            if (!(fabs(gam) <= 1e-3)) gam = 0.0;
          }
          double acc = comp;
          for (int j = 0; j < Z2; ++j) {
            const double gj = __shfl_sync(0xffffffffu, gam, j);
            if (lane < Z2) acc = fma(gj, V[lane * ZP + j], acc);
          }
          comp = acc;
        }
        const double beta_a = __shfl_sync(0xffffffffu, comp, K);
        const double beta_b = __shfl_sync(0xffffffffu, comp, K + 1);
        if (lane < K) out.alpha[(size_t)m * K + lane] = comp;
        if (lane == 0) {
          out.beta[2 * (size_t)m] = beta_a;
          out.beta[2 * (size_t)m + 1] = beta_b;
          out.sidx[2 * (size_t)m] = ia;
          out.sidx[2 * (size_t)m + 1] = ib;
          out.origin[m] = o;
          out.tau[m] = tau;
          out.iters[m] = it;
          out.flags[m] = notconv ? 1 : 0;
          atomicAdd((unsigned long long*)&st->iters_total, (unsigned long long)(it - it32 - itay));
          if (itay) atomicAdd((unsigned long long*)&st->taylor_total, (unsigned long long)itay);
          if (it32) atomicAdd((unsigned long long*)&st->iters32_total, (unsigned long long)it32);
          if (itgj) atomicAdd((unsigned long long*)&st->gj32_total, (unsigned long long)itgj);
          atomicMax(&st->iters_max, it);
          if (notconv) {
            atomicAdd((unsigned long long*)&st->n_notconv, 1ull);
            atomicOr(&st->flags, (int)ST_NOTCONV);
          }
        }
      }
        if (lane == 0) {
          (*s_tay) = tay_next ? 1 : 0;
          (*s_step) = delta;
        }
      }  // !redo
      if (lane == 0) {
        (*s_tau) = tau;
        (*s_lamo) = lam[o];
        (*s_done) = conv ? 1 : 0;
        (*s_ph) = phase32 ? 1 : 0;
        if (redo) (*s_tay) = 0;
      }
    }
    group_sync<E>(g);
    if ((*s_done)) break;
  }
}

template <int K>
__global__ void __launch_bounds__(128) roots_kernel(Sub sub, const int* __restrict__ pole_cnt,
                                                    int max_iter, int* counter, RootOut out,
                                                    DevStatus* st, int m_end) {
  constexpr int E = warps_per_root(K);
  constexpr int G = 4 / E;
  constexpr int KP = K + 1;
  constexpr int Z2 = K + 2;
  constexpr int ZP = K + 3;
  __shared__ double sM[G][K * KP], sN[G][K * KP], sZ[G][Z2 * ZP], sV[G][Z2 * ZP], sA[G][Z2 * ZP],
      sI[G][Z2 * ZP];
  __shared__ double s_tau[G], s_lamo[G];
  __shared__ int s_m[G], s_done[G], s_ia[G], s_ib[G], s_ph[G], s_tay[G];
  __shared__ double s_err[G][2], s_step[G];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = warp / E, e = warp - (warp / E) * E;
  if (input_invalid(sub.st)) return;
  const int n = *sub.n_dev;
  const int stop = min(n, m_end);  // roots [*counter at launch, stop)
  for (;;) {
    if (e == 0 && lane == 0) s_m[g] = atomicAdd(counter, 1);
    group_sync<E>(g);
    const int m = s_m[g];
    if (m >= stop) break;
    root_solve<K>(sub, pole_cnt, max_iter, out, st, n, m, sM[g], sN[g], sZ[g], sV[g], sA[g], sI[g], &s_tau[g],
                  &s_lamo[g], &s_done[g], &s_ia[g], &s_ib[g], &s_ph[g], s_err[g], &s_tay[g], &s_step[g], g, e, lane);
  }
}

// Zero finder for every root of a class (items numbered across the class).
template <int K>
__global__ void __launch_bounds__(128) roots_grouped_kernel(const ProbDesc* __restrict__ P,
                                                            ClassDesc c, int max_iter) {
  constexpr int E = warps_per_root(K);
  constexpr int G = 4 / E;
  constexpr int KP = K + 1;
  constexpr int Z2 = K + 2;
  constexpr int ZP = K + 3;
  __shared__ double sM[G][K * KP], sN[G][K * KP], sZ[G][Z2 * ZP], sV[G][Z2 * ZP], sA[G][Z2 * ZP],
      sI[G][Z2 * ZP];
  __shared__ double s_tau[G], s_lamo[G];
  __shared__ int s_m[G], s_done[G], s_ia[G], s_ib[G], s_ph[G], s_tay[G];
  __shared__ double s_err[G][2], s_step[G];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = warp / E, e = warp - (warp / E) * E;
  const int total = c.pk[c.count];
  for (;;) {
    if (e == 0 && lane == 0) {
      const int slot = atomicAdd(c.counter, 1);
      s_m[g] = (slot < total && c.perm) ? c.perm[slot] : slot;
    }
    group_sync<E>(g);
    const int item = s_m[g];
    if (item >= total) break;
    const int p = find_owner(c.pk, c.count, item);
    const ProbDesc& d = P[c.ids[p]];
    if (input_invalid(d.st)) continue;  // uniform across the group
    const Sub sub = sub_of(d);
    root_solve<K>(sub, d.pole_cnt, max_iter, rootout_of(d), d.st, *sub.n_dev, item - c.pk[p],
                  sM[g], sN[g], sZ[g], sV[g], sA[g], sI[g], &s_tau[g], &s_lamo[g], &s_done[g], &s_ia[g],
                  &s_ib[g], &s_ph[g], s_err[g], &s_tay[g], &s_step[g], g, e, lane);
  }
}

// ----------------------------------------------------------------------------
// Assembly: mu of each secular root, output positions, eq. (10) columns.
// ----------------------------------------------------------------------------
__device__ __forceinline__ int lower_bound_d(const double* a, int n, double v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ int upper_bound_d(const double* a, int n, double v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] <= v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void mu_kernel(Sub sub, RootOut roots, double* __restrict__ mu_sec) {
  if (input_invalid(sub.st)) return;
  const int n = *sub.n_dev;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x)
    mu_sec[m] = sub.lam[roots.origin[m]] + roots.tau[m];
}

// Deflated pairs keep lam_i and the old eigenvector: W column = e_i.
__global__ void deflated_kernel(Sub sub, int64_t n, const int* __restrict__ idx_defl,
                                const double* __restrict__ lam_defl, const DevStatus* st,
                                const double* __restrict__ mu_sec, double* __restrict__ lam_out,
                                double* __restrict__ W, WSlices ws) {
  if (input_invalid(st)) return;
  const int nk = *sub.n_dev;
  const int nd = st->n_defl;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nd; j += gridDim.x * blockDim.x) {
    const double v = lam_defl[j];
    const int64_t pos = j + upper_bound_d(mu_sec, nk, v);
    lam_out[pos] = v;
    if (W) W[(int64_t)idx_defl[j] + pos * n] = 1.0;
    if (ws.Ws) {  // e_i: 1 = 2^(f-8) * 64 with f = 2
      ws.Ws[(size_t)pos * ws.lds + idx_defl[j]] = __double2bfloat16(64.0);
      ws.fcol[pos] = 2;
    }
  }
}

constexpr int kAsmThreads = 256;
constexpr int kAsmCache = 32;
// Dynamic shared memory of the assembly kernels: one column's entries (n' <=
// kAsmThreads * kAsmCache), kept between the norm pass and the writing pass
// (in shared memory, not registers, so that several CTAs share an SM).
constexpr size_t kAsmSmem = sizeof(double) * kAsmThreads * kAsmCache;
// Once per kernel and device (the attribute outlives the launch).
template <typename Kern>
cudaError_t allow_asm_smem(Kern* k) {
  static unsigned long long done = 0ull;  // bit d: set on device d
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (__atomic_load_n(&done, __ATOMIC_ACQUIRE) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAsmSmem);
  if (e == cudaSuccess) __atomic_fetch_or(&done, bit, __ATOMIC_RELEASE);
  return e;
}

// Sum over the CTA of one value per thread (every thread gets the sum); sh
// holds kAsmThreads / 32 doubles and may be reused right after.
__device__ __forceinline__ double block_sum_asm(double v, double* sh) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double a = 0.0;
#pragma unroll
  for (int w = 0; w < kAsmThreads / 32; ++w) a += sh[w];
  return a;
}

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  if (v >= 0.0) atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// One CTA per secular root m: w_i = (u_i^T alpha) / (lam_i - mu), |w| = 1, the
// entry of largest magnitude made positive, scattered to W[idx_i, pos].
// One eq. (10) column: every thread of the CTA takes part (block reductions).
template <int K>
__device__ __forceinline__ void assemble_root(const Sub& sub, const RootOut& roots, int64_t n,
                                              const double* __restrict__ lam_defl, int nd, int nk,
                                              const double* __restrict__ mu_sec,
                                              double* __restrict__ lam_out, double* __restrict__ W,
                                              const WSlices& ws, int m, double* s_n2, double* s_mx,
                                              int* s_ix, double* s_w, int64_t pos_shift = 0,
                                              double* errs = nullptr, DevStatus* stw = nullptr) {
  const int t = threadIdx.x;
  const double mu = mu_sec[m];
  const int64_t pos = m + lower_bound_d(lam_defl, nd, mu) - pos_shift;
  if (t == 0) lam_out[pos] = mu;
  if (!W && !ws.Ws) return;
  const int o = roots.origin[m];
  const double tau = roots.tau[m];
  const double lam_o = sub.lam[o];
  const int ia = roots.sidx[2 * (size_t)m], ib = roots.sidx[2 * (size_t)m + 1];
  const double wa = -roots.beta[2 * (size_t)m], wb = -roots.beta[2 * (size_t)m + 1];
  double al[K];
#pragma unroll
  for (int c = 0; c < K; ++c) al[c] = roots.alpha[(size_t)m * K + c];
  // eq. (10): w_i = u_i^T alpha / (lam_i - mu); the bracketing poles take -beta.
  auto wcomp = [&](int i) -> double {
    if (i == ia) return wa;
    if (i == ib) return wb;
    double ua = 0.0;
#pragma unroll
    for (int c = 0; c < K; ++c) ua = fma(sub.Us[(size_t)c * sub.ld + i], al[c], ua);
    return ua * rcp_nr((sub.lam[i] - lam_o) - tau);
  };
  // Up to kAsmCache entries per thread are kept in registers for the writing
  // pass (n' <= kAsmThreads * kAsmCache); larger columns are recomputed.
  const bool cached = nk <= kAsmThreads * kAsmCache;
  if (!W && ws.Ws != nullptr && sub.Ulo != nullptr && errs == nullptr && cached) {
    // Mixed mode: the eq. (10) entries in double-float arithmetic.  W feeds a
    // split that keeps 2^-40 of each column's largest entry, so a few units of
    // 2^-48 per entry suffice; only d_i = (lam_i - lam_o) - tau is formed in
    // FP64 (next to the root its two terms cancel).  alpha is scaled by a
    // power of 2, which the normalisation cancels.  A column whose values
    // leave the FP32 range takes the FP64 path below.
    double amax = 0.0;
#pragma unroll
    for (int c = 0; c < K; ++c) amax = fmax(amax, fabs(al[c]));
    const double fro2 = sub.st->fro2;
    if (amax > 0x1p-100 && amax < 0x1p100 && fro2 > 0x1p-100 && fro2 < 0x1p100) {  // uniform
      int ea;
      frexp(amax, &ea);
      const double sa = ldexp(1.0, -ea);
      DF a[K];
#pragma unroll
      for (int c = 0; c < K; ++c) df_bits(al[c] * sa, a[c]);  // |.| < 1; below 2^-60 flushes to 0
      DF wa_d, wb_d;
      bool good = df_bits(wa * sa, wa_d) && df_bits(wb * sa, wb_d);
      float2* const wd = reinterpret_cast<float2*>(s_w);  // this thread's entries only
      float n2h = 0.0f, n2l = 0.0f;
      DF mxd = DF{-1.0f, 0.0f};
      int ixd = 0x7fffffff;
#pragma unroll
      for (int c = 0; c < kAsmCache; ++c) {
        const int i = t + c * kAsmThreads;
        DF w = DF{0.0f, 0.0f};
        if (i < nk) {
          if (i == ia) {
            w = wa_d;
          } else if (i == ib) {
            w = wb_d;
          } else {
            // u_i^T alpha: exact FP32 products, two-sum accumulation
            float sh = 0.0f, sl = 0.0f;
#pragma unroll
            for (int cc = 0; cc < K; ++cc) {
              const float uh = __ldg(sub.Usf + (size_t)cc * sub.ld + i);
              const float ul = __ldg(sub.Ulo + (size_t)cc * sub.ld + i);
              const float pr = uh * a[cc].h;
              float e = fmaf(uh, a[cc].h, -pr);
              e = fmaf(uh, a[cc].l, e);
              e = fmaf(ul, a[cc].h, e);
              const DF sm = df_two_sum(sh, pr);
              sh = sm.h;
              sl += sm.l + e;
            }
            DF d;
            good = df_bits((sub.lam[i] - lam_o) - tau, d) && d.h != 0.0f && good;
            w = df_mul(df_two_sum(sh, sl), df_rcp(d));
          }
          good = good && fabsf(w.h) <= 0x1p100f;  // false for NaN
          const float pr = w.h * w.h;
          const float e = fmaf(2.0f * w.h, w.l, fmaf(w.h, w.h, -pr));
          const DF sm = df_two_sum(n2h, pr);
          n2h = sm.h;
          n2l += sm.l + e;
          // largest |w| (the first index on ties), compared as pairs
          const float mh = fabsf(w.h), ml = w.h < 0.0f ? -w.l : w.l;
          if (mh > mxd.h || (mh == mxd.h && ml > mxd.l)) {
            mxd = DF{mh, ml};
            ixd = i;
          }
          wd[i] = make_float2(w.h, w.l);
        }
      }
      if (!__syncthreads_or(!good)) {
        s_n2[t] = d_of_bits(n2h) + d_of_bits(n2l);
        s_mx[t] = d_of_bits(mxd.h) + d_of_bits(mxd.l);
        s_ix[t] = ixd;
        __syncthreads();
        for (int s = kAsmThreads / 2; s > 0; s >>= 1) {
          if (t < s) {
            s_n2[t] += s_n2[t + s];
            const double om = s_mx[t + s];
            const int oi = s_ix[t + s];
            if (om > s_mx[t] || (om == s_mx[t] && oi < s_ix[t])) {
              s_mx[t] = om;
              s_ix[t] = oi;
            }
          }
          __syncthreads();
        }
        const double nrm = sqrt(s_n2[0]);
        const int imax = (s_ix[0] >= 0 && s_ix[0] < nk) ? s_ix[0] : 0;
        __syncthreads();
        // sign and exponent from the FP64 value of the largest entry, formed once
        if (t == 0) s_mx[0] = wcomp(imax) * sa;
        __syncthreads();
        const double wmax = s_mx[0];
        const double scale = (wmax < 0.0 ? -1.0 : 1.0) / nrm;
        const int f = tc_scale_exp(fabs(wmax * scale));
        DF sd;
        if (df_bits(ldexp(scale, 40 - f), sd) && sd.h != 0.0f) {  // uniform
          if (t == 0) ws.fcol[pos] = f;
          __nv_bfloat16* col = ws.Ws + (size_t)pos * ws.lds;
#pragma unroll
          for (int c = 0; c < kAsmCache; ++c) {
            const int i = t + c * kAsmThreads;
            if (i < nk) {
              __nv_bfloat16 dg[kTcSlices];
              const float2 wv = wd[i];
              tc_split_df(df_mul(DF{wv.x, wv.y}, sd), dg);
              const int j = sub.idx[i];
#pragma unroll
              for (int q = 0; q < kTcSlices; ++q) col[(size_t)q * ws.plane + j] = dg[q];
            }
          }
          return;
        }
      }
      __syncthreads();  // the reduction arrays are reused by the FP64 path
    }
  }
  if (!W && stw && t == 0) atomicAdd(reinterpret_cast<unsigned long long*>(&stw->asm_fp64_cols), 1ull);
  double n2 = 0.0, mx = -1.0;
  int ix = 0x7fffffff;
  if (cached) {
#pragma unroll
    for (int c = 0; c < kAsmCache; ++c) {
      const int i = t + c * kAsmThreads;
      const double w = (i < nk) ? wcomp(i) : 0.0;
      if (i < nk) s_w[i] = w;
      n2 = fma(w, w, n2);
      if (i < nk && fabs(w) > mx) {
        mx = fabs(w);
        ix = i;
      }
    }
  } else {
    for (int i = t; i < nk; i += kAsmThreads) {
      const double w = wcomp(i);
      n2 = fma(w, w, n2);
      if (fabs(w) > mx) {
        mx = fabs(w);
        ix = i;
      }
    }
  }
  s_n2[t] = n2;
  s_mx[t] = mx;
  s_ix[t] = ix;
  __syncthreads();
  for (int s = kAsmThreads / 2; s > 0; s >>= 1) {
    if (t < s) {
      s_n2[t] += s_n2[t + s];
      const double om = s_mx[t + s];
      const int oi = s_ix[t + s];
      if (om > s_mx[t] || (om == s_mx[t] && oi < s_ix[t])) {
        s_mx[t] = om;
        s_ix[t] = oi;
      }
    }
    __syncthreads();
  }
  const double nrm = sqrt(s_n2[0]);
  const int imax = (s_ix[0] >= 0 && s_ix[0] < nk) ? s_ix[0] : 0;  // all-NaN column: any row
  __syncthreads();
  const double wmax = wcomp(imax);
  const double scale = (wmax < 0.0 ? -1.0 : 1.0) / nrm;
  if (errs) {
    // Per-eigenpair report in FP64 on the unit vector w = scale * (eq. (10)
    // entries), in the old eigenbasis, where A' is Lambda + U Sigma U^T:
    //   r = (A' - mu) w,  r_i = (lam_i - mu) w_i + u_i^T Sigma s,  s = U^T w,
    // |r| (metric (B) per pair) and w^T r = rho - mu (Rayleigh quotient).
    // Deflated rows are outside the sub-problem (their u_i are below the
    // deflation bound and add at most that much).
    auto for_entries = [&](auto&& f) {
      if (cached) {
#pragma unroll
        for (int c = 0; c < kAsmCache; ++c) {
          const int i = t + c * kAsmThreads;
          if (i < nk) f(i, s_w[i] * scale);
        }
      } else {
        for (int i = t; i < nk; i += kAsmThreads) f(i, wcomp(i) * scale);
      }
    };
    double sp[K];
#pragma unroll
    for (int c = 0; c < K; ++c) sp[c] = 0.0;
    for_entries([&](int i, double w) {
#pragma unroll
      for (int c = 0; c < K; ++c) sp[c] = fma(sub.Us[(size_t)c * sub.ld + i], w, sp[c]);
    });
    double sv[K];
#pragma unroll
    for (int c = 0; c < K; ++c) sv[c] = sigma_of(sub.negmask, c) * block_sum_asm(sp[c], s_mx);
    double r2 = 0.0, rw = 0.0;
    for_entries([&](int i, double w) {
      double r = ((sub.lam[i] - lam_o) - tau) * w;
#pragma unroll
      for (int c = 0; c < K; ++c) r = fma(sub.Us[(size_t)c * sub.ld + i], sv[c], r);
      r2 = fma(r, r, r2);
      rw = fma(r, w, rw);
    });
    r2 = block_sum_asm(r2, s_mx);
    rw = block_sum_asm(rw, s_mx);
    const double normA = sub.st->lam_absmax + sub.st->fro2;
    // Orthogonality against the next root's vector where the two are close.
    double dn = 0.0;
    if (m + 1 < nk && mu_sec[m + 1] - mu <= 1e-6 * normA) {
      const int m2 = m + 1;
      const int o2 = roots.origin[m2];
      const double tau2 = roots.tau[m2], lo2 = sub.lam[o2];
      const int ia2 = roots.sidx[2 * (size_t)m2], ib2 = roots.sidx[2 * (size_t)m2 + 1];
      const double wa2 = -roots.beta[2 * (size_t)m2], wb2 = -roots.beta[2 * (size_t)m2 + 1];
      double al2[K];
#pragma unroll
      for (int c = 0; c < K; ++c) al2[c] = roots.alpha[(size_t)m2 * K + c];
      double dd = 0.0, nn = 0.0;
      for_entries([&](int i, double w) {
        double v;
        if (i == ia2) {
          v = wa2;
        } else if (i == ib2) {
          v = wb2;
        } else {
          double ua = 0.0;
#pragma unroll
          for (int c = 0; c < K; ++c) ua = fma(sub.Us[(size_t)c * sub.ld + i], al2[c], ua);
          v = ua / ((sub.lam[i] - lo2) - tau2);
        }
        dd = fma(w, v, dd);
        nn = fma(v, v, nn);
      });
      dd = block_sum_asm(dd, s_mx);
      nn = block_sum_asm(nn, s_mx);
      dn = fabs(dd) / sqrt(nn);
    }
    if (t == 0) {
      const double e0 = sqrt(r2) / normA, e1 = fabs(rw) / normA;
      errs[pos] = e0;
      errs[pos + n] = e1;
      errs[pos + 3 * n] = dn;
      if (stw) {
        atomic_max_nonneg(&stw->err_max[0], e0);
        atomic_max_nonneg(&stw->err_max[1], e1);
        atomic_max_nonneg(&stw->err_max[2], dn);
      }
    }
    __syncthreads();
  }
  if (W) {
    double* col = W + pos * n;
    if (cached) {
#pragma unroll
      for (int c = 0; c < kAsmCache; ++c) {
        const int i = t + c * kAsmThreads;
        if (i < nk) col[sub.idx[i]] = s_w[i] * scale;
      }
    } else {
      for (int i = t; i < nk; i += kAsmThreads) col[sub.idx[i]] = wcomp(i) * scale;
    }
  } else {
    // Mixed mode: the column goes straight into its BF16 digit slices.
    const int f = tc_scale_exp(fabs(wmax * scale));
    if (t == 0) ws.fcol[pos] = f;
    __nv_bfloat16* col = ws.Ws + (size_t)pos * ws.lds;
    const double s2 = ldexp(scale, 40 - f);  // exact: scale * 2^(40-f), the split's prescale
    if (cached) {
#pragma unroll
      for (int c = 0; c < kAsmCache; ++c) {
        const int i = t + c * kAsmThreads;
        if (i < nk) {
          __nv_bfloat16 d[kTcSlices];
          tc_split_prescaled(s_w[i], s2, d);
          const int j = sub.idx[i];
#pragma unroll
          for (int q = 0; q < kTcSlices; ++q) col[(size_t)q * ws.plane + j] = d[q];
        }
      }
    } else {
      for (int i = t; i < nk; i += kAsmThreads) {
        __nv_bfloat16 d[kTcSlices];
        tc_split_prescaled(wcomp(i), s2, d);
        const int j = sub.idx[i];
#pragma unroll
        for (int q = 0; q < kTcSlices; ++q) col[(size_t)q * ws.plane + j] = d[q];
      }
    }
  }
}

template <int K>
__global__ void __launch_bounds__(kAsmThreads) assemble_kernel(
    Sub sub, RootOut roots, int64_t n, const double* __restrict__ lam_defl, const DevStatus* st,
    const double* __restrict__ mu_sec, double* __restrict__ lam_out, double* __restrict__ W,
    WSlices ws) {
  __shared__ double s_n2[kAsmThreads];
  __shared__ double s_mx[kAsmThreads];
  __shared__ int s_ix[kAsmThreads];
  extern __shared__ __align__(16) double s_w[];
  if (input_invalid(st)) return;
  const int nk = *sub.n_dev;
  const int nd = st->n_defl;
  for (int m = blockIdx.x; m < nk; m += gridDim.x) {
    assemble_root<K>(sub, roots, n, lam_defl, nd, nk, mu_sec, lam_out, W, ws, m, s_n2, s_mx, s_ix, s_w);
    __syncthreads();
  }
}

// ---- grouped assembly over a class --------------------------------------------
__global__ void mu_grouped_kernel(const ProbDesc* __restrict__ P, ClassDesc c) {
  const int total = c.pk[c.count];
  for (int item = blockIdx.x * blockDim.x + threadIdx.x; item < total;
       item += gridDim.x * blockDim.x) {
    const int p = find_owner(c.pk, c.count, item);
    const ProbDesc& d = P[c.ids[p]];
    if (input_invalid(d.st)) continue;
    const int m = item - c.pk[p];
    d.mu_sec[m] = d.lam_keep[d.origin[m]] + d.tau[m];
  }
}

__device__ __forceinline__ WSlices wslices_of(const ProbDesc& d, bool mixed) {
  WSlices ws;
  if (mixed) {
    ws.Ws = d.Ws;
    ws.lds = (d.n + 63) / 64 * 64;
    ws.plane = (size_t)ws.lds * (size_t)d.n;
    ws.fcol = d.fcol;
  }
  return ws;
}

template <int K>
__global__ void __launch_bounds__(kAsmThreads, 2) assemble_grouped_kernel(const ProbDesc* __restrict__ P,
                                                                       ClassDesc c, bool vectors,
                                                                       bool mixed) {
  __shared__ double s_n2[kAsmThreads];
  __shared__ double s_mx[kAsmThreads];
  __shared__ int s_ix[kAsmThreads];
  extern __shared__ __align__(16) double s_w[];
  const int total = c.pk[c.count];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int p = find_owner(c.pk, c.count, item);
    const ProbDesc& d = P[c.ids[p]];
    if (input_invalid(d.st)) continue;  // uniform across the CTA
    const Sub sub = sub_of(d);
    const WSlices ws = wslices_of(d, vectors && mixed);
    assemble_root<K>(sub, rootout_of(d), d.n, d.lam_defl, d.st->n_defl, *sub.n_dev, d.mu_sec, d.lam,
                     (vectors && !mixed) ? d.W : nullptr, ws, item - c.pk[p], s_n2, s_mx, s_ix, s_w, 0,
                     vectors ? d.errors : nullptr, d.st);
    __syncthreads();
  }
}

__global__ void deflated_grouped_kernel(const ProbDesc* __restrict__ P, ClassDesc c, bool vectors,
                                        bool mixed) {
  const int total = c.pd[c.count];
  for (int item = blockIdx.x * blockDim.x + threadIdx.x; item < total;
       item += gridDim.x * blockDim.x) {
    const int p = find_owner(c.pd, c.count, item);
    const ProbDesc& d = P[c.ids[p]];
    if (input_invalid(d.st)) continue;
    const int j = item - c.pd[p];
    const int nk = d.st->n_keep;
    const double v = d.lam_defl[j];
    const int64_t pos = j + upper_bound_d(d.mu_sec, nk, v);
    d.lam[pos] = v;
    if (vectors && !mixed) d.W[(int64_t)d.idx_defl[j] + pos * d.n] = 1.0;
    if (vectors && mixed) {  // e_i: 1 = 2^(f-8) * 64 with f = 2
      const int lds = (d.n + 63) / 64 * 64;
      d.Ws[(size_t)pos * lds + d.idx_defl[j]] = __double2bfloat16(64.0);
      d.fcol[pos] = 2;
    }
    if (vectors && d.errors) {
      // w = e_i: r = U Sigma u_i, |r| <= |U|_F |u_i| (the deflation bound),
      // rho - mu = u_i^T Sigma u_i; e_i is orthogonal to every other vector.
      const int i = d.idx_defl[j];
      double un = 0.0, ray = 0.0;
      for (int cc = 0; cc < d.k; ++cc) {
        const double u = d.U[(size_t)cc * d.n + i];
        un = fma(u, u, un);
        ray = fma(sigma_of(d.negmask, cc) * u, u, ray);
      }
      const double normA = d.st->lam_absmax + d.st->fro2;
      const double e0 = sqrt(d.st->fro2 * un) / normA, e1 = fabs(ray) / normA;
      d.errors[pos] = e0;
      d.errors[pos + d.n] = e1;
      d.errors[pos + 3 * (int64_t)d.n] = 0.0;
      atomic_max_nonneg(&d.st->err_max[0], e0);
      atomic_max_nonneg(&d.st->err_max[1], e1);
    }
  }
}

__global__ void class_prefix_kernel(const ProbDesc* __restrict__ P, ClassDesc c) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int sk = 0, sd = 0;
  c.pk[0] = 0;
  c.pd[0] = 0;
  for (int i = 0; i < c.count; ++i) {
    const DevStatus* st = P[c.ids[i]].st;
    const bool bad = input_invalid(st);
    sk += bad ? 0 : st->n_keep;
    sd += bad ? 0 : st->n_defl;
    c.pk[i + 1] = sk;
    c.pd[i + 1] = sd;
  }
  c.counter[0] = 0;
  c.counter[1] = 0;
  c.counter[2] = 0;
}

// Items of roots in pole intervals with several roots go to the front of perm,
// the rest to the back (the order inside each part does not matter: every root
// is solved independently).
__global__ void order_roots_grouped_kernel(const ProbDesc* __restrict__ P, ClassDesc c) {
  const int total = c.pk[c.count];
  for (int item = blockIdx.x * blockDim.x + threadIdx.x; item < total; item += gridDim.x * blockDim.x) {
    const int q = find_owner(c.pk, c.count, item);
    const ProbDesc& d = P[c.ids[q]];
    bool hard = false;
    if (!input_invalid(d.st)) {
      const int n = d.st->n_keep, m = item - c.pk[q];
      int lo = 0, hi = n;  // p = #{poles with count <= m}
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (d.pole_cnt[mid] <= m) lo = mid + 1; else hi = mid;
      }
      const int c_lo = lo > 0 ? d.pole_cnt[lo - 1] : 0;
      const int c_hi = lo < n ? d.pole_cnt[lo] : n;
      hard = (c_hi - c_lo) > 1;
    }
    if (hard) c.perm[atomicAdd(&c.counter[1], 1)] = item;
    else c.perm[total - 1 - atomicAdd(&c.counter[2], 1)] = item;
  }
}

// ---- eigenpairs in a value interval [vl, vu) ------------------------------------
// out: r0 = #{mu' < vl}, r1 = #{mu' < vu} (secular roots, from the two counts),
// qa / qb = first pole >= vl / >= vu, dlo / dsel = first deflated value >= vl
// and how many lie in [vl, vu), n', n_defl.
__global__ void select_window_kernel(Sub sub, const DevStatus* st, const double* __restrict__ lam_defl,
                                     double vl, double vu, const int* __restrict__ c2, int* __restrict__ out) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  if (input_invalid(st)) {
    for (int i = 0; i < 8; ++i) out[i] = 0;
    return;
  }
  const int nk = *sub.n_dev, nd = st->n_defl;
  const int dlo = lower_bound_d(lam_defl, nd, vl), dhi = lower_bound_d(lam_defl, nd, vu);
  out[0] = c2[0];
  out[1] = c2[1];
  out[2] = lower_bound_d(sub.lam, nk, vl);
  out[3] = lower_bound_d(sub.lam, nk, vu);
  out[4] = dlo;
  out[5] = dhi > dlo ? dhi - dlo : 0;
  out[6] = nk;
  out[7] = nd;
}

// Poles outside [p0, p1) get counts that keep the placement of every root in
// [r0, r1) unchanged: 0 below (their true count is <= r0) and n' above (>= r1).
__global__ void select_fill_kernel(int nk, int p0, int p1, int* __restrict__ pole_cnt) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nk; q += gridDim.x * blockDim.x) {
    if (q < p0) pole_cnt[q] = 0;
    else if (q >= p1) pole_cnt[q] = nk;
  }
}

__global__ void mu_select_kernel(Sub sub, RootOut roots, int r0, int r1, double* __restrict__ mu_sec) {
  for (int m = r0 + blockIdx.x * blockDim.x + threadIdx.x; m < r1; m += gridDim.x * blockDim.x)
    mu_sec[m] = sub.lam[roots.origin[m]] + roots.tau[m];
}

// Selected secular roots: position (m - r0) + #{selected deflated values < mu}.
template <int K>
__global__ void __launch_bounds__(kAsmThreads) assemble_select_kernel(
    Sub sub, RootOut roots, int64_t n, const double* __restrict__ lam_dsel, int dsel, int r0, int r1,
    const double* __restrict__ mu_sec, double* __restrict__ mu_out, double* __restrict__ W) {
  __shared__ double s_n2[kAsmThreads];
  __shared__ double s_mx[kAsmThreads];
  __shared__ int s_ix[kAsmThreads];
  extern __shared__ __align__(16) double s_w[];
  const int nk = *sub.n_dev;
  for (int m = r0 + blockIdx.x; m < r1; m += gridDim.x) {
    assemble_root<K>(sub, roots, n, lam_dsel, dsel, nk, mu_sec, mu_out, W, WSlices(), m, s_n2, s_mx, s_ix,
                     s_w, r0);
    __syncthreads();
  }
}

// Selected deflated pairs: position j + #{selected secular roots <= lam}, W column e_i.
__global__ void deflated_select_kernel(int64_t n, const int* __restrict__ idx_dsel,
                                       const double* __restrict__ lam_dsel, int dsel,
                                       const double* __restrict__ mu_sel, int nsel,
                                       double* __restrict__ mu_out, double* __restrict__ W) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < dsel; j += gridDim.x * blockDim.x) {
    const double v = lam_dsel[j];
    const int64_t pos = j + upper_bound_d(mu_sel, nsel, v);
    mu_out[pos] = v;
    if (W) W[(int64_t)idx_dsel[j] + pos * n] = 1.0;
  }
}

template <int K>
cudaError_t launch_assemble_select_k(const Sub& sub, const RootOut& roots, int64_t n, const int* idx_defl,
                                     const double* lam_defl, int dlo, int dsel, int r0, int r1,
                                     double* mu_sec, double* mu_out, double* W, cudaStream_t s) {
  const int cnt = r1 - r0;
  if (cnt > 0) {
    mu_select_kernel<<<(cnt + 255) / 256, 256, 0, s>>>(sub, roots, r0, r1, mu_sec);
    const cudaError_t e = allow_asm_smem(assemble_select_kernel<K>);
    if (e != cudaSuccess) return e;
    assemble_select_kernel<K><<<cnt < 65535 ? cnt : 65535, kAsmThreads, kAsmSmem, s>>>(
        sub, roots, n, lam_defl + dlo, dsel, r0, r1, mu_sec, mu_out, W);
  }
  if (dsel > 0)
    deflated_select_kernel<<<(dsel + 255) / 256, 256, 0, s>>>(n, idx_defl + dlo, lam_defl + dlo, dsel,
                                                              mu_sec + r0, cnt, mu_out, W);
  return cudaGetLastError();
}

int g_occ_roots[17];

template <int K>
cudaError_t launch_counts_k(const Sub& sub, const double* x, int npts, int* counts,
                            cudaStream_t s, int pt0, int pt_end) {
  constexpr int G = 4 / warps_per_root(K);
  const int pts = x ? npts : min(sub.ld, pt_end) - pt0;
  int blocks = (pts + G - 1) / G;
  if (blocks < 1) blocks = 1;
  if (blocks > 65535) blocks = 65535;
  counts_kernel<K><<<blocks, 128, 0, s>>>(sub, x, npts, counts, pt0, pt_end);
  return cudaGetLastError();
}

template <int K>
cudaError_t launch_roots_k(const Sub& sub, const int* pole_cnt, int max_iter, int* counter,
                           const RootOut& out, DevStatus* st, int num_sms, cudaStream_t s,
                           int m_count, int m_end) {
  constexpr int G = 4 / warps_per_root(K);
  if (g_occ_roots[K] == 0) {
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, roots_kernel<K>, 128, 0);
    if (e != cudaSuccess) return e;
    g_occ_roots[K] = occ > 0 ? occ : 1;
  }
  long long want = ((long long)m_count + G - 1) / G;
  long long cap = (long long)num_sms * g_occ_roots[K];
  int blocks = (int)(want < cap ? want : cap);
  if (blocks < 1) blocks = 1;
  roots_kernel<K><<<blocks, 128, 0, s>>>(sub, pole_cnt, max_iter, counter, out, st, m_end);
  return cudaGetLastError();
}

template <int K>
cudaError_t launch_assemble_k(const Sub& sub, const RootOut& roots, int64_t n,
                              const int* idx_defl, const double* lam_defl, const DevStatus* st,
                              double* mu_sec, double* lam_out, double* W, cudaStream_t s,
                              const WSlices& ws) {
  const int ld = sub.ld;
  mu_kernel<<<(ld + 255) / 256, 256, 0, s>>>(sub, roots, mu_sec);
  int blocks = ld < 65535 ? ld : 65535;
  const cudaError_t e = allow_asm_smem(assemble_kernel<K>);
  if (e != cudaSuccess) return e;
  assemble_kernel<K><<<blocks, kAsmThreads, kAsmSmem, s>>>(sub, roots, n, lam_defl, st, mu_sec, lam_out, W,
                                                     ws);
  int nb = (int)((n + 255) / 256);
  if (nb > 4096) nb = 4096;
  deflated_kernel<<<nb, 256, 0, s>>>(sub, n, idx_defl, lam_defl, st, mu_sec, lam_out, W, ws);
  return cudaGetLastError();
}



int g_occ_roots_grouped[17];

template <int K>
cudaError_t counts_grouped_k(const ProbDesc* P, const ClassDesc& c, int max_items, bool mixed, int passes,
                             cudaStream_t s) {
  constexpr int G = 4 / warps_per_root(K);
  int blocks = (max_items + G - 1) / G;
  if (blocks < 1) blocks = 1;
  if (blocks > 65535) blocks = 65535;
  if (!mixed) {
    counts_grouped_kernel<K, 0><<<blocks, 128, 0, s>>>(P, c);
    return cudaGetLastError();
  }
  if (passes & 1) {
    counts_grouped_kernel<K, 1><<<blocks, 128, 0, s>>>(P, c);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (!(passes & 2)) return cudaSuccess;
  constexpr int G2 = (K >= 7) ? 1 : (K >= 3 ? 2 : 4);  // points per CTA of the recount
  int blocks2 = (max_items + G2 - 1) / G2;
  if (blocks2 < 1) blocks2 = 1;
  if (blocks2 > 65535) blocks2 = 65535;
  counts_grouped_kernel<K, 2><<<blocks2, 128, 0, s>>>(P, c);
  return cudaGetLastError();
}

template <int K>
cudaError_t roots_grouped_k(const ProbDesc* P, const ClassDesc& c, int max_items, int max_iter,
                            int num_sms, cudaStream_t s, int occ_div) {
  constexpr int G = 4 / warps_per_root(K);
  if (g_occ_roots_grouped[K] == 0) {
    int occ = 0;
    cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, roots_grouped_kernel<K>, 128, 0);
    if (e != cudaSuccess) return e;
    g_occ_roots_grouped[K] = occ > 0 ? occ : 1;
  }
  long long want = ((long long)max_items + G - 1) / G;
  const int per_sm = g_occ_roots_grouped[K] / (occ_div > 1 ? occ_div : 1);
  long long cap = (long long)num_sms * (per_sm > 0 ? per_sm : 1);
  int blocks = (int)(want < cap ? want : cap);
  if (blocks < 1) blocks = 1;
  roots_grouped_kernel<K><<<blocks, 128, 0, s>>>(P, c, max_iter);
  return cudaGetLastError();
}

template <int K>
cudaError_t assemble_grouped_k(const ProbDesc* P, const ClassDesc& c, int max_items, int max_defl,
                               bool vectors, bool mixed, cudaStream_t s) {
  const int mb = max_items > 0 ? (max_items + 255) / 256 : 1;
  mu_grouped_kernel<<<mb < 4096 ? mb : 4096, 256, 0, s>>>(P, c);
  const int ab = max_items > 0 ? (max_items < 65535 ? max_items : 65535) : 1;
  const cudaError_t e = allow_asm_smem(assemble_grouped_kernel<K>);
  if (e != cudaSuccess) return e;
  assemble_grouped_kernel<K><<<ab, kAsmThreads, kAsmSmem, s>>>(P, c, vectors, mixed);
  const int db = max_defl > 0 ? (max_defl + 255) / 256 : 1;
  deflated_grouped_kernel<<<db < 4096 ? db : 4096, 256, 0, s>>>(P, c, vectors, mixed);
  return cudaGetLastError();
}

}  // namespace

#ifdef EIG_SECULAR_K
// Per-rank entry points (declared in secular_entries.cuh), defined only in the
// translation unit that instantiates them.
template <int K>
cudaError_t sec_counts(const Sub& sub, const double* x, int npts, int* counts, cudaStream_t s, int pt0,
                       int pt_end) {
  return launch_counts_k<K>(sub, x, npts, counts, s, pt0, pt_end);
}
template <int K>
cudaError_t sec_roots(const Sub& sub, const int* pole_cnt, int max_iter, int* counter, const RootOut& out,
                      DevStatus* st, int num_sms, cudaStream_t s, int m_count, int m_end) {
  return launch_roots_k<K>(sub, pole_cnt, max_iter, counter, out, st, num_sms, s, m_count, m_end);
}
template <int K>
cudaError_t sec_assemble(const Sub& sub, const RootOut& roots, int64_t n, const int* idx_defl,
                         const double* lam_defl, const DevStatus* st, double* mu_sec, double* lam_out, double* W,
                         cudaStream_t s, const WSlices& ws) {
  return launch_assemble_k<K>(sub, roots, n, idx_defl, lam_defl, st, mu_sec, lam_out, W, s, ws);
}
template <int K>
cudaError_t sec_assemble_select(const Sub& sub, const RootOut& roots, int64_t n, const int* idx_defl,
                                const double* lam_defl, int dlo, int dsel, int r0, int r1, double* mu_sec,
                                double* mu_out, double* W, cudaStream_t s) {
  return launch_assemble_select_k<K>(sub, roots, n, idx_defl, lam_defl, dlo, dsel, r0, r1, mu_sec, mu_out, W, s);
}
template <int K>
cudaError_t sec_counts_grouped(const ProbDesc* P, const ClassDesc& c, int max_items, bool mixed, int passes,
                               cudaStream_t s) {
  return counts_grouped_k<K>(P, c, max_items, mixed, passes, s);
}
template <int K>
cudaError_t sec_roots_grouped(const ProbDesc* P, const ClassDesc& c, int max_items, int max_iter, int num_sms,
                              cudaStream_t s, int occ_div) {
  return roots_grouped_k<K>(P, c, max_items, max_iter, num_sms, s, occ_div);
}
template <int K>
cudaError_t sec_assemble_grouped(const ProbDesc* P, const ClassDesc& c, int max_items, int max_defl,
                                 bool vectors, bool mixed, cudaStream_t s) {
  return assemble_grouped_k<K>(P, c, max_items, max_defl, vectors, mixed, s);
}
#endif
}  // namespace eig
