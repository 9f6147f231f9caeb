// eig_internal.cuh -- shared declarations of the CUDA path (device helpers and
// launch wrappers).  Everything here belongs to the product library only.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/eig_update.h"

namespace eig {

constexpr int kWarp = 32;
constexpr double kEps = 2.220446049250313e-16;  // 2^-52, FP64 machine epsilon

// Ranks with a compiled secular kernel; other k are padded with zero columns
// of U carrying sigma = +1, which leaves the count, det and null vector of the
// k x k problem unchanged (an extra eigenvalue +1, counted in k_plus).
__host__ __device__ constexpr int padded_rank(int k) { return k <= 8 ? k : ((k + 1) / 2) * 2; }

// Warps that share one root.  Rows a and K-1-a of the k x k matrices are
// paired (K+1 upper-triangle entries per pair); pairs are dealt round-robin to
// the warps so that each warp keeps <= 39 entries of M(x) and of N(x) in
// registers.
__host__ __device__ constexpr int warps_per_root(int K) { return K <= 8 ? 1 : K <= 12 ? 2 : 4; }

// Status bits written by the kernels into the handle's device status block.
enum : int {
  ST_UNSORTED = 1,
  ST_NONFINITE = 2,
  ST_NOTCONV = 4,
  ST_TIMEOUT = 8,
};

// Per-update device status block (one cache line).
struct DevStatus {
  int flags;
  int n_keep;
  int n_defl;
  int iters_max;
  long long iters_total;   // FP64 evaluations of the zero finder
  long long n_notconv;
  double lam_absmax;
  double fro2;
  double lo_sent;
  double hi_sent;
  long long iters32_total; // FP32 (coarse-phase) evaluations
  long long redo32_total;  // FP32 evaluations whose count was not certified
  long long gj32_total;    // certified FP32 evaluations whose k x k step was a Gauss-Jordan inverse
  long long taylor_total;  // evaluations by a first-order update of the K x K sums
  int n_runs;              // runs of exactly repeated lam rotated before deflation
  int run_rows;            // rows in those runs
  double err_max[3];       // per-eigenpair report maxima: residual, Rayleigh shift,
                           // next-vector dot (non-negative: atomicMax on the bits)
  long long tc_pair_tiles; // 128 x 128 x 32 BF16 slice-pair products the split GEMM issues
  long long asm_fp64_cols; // mixed mode: columns of W whose entries were formed in FP64
};

// Public status of a finished update from its device status block (shared by
// every entry point, so that they map the flags the same way).
inline int status_of(const DevStatus& s) {
  if (s.flags & (ST_UNSORTED | ST_NONFINITE)) return EIG_EINVAL;
  if (s.flags & ST_TIMEOUT) return EIG_ETIMEOUT;
  if (s.flags & ST_NOTCONV) return EIG_ENOTCONV;
  return EIG_OK;
}

// sigma (host k entries of +1/-1, NULL = all +1) as the bit mask of the -1
// columns and the number of +1 columns; false for any other entry.
inline bool sigma_info(const int8_t* sigma, int k, unsigned long long* negmask, int* kplus) {
  unsigned long long m = 0;
  int kp = 0;
  for (int c = 0; c < k; ++c) {
    const int v = sigma ? sigma[c] : 1;
    if (v == 1) {
      ++kp;
    } else if (v == -1) {
      m |= 1ull << c;
    } else {
      return false;
    }
  }
  *negmask = m;
  *kplus = kp;
  return true;
}

// The non-deflated sub-problem in the layout the secular kernels read.  Its
// size n' is only known on the device (written by the deflation kernel), so
// kernels read it through n_dev and are launched for the worst case ld.
struct Sub {
  const int* n_dev; // n' (rows kept), device
  int ld;           // leading dimension of Us (>= n, multiple of 32)
  int K;            // padded rank
  int kplus;        // #{sigma = +1} including padding columns
  const double* lam;  // n' ascending
  const double* Us;   // K arrays of ld doubles: Us[c*ld + i] = U'[i][c]
  const int* idx;     // n': original row index of kept row i
  const DevStatus* st;       // lo_sent / hi_sent: strict bounds on every root (Weyl)
  unsigned long long negmask;  // bit c set when sigma_c = -1
  // FP32 copies for the coarse phase of the zero finder (null: FP64 only):
  // lam' as (hi, lo) float pairs, U' as K float arrays of ld.
  const float2* lamf = nullptr;
  const float* Usf = nullptr;
  // Mixed mode with vectors: U' - Usf rounded to FP32 (U' = Usf + Ulo to 2^-48
  // relative), for the double-float eq. (10) entries of the assembly; or null.
  const float* Ulo = nullptr;
  // Products u_ia u_ib (a <= b, row-major over the upper triangle) of every
  // kept row, K(K+1)/2 arrays of ld doubles (null: form them from Us).  The
  // zero finder's FP64 sums then take M^_ab += r_i (u_ia u_ib) without the K
  // multiplications t = r u per term.
  const double* Pp = nullptr;
};

// Per-root outputs of the zero finder.
struct RootOut {
  int* origin;      // pole index (into Sub) the root is measured from
  double* tau;      // mu - lam[origin]
  int* iters;       // evaluations
  int* flags;       // 1 = hit the cap
  double* alpha;    // K per root: null vector of Sigma - M(mu) (eq. (10) alpha_0)
  double* beta;     // 2 per root: u_i^T alpha / (mu - lam_i) at the bracketing poles
  int* sidx;        // 2 per root: indices of the bracketing poles (-1: none)
};

// Reciprocal of d to within about one ulp, cheaper on the FP64 pipe than the
// correctly rounded division: the hardware's fast approximation y0 =
// rcp.approx.ftz.f64(d), refined by one step of the cubically convergent
// Newton-Raphson iteration for f(y) = 1/y - d,
//   e = 1 - d y0,  y1 = y0 (1 + e + e^2)   (the series of 1/(1 - e) truncated),
// so the relative error of y0 is cubed.  d with a zero, subnormal, infinite
// or NaN exponent field goes through the division (checked on the integer
// pipe), so the result equals 1/d's special cases.
__device__ __forceinline__ double rcp_nr(double d) {
  const unsigned ex = ((unsigned)__double2hiint(d) >> 20) & 0x7ffu;
  if (ex == 0u || ex >= 0x7feu) return 1.0 / d;
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
  const double e = fma(-d, y, 1.0);
  return fma(y, fma(e, e, e), y);
}

// ---- split-BF16 tensor-core GEMM (gemm_tc.cu) ------------------------------
constexpr int kTcSlices = 5;

// Exponent e with |v| < 2^(e-1) for mx = max |v| (0 for an all-zero vector).
__device__ __forceinline__ int tc_scale_exp(double mx) {
  if (!(mx > 0.0)) return 0;
  int E;
  frexp(mx, &E);  // mx = f 2^E, f in [1/2, 1)
  return E + 1;
}

// Five balanced 8-bit digits of a scaled value.  R = rint(y * 2^40) is formed
// exactly with one FMA against the constant 1.5 * 2^52 (valid while
// |y 2^40| < 2^51), then peeled into base-256 digits m_4..m_0 in [-128, 128]
// (least significant first, each digit chosen in [-128, 127] and the carry
// shifted up), so that y = 2^-8 sum_p m_p 2^(-8p) up to 2^-41.  Slice p holds
// m_p 2^(-8p) (exact in BF16).  tc_split_scaled takes x and the exact power-of-
// two factor s with y = x * s, so the product is rounded only once.
// s40 = s * 2^40 (exact): callers that split many entries with one scale pass
// it precomputed, leaving one FMA per entry on the FP64 pipe.
__device__ __forceinline__ void tc_split_prescaled(double x, double s40, __nv_bfloat16 (&out)[kTcSlices]) {
  const double magic = 6755399441055744.0;  // 1.5 * 2^52
  long long R = __double_as_longlong(fma(x, s40, magic)) - __double_as_longlong(magic);
  int m[kTcSlices];
#pragma unroll
  for (int p = kTcSlices - 1; p > 0; --p) {
    int d = (int)(R & 255);
    if (d >= 128) d -= 256;
    m[p] = d;
    R = (R - d) >> 8;
  }
  m[0] = (int)R;
#pragma unroll
  for (int p = 0; p < kTcSlices; ++p) out[p] = __float2bfloat16_rn(ldexpf((float)m[p], -8 * p));
}

__device__ __forceinline__ void tc_split_scaled(double x, double s, __nv_bfloat16 (&out)[kTcSlices]) {
  tc_split_prescaled(x, s * 1099511627776.0, out);
}

// ---- double-float arithmetic (pairs of FP32) ---------------------------------
// A value h + l with |l| <= ulp(h) / 2: 48 significant bits on the FP32 pipe,
// whose rate on this part is 64 times the FP64 pipe's.  Error-free transforms
// after Knuth (two-sum) and the FMA product; the products and quotients below
// carry relative errors of a few units of 2^-48.
struct DF {
  float h, l;
};
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return DF{s, (a - (s - bb)) + (b - bb)};
}
// h + l renormalised when |h| >= |l| (or h = 0).
__device__ __forceinline__ DF df_fast(float h, float l) {
  const float s = h + l;
  return DF{s, l - (s - h)};
}
// x as a pair from the bits of x, with no FP64 arithmetic and no FP64/FP32
// conversion (those take many FP64-pipe cycles on this part): h = x
// truncated to 24 significant bits, l = the other 29 fraction bits rounded to
// 24.  Zero and |x| in [2^-60, 2^60) return true; other x (tiny, huge, Inf,
// NaN) return false and a zero pair.
__device__ __forceinline__ bool df_bits(double x, DF& out) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32);
  const int ex = (int)((hi >> 20) & 0x7ffu) - 1023;
  const unsigned sign = hi & 0x80000000u;
  if (ex < -60 || ex > 59) {
    out = DF{0.0f, 0.0f};
    return (b << 1) == 0ull;
  }
  const float h = __uint_as_float(sign | ((unsigned)(ex + 127) << 23) | (unsigned)((b >> 29) & 0x7fffffu));
  const unsigned r = (unsigned)(b & 0x1fffffffu);
  // r < 2^29 as r_hi 2^16 + r_lo, both exact in FP32 (2^23 + v - 2^23)
  const float rh = __uint_as_float(0x4b000000u | (r >> 16)) - 8388608.0f;
  const float rl = __uint_as_float(0x4b000000u | (r & 0xffffu)) - 8388608.0f;
  const float l = fmaf(rh, 65536.0f, rl) * __uint_as_float((unsigned)(ex - 52 + 127) << 23);
  out = DF{h, sign ? -l : l};
  return true;
}
// An FP32 value as FP64 from its bits, exactly (zero, subnormal, Inf and NaN
// included), without the conversion's FP64-pipe cycles.
__device__ __forceinline__ double d_of_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  unsigned e = (u >> 23) & 0xffu;
  unsigned m = u & 0x7fffffu;
  if (e == 0u) {
    if (m == 0u) return __longlong_as_double((long long)sign);
    const int sh = __clz(m) - 8;  // normalise: leading one to bit 23
    m = (m << sh) & 0x7fffffu;
    e = 1u - (unsigned)sh;        // as a biased FP32 exponent (may wrap below 1)
    return __longlong_as_double((long long)(sign | ((unsigned long long)(e + 896u) << 52) |
                                            ((unsigned long long)m << 29)));
  }
  const unsigned long long de = (e == 0xffu) ? 0x7ffull : (unsigned long long)(e + 896u);
  return __longlong_as_double((long long)(sign | (de << 52) | ((unsigned long long)m << 29)));
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return df_fast(p, e);
}
// 1 / d from an FP32 seed and one Newton step carried in the pair:
// r = r0 (1 + e + e^2), e = 1 - d r0 (|e| <= 2^-22).
__device__ __forceinline__ DF df_rcp(DF d) {
  float r0;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(d.h));
  float e = fmaf(-d.h, r0, 1.0f);
  e = fmaf(-d.l, r0, e);
  const float re = r0 * e;
  return df_fast(r0, fmaf(re, e, re));
}

// The five digits of tc_split_prescaled from a pair y = h + l, |y| < 2^39:
// digits are peeled from the top (q = rint(h / 2^(8j)), h -= q 2^(8j), exact),
// the pair renormalised after each step so that h carries the rounded value.
// The digits sum to rint(y) up to the last place; |m_p| <= 129 (exact in
// BF16, and within the exact-accumulation bound of the GEMM).
__device__ __forceinline__ void tc_split_df(DF y, __nv_bfloat16 (&out)[kTcSlices]) {
  float h = y.h, l = y.l;
  float m[kTcSlices];
#pragma unroll
  for (int p = 0; p < kTcSlices - 1; ++p) {
    const float unit = __int_as_float((127 + 8 * (kTcSlices - 1 - p)) << 23);  // 2^(8(4-p))
    const float q = rintf(h * __int_as_float((127 - 8 * (kTcSlices - 1 - p)) << 23));
    h = fmaf(-q, unit, h);
    const DF r = df_two_sum(h, l);
    h = r.h;
    l = r.l;
    m[p] = q;
  }
  m[kTcSlices - 1] = rintf(h + l);
#pragma unroll
  for (int p = 0; p < kTcSlices; ++p) out[p] = __float2bfloat16_rn(ldexpf(m[p], -8 * p));
}

__device__ __forceinline__ void tc_split(double r, __nv_bfloat16 (&out)[kTcSlices]) {
  tc_split_scaled(r, 1.0, out);
}

// W written directly as slices (mixed mode): Ws[q][r][j] for W[j, r], leading
// dimension lds, plane stride `plane`; fcol[r] = column exponent.
struct WSlices {
  __nv_bfloat16* Ws = nullptr;
  size_t plane = 0;
  int lds = 0;
  int* fcol = nullptr;
};

// Words of the non-zero map of W's two leading digit slices for an n x n
// update: word (r / 128) * ceil(n / 32) + j / 32 has bit q set when slice q
// (q = 0, 1) holds a non-zero entry in that 128-column x 32-row tile of W^T,
// the operand tiles of the split GEMM, which skips MMAs against all-zero ones.
__host__ __device__ inline size_t wnz_words(int n) { return (size_t)((n + 127) / 128) * (size_t)((n + 31) / 32); }

// ---- one update as seen by the grouped kernels -------------------------------
// Every launch processes a table of updates (a single update is a table of
// one).  Work items of a stage are numbered across the table; a kernel maps
// an item to (update, local index) by binary search in a prefix array.
struct ProbDesc {
  int n, k, K, ld, kplus, pad_;
  unsigned long long negmask;
  const double* Q;   // caller: n x n old eigenvectors (column-major)
  double* lam;       // caller: n eigenvalues, in/out
  const double* Km;  // caller: n x k perturbation
  double* Xout;      // n x n new eigenvectors (caller's Q_out or workspace)
  double* Qback;     // caller's Q when the update is in place (X copied back), else null
  double* U;
  double* lam_keep;
  double* Us;
  int* idx_keep;
  int* idx_defl;
  double* lam_defl;
  int* pole_cnt;
  int* origin;
  double* tau;
  int* iters;
  int* rflags;
  double* alpha;
  double* beta;
  int* sidx;
  double* mu_sec;
  double* lam_old;
  double* W;               // FP64 mode
  __nv_bfloat16* Qs;       // mixed mode
  __nv_bfloat16* Ws;
  int* erow;
  int* fcol;
  unsigned long long* rmax;
  DevStatus* st;
  float2* lamf;            // mixed mode: FP32 copies for the coarse zero-finder phase
  float* Usf;
  float* Ulo;              // mixed mode with vectors: low parts of U' (see Sub)
  double* Vr;              // reflectors of the runs of equal lam (n x k), see runs.cu
  double* taur;            // their scalars (n)
  int* runs;               // (g0, m) pairs (n ints)
  double* errors;          // caller: n x 4 per-eigenpair report (column-major), or null
  double* Pp;              // products u_ia u_ib of the kept rows, K(K+1)/2 arrays of ld (see Sub)
  unsigned* wnz;           // mixed mode: non-zero map of W's two leading slices (see WSlices)
  float* Kh;               // mixed mode: K's columns scaled by 2^-Kexp[c], FP32 high parts (n x k)
  float* Kl;               // and low parts
  int* Kexp;               // per column of K (16 entries)
};

__host__ __device__ inline Sub sub_of(const ProbDesc& d) {
  Sub s;
  s.n_dev = &d.st->n_keep;
  s.ld = d.ld;
  s.K = d.K;
  s.kplus = d.kplus;
  s.lam = d.lam_keep;
  s.Us = d.Us;
  s.idx = d.idx_keep;
  s.st = d.st;
  s.negmask = d.negmask;
  s.lamf = d.lamf;
  s.Usf = d.Usf;
  s.Ulo = d.Ulo;
  s.Pp = d.Pp;
  return s;
}

__host__ __device__ inline RootOut rootout_of(const ProbDesc& d) {
  RootOut r;
  r.origin = d.origin;
  r.tau = d.tau;
  r.iters = d.iters;
  r.flags = d.rflags;
  r.alpha = d.alpha;
  r.beta = d.beta;
  r.sidx = d.sidx;
  return r;
}

// Index of the last prefix entry <= item (prefix[0] = 0, ascending, count+1 entries).
template <typename T>
__device__ __forceinline__ int find_owner(const T* prefix, int count, T item) {
  int lo = 0, hi = count;  // answer in [0, count)
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= item) lo = mid; else hi = mid;
  }
  return lo;
}

// A set of updates sharing one padded rank K (the secular kernels are
// compiled per K).  ids: device indices into the ProbDesc table; pk / pd:
// device prefix sums (count+1) of the kept / deflated sizes, written by
// launch_class_prefix after deflation; counter: device work counter.
struct ClassDesc {
  int K;
  int count;
  const int* ids;
  int* pk;
  int* pd;
  int* counter;   // 3 ints: the zero finder's work counter, then two partition counters
  int* perm;      // class items in the order the zero finder takes them (null: natural order)
};

// Launch schedule of a table's secular stages (results are identical for
// every schedule: it orders and overlaps work, it does not change arithmetic).
struct Sched {
  int streams = 1;  // > 1: each rank class's stages on its own stream (classes overlap)
  int order = 1;    // 1: roots of multi-root pole intervals first; 0: natural order
  int occ_div = 1;  // zero-finder persistent grid at 1/occ_div of the resident blocks
  bool side = true; // mixed mode: Q's slices on a side stream, overlapping the secular stages
};

// ---- launch wrappers (defined in the .cu files) ----------------------------
cudaError_t launch_project_f64(int64_t n, int k, const double* Q, const double* K, double* U,
                               cudaStream_t s);
// U = Q^T K for every update of the table; col_prefix (device, count+1): prefix
// sums of n over the table.
// U = Q^T K of one update in double-float arithmetic (as the mixed-mode table
// forms it): Kh, Kl n x k floats, Kexp k ints of scratch.
cudaError_t launch_project_mixed(int64_t n, int k, const double* Q, const double* K, double* U, float* Kh,
                                 float* Kl, int* Kexp, cudaStream_t s);
// mixed: U in double-float arithmetic (K split by a kernel first; ProbDesc::Kh,
// Kl, Kexp), a column with values outside that range in FP64.
cudaError_t launch_project_grouped(const ProbDesc* P, int count, const long long* col_prefix,
                                   long long total_cols, cudaStream_t s, bool mixed = false);
// Deflation + compaction for every update (one CTA each); also keeps lam_old.
cudaError_t launch_deflate_grouped(const ProbDesc* P, int count, cudaStream_t s);
// Products u_ia u_ib of the kept rows into ProbDesc::Pp (updates with Pp set);
// colpre: device prefix of n over the table.
cudaError_t launch_products_grouped(const ProbDesc* P, int count, const long long* colpre, long long total,
                                    cudaStream_t s);
// The same for one sub-problem (Us: K arrays of ld; n' read from st).
cudaError_t launch_products(const double* Us, int K, int ld, const DevStatus* st, double* Pp, cudaStream_t s);
// Runs of exactly repeated lam (runs.cu): QR of each run's rows of U before
// deflation, then B applied to W's rows (FP64 GEMM paths) or Q~ = Q B written
// to Xout (split-BF16 path).
cudaError_t launch_runs_qr(int64_t n, int k, const double* lam, double* U, double* V, double* tau, int* runs,
                           DevStatus* st, cudaStream_t s);
cudaError_t launch_runs_qr_grouped(const ProbDesc* P, int count, int64_t max_n, cudaStream_t s);
cudaError_t launch_runs_apply_w(int64_t n, int k, const double* V, const double* tau, const int* runs,
                                const DevStatus* st, double* W, int64_t ldw, int64_t ncols, int num_sms,
                                cudaStream_t s);
cudaError_t launch_runs_apply_w_grouped(const ProbDesc* P, int count, int num_sms, cudaStream_t s);
cudaError_t launch_runs_rotate_q_grouped(const ProbDesc* P, int count, int num_sms, cudaStream_t s);
// Prefix sums of n_keep and n_defl over a class (one small kernel).
cudaError_t launch_class_prefix(const ProbDesc* P, const ClassDesc& c, cudaStream_t s);
// Grouped secular stages for one class (pole counts, zero finder, assembly).
// Mixed-mode pole counts run as two launches: passes bit 1 = the certified
// FP32 pass (an uncertified count is written as -1), bit 2 = the FP64 recount
// of those; FP64 mode ignores passes.
cudaError_t launch_counts_grouped(const ProbDesc* P, const ClassDesc& c, int max_items, bool mixed,
                                  cudaStream_t s, int passes = 3);
// occ_div > 1 caps the persistent grid at 1/occ_div of the resident blocks
// per SM (a schedule choice of the batch tuner; results are unchanged).
cudaError_t launch_roots_grouped(const ProbDesc* P, const ClassDesc& c, int max_items, int max_iter,
                                 int num_sms, cudaStream_t s, int occ_div = 1);
// Order the zero finder's work: roots in pole intervals that hold several roots
// (the ones that need the most evaluations) first, so they do not finish last.
cudaError_t launch_order_roots_grouped(const ProbDesc* P, const ClassDesc& c, int max_items, cudaStream_t s);
cudaError_t launch_assemble_grouped(const ProbDesc* P, const ClassDesc& c, int max_items,
                                    int max_defl, bool vectors, bool mixed, cudaStream_t s);
cudaError_t launch_make_rank2(int64_t n, int64_t j, const double* a, double* K, cudaStream_t s);
// lamf / Usf (optional): FP32 copies of the kept lam' (hi, lo pairs) and U'.
cudaError_t launch_deflate(int64_t n, int k, int K, const double* lam, const double* U,
                           unsigned long long negmask, double* lam_keep, double* Us, int ld,
                           int* idx_keep, int* idx_defl, double* lam_defl, DevStatus* st,
                           cudaStream_t s, float2* lamf = nullptr, float* Usf = nullptr);
// Root counts #{mu < x}: at the poles [pt0, min(n', pt_end)) of the sub-problem
// (x == nullptr; counts[q] for pole q) or at npts absolute points x.
cudaError_t launch_counts(const Sub& sub, const double* x, int npts, int* counts, cudaStream_t s,
                          int pt0 = 0, int pt_end = 0x7fffffff);
// Zero finder over the roots [*work_counter, min(n', m_end)); m_count (an upper
// bound on how many, -1 = ld) sizes the grid.
cudaError_t launch_roots(const Sub& sub, const int* pole_cnt, int max_iter, int* work_counter,
                         const RootOut& out, DevStatus* st, int num_sms, cudaStream_t s,
                         int m_count = -1, int m_end = 0x7fffffff);
// mu of every secular root, output positions, new eigenvalues (ascending,
// merged with the deflated ones) and, when W != nullptr, the eq. (10) columns
// of W (n x n, column-major, zero-filled beforehand by the caller).
cudaError_t launch_assemble(const Sub& sub, const RootOut& roots, int64_t n, const int* idx_defl,
                            const double* lam_defl, const DevStatus* st, double* mu_sec,
                            double* lam_out, double* W, cudaStream_t s,
                            const WSlices& ws = WSlices());
// Eigenpairs in [vl, vu) (secular.cu): the window of counts and indices (8 ints,
// see select_window_kernel), placeholder pole counts outside the pole window
// [p0, p1), and the assembly of the selected pairs into mu_out (ascending) and
// W (n x m, zero-filled beforehand; may be null).
cudaError_t launch_select_window(const Sub& sub, const DevStatus* st, const double* lam_defl, double vl,
                                 double vu, const int* c2, int* out, cudaStream_t s);
cudaError_t launch_select_fill(int nk, int p0, int p1, int* pole_cnt, cudaStream_t s);
cudaError_t launch_assemble_select(const Sub& sub, const RootOut& roots, int64_t n, const int* idx_defl,
                                   const double* lam_defl, int dlo, int dsel, int r0, int r1, double* mu_sec,
                                   double* mu_out, double* W, cudaStream_t s);
cudaError_t launch_gemm_f64(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda,
                            const double* B, int64_t ldb, double* C, int64_t ldc, cudaStream_t s);
// Same, but skipped on the device when st reports invalid input.
cudaError_t launch_gemm_f64_guarded(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda,
                                    const double* B, int64_t ldb, double* C, int64_t ldc,
                                    const DevStatus* st, cudaStream_t s);
// First-order perturbation estimate of eq. (11) (perturb.cu).  W = I + E with
// E_ij = u_i^T Sigma u_j / (lam_j - lam_i) (0 where lam_i == lam_j), written
// column-major, or as W^T column-major when transposed.  mu_j = lam_j + u_j^T Sigma u_j.
cudaError_t launch_perturb_w(int64_t n, int k, const double* lam, const double* U, unsigned long long negmask,
                             bool transposed, double* W, cudaStream_t s);
cudaError_t launch_perturb_mu(int64_t n, int k, const double* lam, const double* U, unsigned long long negmask,
                              double* mu, cudaStream_t s);
// Column 2 (nearest-eigenvalue gap) of the per-eigenpair report of every
// update of the table that asked for one; colpre: device prefix of n.
cudaError_t launch_errors_gap_grouped(const ProbDesc* P, int count, const long long* colpre, long long total,
                                      cudaStream_t s);
// Small helpers (util.cu).
cudaError_t launch_copy_guarded(double* dst, const double* src, int64_t count, const DevStatus* st,
                                cudaStream_t s);
cudaError_t launch_prepare_undeflated(int64_t n, int k, int K, const double* lam, const double* U,
                                      double* lam_keep, double* Us, int ld, int* idx_keep,
                                      DevStatus* st, cudaStream_t s);
cudaError_t launch_scatter_iters(const Sub& sub, int64_t n, const int* root_iters,
                                 const double* lam_defl, const double* mu_sec, int* iters_out,
                                 cudaStream_t s);
// Residual |A' x - mu x| and pairwise x_i^T x_j for ncols sampled columns
// (A' = Q diag(lam) Q^T + K Sigma K^T with the OLD Q and lam).  out: ncols
// residuals followed by ncols*ncols Gram entries.  tmp: 3*n*ncols doubles.
cudaError_t launch_check_pairs(int64_t n, int k, const double* Q, const double* lam,
                               const double* K, unsigned long long negmask, const double* X,
                               const double* mu, const int* cols, int ncols, double* tmp,
                               double* out, cudaStream_t s);


// Slice arrays hold tc_num_slices() planes of n rows x tc_slice_ld(n) BF16.
int tc_slice_ld(int n);
size_t tc_slice_plane(int n);
int tc_num_slices();
// Row exponents and slices of Q (column-major FP64).  rmax: n u64 scratch.
cudaError_t launch_slice_q(int n, const double* Q, unsigned long long* rmax, int* erow,
                           __nv_bfloat16* Qs, const DevStatus* st, cudaStream_t s);
// Column exponents f_r and slices of the m columns of a column-major n x m W
// (as rows of W^T: Ws holds tc_num_slices() planes of m x tc_slice_ld(n)).
cudaError_t launch_slice_cols(int n, int m, const double* W, int* fcol, __nv_bfloat16* Ws, cudaStream_t s);
// X (column-major, ldx; n x ncols) = 2^(e_i+f_r-16) sum_{p+q<=6} Qs_p Ws_q^T,
// ncols = n when negative.  err: status word that receives ST_TIMEOUT if a
// bounded wait gave up.
cudaError_t launch_gemm_tc(int n, const __nv_bfloat16* Qs, const __nv_bfloat16* Ws, const int* erow,
                           const int* fcol, double* X, int ldx, const DevStatus* st, int* err,
                           cudaStream_t s, int ncols = -1);
// Grouped versions over a table of updates.  Host-side prefix arrays (count+1)
// of per-update work: row blocks of 256 (rowmax), 32x32 slice tiles, 128x128
// GEMM tiles.  maps: device array of 2*count tensor maps (Q slices, W slices)
// built by tc_encode_maps.
cudaError_t launch_slice_q_grouped(const ProbDesc* P, int count, const int* rb_prefix, int total_rb,
                                   const int* tile_prefix, int total_tiles, cudaStream_t s);
int tc_encode_map(void* map64, const void* base, int n);  // 0 on success
cudaError_t launch_gemm_tc_grouped(const ProbDesc* P, int count, const void* maps, const int* tile_prefix,
                                   int total_tiles, cudaStream_t s);
// The non-zero map (ProbDesc::wnz) of every update's W slices, one CTA per
// 128 x 128 GEMM tile (tile_prefix as for the GEMM).
cudaError_t launch_wnz_scan_grouped(const ProbDesc* P, int count, const int* tile_prefix, int total_tiles,
                                    cudaStream_t s);
cudaError_t launch_gemm_f64_grouped(const ProbDesc* P, int count, const int* tile_prefix, int total_tiles,
                                    cudaStream_t s);
// X -> Q copy-back for in-place updates; elem_prefix: prefix of n*n (device).
cudaError_t launch_copyback_grouped(const ProbDesc* P, int count, const long long* elem_prefix,
                                    long long total, cudaStream_t s);

}  // namespace eig
