/*
 * eig_update.h -- C ABI of the GB300 (sm_103a) rank-k symmetric eigen-update.
 *
 * Problem (Oh & Hu, "Multiple-rank Modification of Symmetric Eigenvalue
 * Problem", arXiv 1706.00773, Sec. 2.1): a symmetric A = Q diag(lambda) Q^T is
 * known; a symmetric low-rank perturbation K Sigma K^T is added
 * (Sigma = diag(sigma), sigma_c = +1 or -1; the PSD case K K^T has every
 * sigma_c = +1).  The library returns the eigenpairs of A' = A + K Sigma K^T:
 *   U = Q^T K                                   (Sec. 2.1, below eq. (1))
 *   mu = roots of f(x) = det(I - Sigma U^T (xI - Lambda)^{-1} U)   (eq. (1))
 *        located by the root count of Sec. 2.2 and refined by the zero finder
 *        of Sec. 2.3
 *   X = Q W,  W[:,r] = (Lambda - mu_r I)^{-1} U alpha_r / |.|   (Sec. 2.4, eq. (10))
 *
 * Conventions shared by every entry point
 *   - Matrices are column-major FP64 in device memory.  Q is n x n with
 *     eigenvectors as columns; K is n x k; U is n x k.
 *   - lambda is ascending on input and on output (EIG_EINVAL otherwise).
 *   - sigma is a HOST array of k int8 (+1/-1); NULL means all +1.
 *   - Streams are cudaStream_t passed as void* (NULL = legacy default stream).
 *   - Return value 0 = success, negative EIG_E* codes otherwise.  No C++
 *     exception crosses this boundary.
 *   - Device arrays passed in are owned by the caller; the library never frees
 *     them.  The handle owns its workspace (device memory, grown on demand and
 *     freed by eig_update_destroy).
 *   - A handle is not thread-safe: one host thread at a time, except
 *     eig_update_query, which may be called concurrently.
 */
#ifndef EIG_UPDATE_H_
#define EIG_UPDATE_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define EIG_OK 0
#define EIG_EINVAL (-1)   /* bad argument: n<1, k<1, k>EIG_MAX_K, NULL pointer,
                             unsorted lambda, non-finite input, bad sigma */
#define EIG_ENOMEM (-2)   /* workspace allocation failed or hbm_budget exceeded */
#define EIG_ENOTCONV (-3) /* a root hit the iteration cap; results are still
                             written and the report counts the roots */
#define EIG_ETIMEOUT (-4) /* a bounded device wait gave up */
#define EIG_ECUDA (-5)    /* a CUDA runtime call failed */
#define EIG_ENOTSUP (-6)  /* valid request this build does not implement */
#define EIG_EBUSY (-7)    /* ticket not finished yet (eig_update_query) */
#define EIG_ETOOBIG (-8)  /* problem larger than eig_secular_values_static's
                             fixed scratch holds (n > EIG_STATIC_MAX_N), or
                             more selected pairs than eig_update_select's
                             output holds (max_m) */

#define EIG_MAX_K 16      /* largest rank this build accepts */

/* ---- precision modes (eig_init_params.mode) ----------------------------- */
#define EIG_FP64 0u  /* every step in FP64 on the CUDA cores */
#define EIG_MIXED 1u /* U = Q^T K and the eq. (10) entries of W in
                        double-float arithmetic (pairs of FP32, a few units
                        of 2^-48; values outside that range in FP64); pole
                        counts and the zero finder's coarse steps on FP32
                        sums, taken only where an error bound certifies them,
                        every root finished in FP64; X = Q W as split-BF16
                        products on the tensor cores with exact FP32 chunks
                        and double-float accumulation */

/* ---- what to compute (eig_problem.want) --------------------------------- */
#define EIG_VALUES 1u  /* eigenvalues into lambda */
#define EIG_VECTORS 2u /* eigenvectors into Q (or Q_out) */
#define EIG_REPORT 4u  /* fill the report's residual / orthogonality checks
                          (sampled, FP64) */
#define EIG_ASYNC 8u   /* do not synchronise at the end; the status is then
                          read with eig_update_query(EIG_Q_LAST_STATUS) */

typedef struct eig_ctx* eig_handle;

typedef struct {
  int32_t device;      /* CUDA device ordinal */
  uint32_t mode;       /* EIG_FP64 or EIG_MIXED */
  uint64_t hbm_budget; /* max bytes of workspace the handle may hold; 0 = no limit */
  int32_t max_iter;    /* per-root iteration cap of the zero finder; 0 = 128 */
  uint32_t flags;      /* 0 or EIG_TUNE */
} eig_init_params;

/* eig_init_params.flags: tune the launch schedule of eig_update_batch.  The
   first batch of each signature (mode, vectors or not, and per padded rank
   the number of updates and their total size, in powers of two) times the
   candidate schedules -- rank classes in sequence or overlapped on one stream
   each, multi-root pole intervals first or natural root order, the zero
   finder's persistent grid at full or half residency -- on a values-only copy
   of the batch (the caller's data is not touched; a few extra passes of the
   secular stages), keeps the fastest, and reuses it for later batches of that
   signature.  Results are identical under every schedule.  With the
   environment variable EIG_TUNE_CACHE naming a file, the choices are read
   from it at eig_update_init and appended to it as they are made, so a later
   process starts tuned.  eig_update_rank_k and the serving engine keep the
   default schedule. */
#define EIG_TUNE 1u

typedef struct {
  int64_t n;           /* size, >= 1 */
  int32_t k;           /* rank, 1..EIG_MAX_K */
  int32_t pad_;
  double* Q;           /* device n x n; in: old eigenvectors; out: new ones
                          unless Q_out is given */
  double* lambda;      /* device n; in: old eigenvalues ascending; out: new */
  const double* K;     /* device n x k */
  const int8_t* sigma; /* host k entries of +1/-1, NULL = all +1 */
  double* Q_out;       /* device n x n output for the eigenvectors, or NULL */
  uint32_t want;       /* EIG_VALUES | EIG_VECTORS | EIG_REPORT | EIG_ASYNC */
  uint32_t pad2_;
  double* errors;      /* device n x 4 (column-major, ld n) per-eigenpair error
                          report, or NULL; filled when want has EIG_VECTORS.
                          Row r belongs to the r-th new eigenpair (ascending):
                            [r, 0] |(A' - mu_r) x_r|_2 / |A|, the residual of
                                   the FP64 eq. (10) vector in the old
                                   eigenbasis, (Lambda + U Sigma U^T - mu_r) w_r
                                   with w_r unit (Sec. 3 metric (B) per pair;
                                   deflated pairs: the bound |U|_F |u_i| / |A|);
                            [r, 1] |rho_r - mu_r| / |A|, rho_r = w_r^T A' w_r
                                   the Rayleigh quotient in FP64;
                            [r, 2] min_{s != r} |mu_r - mu_s| / |A|;
                            [r, 3] |w_r^T w_{r+1}| with the next secular root's
                                   vector when that gap is below 1e-6 |A|
                                   (Sec. 3 metric (C) where it is at risk), else 0.
                          |A| = max|lambda_old| + |U|_F^2 (report.norm_A).  X = Q W
                          adds the GEMM's own error on top (EIG_MIXED: the
                          split-BF16 representation, <= 2^-41 per factor entry
                          relative to its row / column maximum). */
} eig_problem;

typedef struct {
  int64_t n;            /* problem size */
  int64_t n_deflated;   /* pairs kept unchanged (|u_i| below the deflation bound) */
  int64_t iters_total;  /* zero-finder FP64 evaluations summed over roots */
  int64_t n_notconv;    /* roots that hit the iteration cap */
  int32_t k;
  int32_t status;       /* final status of this update */
  int32_t iters_max;    /* largest per-root evaluation count */
  int32_t n_checked;    /* eigenpairs sampled for the two norms below */
  double max_residual;  /* max |A' x - mu x|_2 over the sampled pairs */
  double max_orth;      /* max |x_i^T x_j - delta_ij| over the sampled pairs */
  double norm_A;        /* max |lambda_old| + |U|_F^2, the scale of A' */
  double ms_total;      /* device time of the update (CUDA events), ms */
  /* Device time per stage (CUDA events on the caller's stream), ms: */
  double ms_project;    /* U = Q^T K */
  double ms_deflate;    /* deflation and compaction */
  double ms_counts;     /* root count at every pole */
  double ms_roots;      /* zero finder, every root */
  double ms_assemble;   /* eq. (10) columns of W, new eigenvalues */
  double ms_slice;      /* EIG_MIXED: BF16 digit slices of Q (0 in EIG_FP64) */
  double ms_gemm;       /* X = Q W */
  int32_t launches;     /* kernels this update launched */
  int32_t n_runs;       /* runs of exactly equal old eigenvalues, each rotated
                           inside its eigenspace before deflation so that at
                           most k of its rows stay in the secular problem */
  int64_t iters32_total; /* EIG_MIXED: coarse FP32 evaluations of the zero finder
                            (iters_total counts the FP64 ones) */
  int64_t redo32_total;  /* EIG_MIXED: FP32 evaluations whose root count the
                            error bound could not certify (redone in FP64) */
  int64_t taylor_total;  /* evaluations taken by a first-order update of the
                            k x k sums after a tiny Newton step (no pass over
                            the terms) */
  double max_pair_residual; /* with eig_problem.errors: max of its columns 0, */
  double max_pair_rayleigh; /* 1 and 3 over every eigenpair (0 without) */
  double max_pair_orth;
  int64_t tc_pair_tiles;    /* EIG_MIXED full update with vectors: 128 x 128 x 32
                               BF16 slice-pair products the tcgen05 GEMM issued
                               (2 * 128 * 128 * 32 flops each): 15 per output
                               tile and 32-deep step, less the pairs against
                               all-zero tiles of W's two leading slices, which
                               it skips (their products are exactly zero).
                               0 where that GEMM did not run. */
  int64_t asm_fp64_cols;    /* EIG_MIXED with vectors: columns of W whose eq. (10)
                               entries were formed in FP64 instead of the
                               double-float path: those asking for
                               eig_problem.errors, those of a sub-problem above
                               8192 rows, and those whose values leave the
                               double-float range (magnitudes outside
                               [2^-60, 2^60]).  0 otherwise. */
  int64_t gj32_total;       /* EIG_MIXED: certified FP32 evaluations whose k x k
                               step was a Gauss-Jordan inverse of the bordered
                               matrix (one root in the bracket: the count from
                               the sign of its determinant); the other counted
                               FP32 evaluations took its eigen-decomposition. */
} eig_report;

/* ---- lifetime ----------------------------------------------------------- */

/* Create a handle on params->device.  params may be NULL (device 0, FP64,
   no budget).  On success *out holds the handle.  EIG_EINVAL on bad params,
   EIG_ECUDA if the device cannot be used. */
int eig_update_init(const eig_init_params* params, eig_handle* out);

/* Free the handle's workspace and the handle.  NULL is accepted. */
int eig_update_destroy(eig_handle h);

/* ---- one update ---------------------------------------------------------
 * Rank-k update of one decomposition (Sec. 2.1-2.4): U = Q^T K, deflation of
 * rows of U below the bound, root count at every pole, safeguarded Newton /
 * bisection per root, eq. (10) eigenvector coefficients, X = Q W.  On return
 * lambda holds the new eigenvalues ascending and Q (or Q_out) the matching
 * eigenvectors.  Q_out, if given, must not alias Q.  Stream-ordered on
 * `stream`; unless want has EIG_ASYNC the call synchronises the stream before
 * returning and returns the final status.  rep (host, may be NULL) receives
 * the report.  Errors: EIG_EINVAL (arguments, unsorted or non-finite lambda),
 * EIG_ENOMEM, EIG_ENOTCONV (results written, some roots capped), EIG_ECUDA. */
int eig_update_rank_k(eig_handle h, eig_problem* prob, eig_report* rep, void* stream);

/* ---- many updates ---------------------------------------------------------
 * Enqueue `count` independent updates (different n and k allowed) and return
 * one ticket per problem in tickets[] (host).  The problems of one call form
 * one table (two when some want eigenvectors and some do not), and every
 * stage runs as one grouped launch over all of them.  Asynchronous: poll with
 * eig_update_query(EIG_Q_STATUS / EIG_Q_REPORT).  The problem arrays must stay
 * valid until their tickets complete.  A ticket holds host resources until
 * eig_update_release (or eig_update_destroy); its id is never reused. */
int eig_update_batch(eig_handle h, int32_t count, eig_problem* probs, uint64_t* tickets,
                     void* stream);

/* Release a finished ticket of eig_update_batch: its status is folded into the
 * EIG_Q_METRICS counters and the id becomes invalid (EIG_EINVAL from then on).
 * The pinned status block and event of a batch call are freed with the last of
 * its tickets.  Returns EIG_OK, EIG_EBUSY (still running: nothing released) or
 * EIG_EINVAL (unknown or already released id). */
int eig_update_release(eig_handle h, uint64_t ticket);

/* ---- queries --------------------------------------------------------------
 * what = EIG_Q_STATUS:      in = const uint64_t* ticket, out = int32_t* status
 *                           (EIG_EBUSY while running; the return value is the
 *                           same code)
 * what = EIG_Q_REPORT:      in = const uint64_t* ticket, out = eig_report*
 * what = EIG_Q_LAST_STATUS: in = NULL, out = int32_t* (synchronises the handle's
 *                           last stream first)
 * what = EIG_Q_COUNT:       in = const eig_count_args*, out = NULL.  Root count
 *                           #{mu < x_j} of diag(lambda) + U Sigma U^T at device
 *                           points (the location sub-problem, Sec. 2.2), taken
 *                           in FP64 in both modes (the mixed path's certified
 *                           FP32 counts run at poles: eig_pole_counts);
 *                           synchronous.
 * what = EIG_Q_WORKSPACE:   in = const eig_problem*, out = uint64_t* bytes the
 *                           handle needs for that problem.
 * what = EIG_Q_METRICS:     in = NULL, out = eig_metrics*: the handle's
 *                           counters since eig_update_init (host-side, no
 *                           device synchronisation; batch tickets still running
 *                           count as pending).
 * out_bytes is the size of *out; EIG_EINVAL if too small. */
#define EIG_Q_STATUS 1
#define EIG_Q_REPORT 2
#define EIG_Q_LAST_STATUS 3
#define EIG_Q_COUNT 4
#define EIG_Q_WORKSPACE 5
#define EIG_Q_METRICS 6

typedef struct {
  int64_t calls;            /* eig_update_rank_k and eig_update_batch calls */
  int64_t updates;          /* problems submitted (each problem of a batch) */
  int64_t eigenpairs;       /* sum of n over the problems submitted */
  int64_t updates_ok;       /* finished with EIG_OK */
  int64_t updates_failed;   /* finished or rejected with an error status
                               (EIG_ENOTCONV included) */
  int64_t updates_pending;  /* submitted, final status not read yet (an
                               EIG_ASYNC update stays here when another
                               update starts before EIG_Q_LAST_STATUS) */
  int64_t launches;         /* kernels launched by the update paths */
  int64_t workspace_allocs; /* workspace (re)allocations */
  uint64_t workspace_bytes; /* current workspace size */
  int64_t tune_trials;      /* EIG_TUNE: schedules timed by the batch tuner */
  int64_t tune_hits;        /* EIG_TUNE: batch tables that reused a tuned schedule */
} eig_metrics;

typedef struct {
  int64_t n;             /* size of the (already projected) problem */
  int32_t k;
  int32_t npts;          /* number of evaluation points */
  const double* lambda;  /* device n, ascending */
  const double* U;       /* device n x k (column-major) */
  const int8_t* sigma;   /* host k, NULL = all +1 */
  const double* x;       /* device npts points */
  int32_t* counts;       /* device npts output: #{mu < x_j} (at a pole: the
                            limit from the left) */
  void* stream;
} eig_count_args;

int eig_update_query(eig_handle h, int32_t what, const void* in, void* out, size_t out_bytes);

/* ---- stage entry points (for callers that hold U already) ----------------- */

/* U = Q^T K (Sec. 2.1).  Q n x n, K n x k, U n x k, all device, column-major.
   Uses the handle's mode for the arithmetic (FP64 only in this build). */
int eig_project(eig_handle h, int64_t n, int32_t k, const double* Q, const double* K, double* U,
                void* stream);

/* Eigenvalues of diag(lambda) + U Sigma U^T (Sec. 2.2-2.3) without vectors:
   mu (device n, ascending) receives them; iters (device int32 n, may be NULL)
   the evaluations each root took (0 for deflated pairs).  U is read only: runs
   of exactly equal lambda are rotated in a workspace copy.  Synchronous. */
int eig_secular_values(eig_handle h, int64_t n, int32_t k, const double* lambda, const double* U,
                       const int8_t* sigma, double* mu, int32_t* iters, void* stream);

/* Root counts at the poles (Sec. 2.2, location sub-problem), exactly as the
   update computes them in the handle's mode.  Input as eig_secular_values
   (device lambda ascending, device U n x k column-major, host sigma).  Runs of
   equal lambda are rotated in a workspace copy of U and small rows deflated
   (the update's own rule); the n' kept poles lambda'_0 < ... < lambda'_{n'-1}
   form the sub-problem, and for every kept pole q:
     counts[q]   = #{mu' < lambda'_q} of diag(lambda') + U' Sigma U'^T (the
                   limit from the left), the count the zero finder uses;
     counts32[q] = EIG_MIXED: the certified FP32 pass's count, or -1 where its
                   error bound could not certify it and the FP64 recount
                   decided; EIG_FP64: -1 (there is no FP32 pass);
     idx_keep[q] = the row of lambda / U that kept pole q came from.
   counts, counts32 and idx_keep are device int32 arrays of n entries (the last
   two may be NULL); entries q >= n' are left unspecified.  *n_keep (host)
   receives n'.  Synchronous.  EIG_EINVAL for bad arguments or unsorted /
   non-finite input (*n_keep = 0, outputs unspecified). */
int eig_pole_counts(eig_handle h, int64_t n, int32_t k, const double* lambda, const double* U,
                    const int8_t* sigma, int32_t* counts, int32_t* counts32, int32_t* idx_keep,
                    int64_t* n_keep, void* stream);

/* ---- eigenvalues without any device allocation ---------------------------
 * The paper has no counterpart to this entry point.  It serves callers that
 * cannot allocate device memory: code whose HBM is owned by another memory
 * manager (a framework's caching allocator, a serving process that reserves
 * memory up front) and latency-critical loops that cannot absorb a
 * cudaMalloc/cudaFree (cudaFree synchronises the device).  It computes what
 * eig_secular_values computes, for n <= EIG_STATIC_MAX_N and k <= EIG_MAX_K,
 * with every temporary in one fixed 6 MiB device array that the library
 * defines at file scope; the caller passes inputs and outputs only, and no
 * handle is needed.  Larger problems return EIG_ETOOBIG.
 *   - Every GPU that loads the library holds that array until the process exits.
 *   - All calls share the array: calls whose work overlaps on the GPU (two
 *     streams or two host threads at once) race and give wrong results.
 *   - The first call on a device looks up the array's device address (set-up,
 *     with that device current); make that first call before any stream capture.
 *     The address is kept with the device's context: after cudaDeviceReset the
 *     next call on that device does the set-up again.
 * Arguments as eig_secular_values (device lambda, U, mu, iters; host sigma),
 * plus max_iter (0 = 128).  Synchronises `stream` before returning. */
#define EIG_STATIC_MAX_N 8192
int eig_secular_values_static(int64_t n, int32_t k, const double* lambda, const double* U,
                              const int8_t* sigma, double* mu, int32_t* iters, int32_t max_iter,
                              void* stream);

/* ---- serving: resident decompositions, continuous batching -----------------
 * A server keeps decompositions (Q, lambda) resident on the device and applies
 * rank-k update requests to them in order (chained updates).  Requests carry
 * K on the host; eig_server_poll reaps finished batches and admits pending
 * requests into new batches whenever a batch slot (stream + workspace of
 * hbm_budget / slots bytes) is free: at most one request per resident per
 * batch (so a chain stays ordered), as many as fit the slot's workspace.
 * Batches on different slots overlap on the device.  Every batch is one
 * grouped eig_update_batch-style launch sequence; each result is identical to
 * the same update applied alone.  Not thread-safe: one host thread drives a
 * server. */
typedef struct eig_srv* eig_server;

typedef struct {
  int32_t device;
  uint32_t mode;        /* EIG_FP64 or EIG_MIXED */
  uint64_t hbm_budget;  /* workspace bytes over all slots; 0 = 8 GiB */
  int32_t slots;        /* batches in flight; 0 = 2 */
  int32_t max_batch;    /* requests per batch; 0 = 64 */
} eig_server_params;

typedef struct {
  int32_t status;       /* EIG_EBUSY while queued or running */
  int32_t resident;
  int32_t k;
  int32_t batch_size;   /* requests in the batch that carried it */
  double submit_ms;     /* host clock, ms since the server was created */
  double launch_ms;
  double done_ms;       /* when eig_server_poll saw the batch finish */
} eig_request_info;

int eig_server_create(const eig_server_params* params, eig_server* out);
int eig_server_destroy(eig_server srv);
/* Register a resident decomposition: device Q (n x n, column-major) and lambda
   (n, ascending), owned by the caller and updated in place by every request. */
int eig_server_add_resident(eig_server srv, int64_t n, double* Q, double* lambda, int32_t* id);
/* Queue a rank-k update of resident `id`: K (host, n x k column-major) and
   sigma (host, NULL = all +1) are copied at submit.  Returns a ticket. */
int eig_server_submit(eig_server srv, int32_t id, int32_t k, const double* K, const int8_t* sigma,
                      uint64_t* ticket);
/* Reap finished batches and launch new ones; waits up to wait_us for one
   batch to finish when nothing can be launched.  Returns the number of
   requests completed by this call (>= 0) or an EIG_E* code. */
int eig_server_poll(eig_server srv, int32_t wait_us);
int eig_server_query(eig_server srv, uint64_t ticket, eig_request_info* out);
/* Requests still queued or running. */
int eig_server_pending(eig_server srv);

/* Sec. 2.2 Steps 1-2: write K = [(e_j + a)/sqrt(2), (e_j - a)/sqrt(2)] (device
   n x 2) and sigma = {+1, -1} (host) so that K Sigma K^T = e_j a^T + a e_j^T.
   a is device n.  Stream-ordered. */
int eig_make_rank2(int64_t n, int64_t j, const double* a, double* K, int8_t* sigma, void* stream);

/* Sec. 2.2, eq. (3) and Algorithms 1a-1c: the location vector of a rank-2
   update diag(lambda) + U Sigma U^T.  lambda (device n, strictly ascending:
   deflated, distinct poles), U (device n x 2, column-major), sigma (host 2
   entries of +1/-1; NULL = {+1, +1}).  Writes alpha (device n) = the residues
   of f(x) = 1 + sum_i alpha_i / (lambda_i - x), and L (device int32 n+1):
   L[0] roots below lambda_0, L[i] roots in (lambda_{i-1}, lambda_i), L[n]
   roots above lambda_{n-1}.  Both sigma > 0 scans from the left (1a), both
   < 0 from the right (1b), opposite signs from the left after placing 0 or 1
   root below lambda_0 by the sign of alpha_0 (1c, with the bound of at most
   i+1 roots below lambda_i).  The roots are counted from residue signs only,
   so a residue that rounds to the wrong sign (a pole that nearly deflates)
   misplaces roots: the inertia count of eig_update_query(EIG_Q_COUNT) has no
   such limit.  O(n^2) work.  Stream-ordered; the caller owns every buffer.
   EIG_EINVAL for n < 2, NULL buffers or sigma entries other than +1/-1. */
int eig_location_rank2(int64_t n, const double* lambda, const double* U, const int8_t* sigma,
                       double* alpha, int32_t* L, void* stream);

/* Sec. 3, eq. (11): the first-order perturbation estimate the paper compares
   against for a small K.  With U = Q^T K (u_j its rows):
     mu_j = lambda_j + u_j^T Sigma u_j,
     X    = Q W,  W_jj = 1,  W_ij = u_i^T Sigma u_j / (lambda_j - lambda_i)  (i != j),
   with W_ij = 0 where lambda_i == lambda_j.  mu_j pairs with column j of X;
   nothing is sorted or normalised.  Its error grows as |K|^4 (it is exact only to
   first order): use it as the comparison the paper draws, not as an update.
   Q (device n x n), lambda (device n), K (device n x k, k <= EIG_MAX_K), all
   column-major; sigma host k entries of +1/-1 or NULL (all +1).  mu (device n)
   may be lambda itself; X (device n x n) must not be Q.  X = Q W runs in the
   handle's mode (FP64, or the split-BF16 tensor-core product in EIG_MIXED).
   Uses the handle's workspace (n^2 doubles, plus slices in EIG_MIXED).
   Synchronous on `stream`.  EIG_EINVAL for bad sizes, pointers or sigma,
   EIG_ENOMEM when the workspace cannot grow, EIG_ETIMEOUT when a bounded
   device wait gave up. */
int eig_perturbation(eig_handle h, int64_t n, int32_t k, const double* Q, const double* lambda,
                     const double* K, const int8_t* sigma, double* mu, double* X, void* stream);

/* Sec. 2.1 (only the eigenvalues of an interval) and Sec. 3 (a subset of the
   eigenvectors): the eigenpairs of A' = Q diag(lambda) Q^T + K Sigma K^T whose
   eigenvalues lie in [vl, vu), without the others.  Two counts give the
   secular roots in the interval, the zero finder solves only those (pole
   counts only at the poles around the interval), deflated pairs in the
   interval are merged in, and X = Q W_sel (n x m) is formed like the full
   update's X: the FP64 GEMM in EIG_FP64, split-BF16 tensor-core products in
   EIG_MIXED.  Q, lambda, K are read, not modified.
   Q (device n x n), lambda (device n, ascending), K (device n x k), all
   column-major; sigma host k entries or NULL.  mu (device max_m) receives the
   m selected eigenvalues, ascending; X (device n x max_m, column-major, may
   be NULL for values only) their unit eigenvectors (sign: largest entry of W's
   column positive).  *m_out = m.  If m > max_m nothing is written and the
   call returns EIG_ETOOBIG with *m_out = m (size the buffers and call again).
   vl < vu required (use +-HUGE_VAL for half-open intervals).  Uses the
   handle's workspace; synchronous on `stream`.  EIG_EINVAL / EIG_ENOMEM /
   EIG_ENOTCONV / EIG_ETIMEOUT as eig_update_rank_k. */
int eig_update_select(eig_handle h, int64_t n, int32_t k, const double* Q, const double* lambda,
                      const double* K, const int8_t* sigma, double vl, double vu, int64_t max_m,
                      double* mu, double* X, int64_t* m_out, void* stream);

/* ---- measurement -----------------------------------------------------------
 * FP64 FMA throughput of `device`, the denominator of the FP64-pipe rooflines
 * (the zero finder, pole counts, assembly and the FP64 GEMM are bound by that
 * pipe).  The paper has no counterpart: it is a measurement of the machine.
 * Runs a kernel of independent FMA chains (no memory traffic) on every SM,
 * `reps` timed launches (CUDA events on `stream`) after one warm-up, and
 * writes the best rate to *gflops as 2 x FMAs / s / 1e9.  About 10-20 ms per
 * launch.  Synchronous.  EIG_EINVAL for reps < 1 or a NULL output, EIG_ECUDA
 * if the device cannot be used. */
int eig_fp64_fma_rate(int32_t device, int32_t reps, double* gflops, void* stream);

/* ---- diagnostics -----------------------------------------------------------
 * The CUDA runtime error behind the calling thread's most recent EIG_ECUDA
 * from a checked stream-ordered call (0 if there was none; later successful
 * calls do not clear it).  When msg is not NULL and len > 0, writes at most
 * len bytes, NUL-terminated: the error's name and description and the call
 * that returned it ("" if none).  Returns the cudaError_t value.  Never
 * touches the device. */
int eig_last_cuda_error(char* msg, int32_t len);

/* Library version string (static storage). */
const char* eig_version(void);

#ifdef __cplusplus
}
#endif
#endif /* EIG_UPDATE_H_ */
