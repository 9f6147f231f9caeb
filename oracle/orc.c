/*
 * orc.c -- plain, slow CPU FP64 oracle for the rank-k modification of a
 * symmetric eigendecomposition (Oh & Hu, "Multiple-rank Modification of
 * Symmetric Eigenvalue Problem", arXiv 1706.00773).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header or table with the CUDA
 * path.
 *
 * Problem (Sec. 2.1): A = Q diag(lam) Q^T is known; A' = A + K Sigma K^T with
 * Sigma = diag(sigma), sigma_c in {+1,-1}.  In the eigenbasis the update is
 * diag(lam) + U Sigma U^T with U = Q^T K (the matrix L of Sec. 2.4).
 *
 * Layouts: every matrix is column-major FP64; U is n x k, row i of U is u_i.
 *
 * What each routine follows:
 *  - orc_jacobi: plain cyclic two-sided Jacobi (the textbook definition of a
 *    symmetric eigendecomposition), used both for dense A' (the "direct EVD"
 *    comparison system of Sec. 3) and for the k x k matrices below.
 *  - orc_count: the root-count sub-problem of Sec. 2.1/2.2.  The modified
 *    Sturm count of Sec. 2.2 (eqs. 4-6) delivers #{mu < x}; here that same
 *    integer is obtained from Sylvester's law of inertia applied to the bordered
 *    matrix [[diag(lam) - xI, U], [U^T, -Sigma]] (Haynsworth):
 *        #{mu < x} = #{lam_i < x} + neg(M(x) - Sigma) - k_plus,
 *        M(x) = sum_i u_i u_i^T / (x - lam_i)   (k x k),
 *    where neg() counts negative eigenvalues (k x k Jacobi).  M(x) is the
 *    k x k matrix inside the determinant of eq. (1):
 *        f(x) = det(I - Sigma U^T (xI - Lambda)^{-1} U) = det(Sigma) det(Sigma - M(x)).
 *  - orc_roots: the root-value sub-problem, Sec. 2.3 Divide-and-Conquer zero
 *    finder with m = 1 point (bisection), the side test taken from the count
 *    above, starting from the Courant-Weyl interlacing brackets of Sec. 2.2
 *    generalised to lam_{m-k_minus} <= mu_m <= lam_{m+k_plus}.  After the
 *    absolute bracket is tight the search continues in coordinates shifted to
 *    the nearest pole (x = lam_o + tau) so that tau = mu - lam_o keeps full
 *    relative accuracy.
 *  - orc_vectors: eigenvector update of Sec. 2.4 / eq. (10): alpha_0 spans the
 *    null space of the k x k matrix Sigma - M(mu) (eigenvector of the
 *    eigenvalue nearest zero), w_i = (u_i^T alpha_0) / (lam_i - mu), then
 *    w / ||w||.
 */
#include <float.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EPS DBL_EPSILON
#define IX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

enum {
  ORC_OK = 0,
  ORC_EINVAL = -1,
  ORC_ENOMEM = -2,
  ORC_FLAG_CAP = 1,      /* bisection hit the iteration cap */
  ORC_FLAG_AT_POLE = 2,  /* root coincides with a pole: eq. (10) undefined */
};

/* ------------------------------------------------------------------------ */
/* Cyclic Jacobi eigendecomposition of a symmetric n x n matrix.             */
/* A is overwritten.  w receives eigenvalues ascending; V (may be NULL)      */
/* receives the matching orthonormal eigenvectors as columns.                */
/* ------------------------------------------------------------------------ */
int orc_jacobi(int n, double* A, double* w, double* V, int max_sweeps) {
  if (n < 1 || !A || !w) return ORC_EINVAL;
  if (V) {
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) V[IX(i, j, n)] = (i == j) ? 1.0 : 0.0;
  }
  double fro = 0.0;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) fro += A[IX(i, j, n)] * A[IX(i, j, n)];
  fro = sqrt(fro);
  int sweep;
  for (sweep = 0; sweep < max_sweeps; ++sweep) {
    double off = 0.0;
    for (int q = 1; q < n; ++q)
      for (int p = 0; p < q; ++p) off += A[IX(p, q, n)] * A[IX(p, q, n)];
    off = sqrt(2.0 * off);
    if (off <= 1e-17 * fro || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        double apq = A[IX(p, q, n)];
        if (apq == 0.0) continue;
        double app = A[IX(p, p, n)], aqq = A[IX(q, q, n)];
        /* Entry already negligible next to both diagonals: drop it. */
        if (sweep > 3 && fabs(apq) * 1e18 < fabs(app) && fabs(apq) * 1e18 < fabs(aqq)) {
          A[IX(p, q, n)] = 0.0;
          A[IX(q, p, n)] = 0.0;
          continue;
        }
        /* 2x2 symmetric Schur decomposition: tan of the rotation angle is the
           smaller root of t^2 + 2 theta t - 1 = 0. */
        double theta = (aqq - app) / (2.0 * apq);
        double t;
        if (fabs(theta) > 1e150) {
          t = 0.5 / theta;
        } else {
          t = 1.0 / (fabs(theta) + sqrt(1.0 + theta * theta));
          if (theta < 0.0) t = -t;
        }
        double c = 1.0 / sqrt(1.0 + t * t);
        double s = t * c;
        for (int r = 0; r < n; ++r) {
          if (r == p || r == q) continue;
          double arp = A[IX(r, p, n)], arq = A[IX(r, q, n)];
          double nrp = c * arp - s * arq;
          double nrq = s * arp + c * arq;
          A[IX(r, p, n)] = nrp;
          A[IX(p, r, n)] = nrp;
          A[IX(r, q, n)] = nrq;
          A[IX(q, r, n)] = nrq;
        }
        A[IX(p, p, n)] = app - t * apq;
        A[IX(q, q, n)] = aqq + t * apq;
        A[IX(p, q, n)] = 0.0;
        A[IX(q, p, n)] = 0.0;
        if (V) {
          for (int r = 0; r < n; ++r) {
            double vrp = V[IX(r, p, n)], vrq = V[IX(r, q, n)];
            V[IX(r, p, n)] = c * vrp - s * vrq;
            V[IX(r, q, n)] = s * vrp + c * vrq;
          }
        }
      }
    }
  }
  for (int i = 0; i < n; ++i) w[i] = A[IX(i, i, n)];
  /* Selection sort, ascending, carrying the vectors along. */
  for (int i = 0; i < n - 1; ++i) {
    int m = i;
    for (int j = i + 1; j < n; ++j)
      if (w[j] < w[m]) m = j;
    if (m != i) {
      double tmp = w[i];
      w[i] = w[m];
      w[m] = tmp;
      if (V) {
        for (int r = 0; r < n; ++r) {
          double tv = V[IX(r, i, n)];
          V[IX(r, i, n)] = V[IX(r, m, n)];
          V[IX(r, m, n)] = tv;
        }
      }
    }
  }
  return sweep;
}

/* ------------------------------------------------------------------------ */
/* Secular building blocks.  The evaluation point is x = lam[o] + tau when   */
/* o >= 0 and x = tau when o < 0; the differences x - lam_i are formed as    */
/* tau - (lam_i - lam_o) so that they keep full relative accuracy near the   */
/* origin pole.                                                              */
/* ------------------------------------------------------------------------ */
static inline double diff_at(const double* lam, int64_t i, int64_t o, double tau) {
  return (o >= 0) ? tau - (lam[i] - lam[o]) : tau - lam[i];
}

/* Fill Mk (k x k, col-major) with M(x) = sum_i u_i u_i^T / (x - lam_i) and
   return #{lam_i < x}; returns -1 if x coincides with a pole. */
static int64_t build_M(int64_t n, int k, const double* lam, const double* U, int64_t o,
                       double tau, double* Mk) {
  memset(Mk, 0, sizeof(double) * (size_t)k * (size_t)k);
  int64_t below = 0;
  for (int64_t i = 0; i < n; ++i) {
    double d = diff_at(lam, i, o, tau);
    if (d == 0.0) return -1;
    if (d > 0.0) ++below;
    double r = 1.0 / d;
    for (int b = 0; b < k; ++b) {
      double ub = U[IX(i, b, n)] * r;
      for (int a = 0; a < k; ++a) Mk[IX(a, b, k)] += U[IX(i, a, n)] * ub;
    }
  }
  return below;
}

static int kplus_of(int k, const int8_t* sigma) {
  int kp = 0;
  for (int c = 0; c < k; ++c) kp += (sigma[c] > 0);
  return kp;
}

/* #{mu < x}; -1 if x is a pole.  work: 3*k*k doubles. */
static int64_t count_impl(int64_t n, int k, const double* lam, const double* U,
                          const int8_t* sigma, int64_t o, double tau, double* work) {
  double* Mk = work;
  double* ev = work + (size_t)k * k;
  int64_t below = build_M(n, k, lam, U, o, tau, Mk);
  if (below < 0) return -1;
  for (int c = 0; c < k; ++c) Mk[IX(c, c, k)] -= (double)sigma[c];
  orc_jacobi(k, Mk, ev, NULL, 60);
  int neg = 0;
  for (int c = 0; c < k; ++c) neg += (ev[c] < 0.0);
  return below + neg - kplus_of(k, sigma);
}

int64_t orc_count(int64_t n, int k, const double* lam, const double* U, const int8_t* sigma,
                  int64_t o, double tau) {
  if (n < 1 || k < 1 || !lam || !U || !sigma || o >= n) return -2;
  double* work = (double*)malloc(sizeof(double) * 3 * (size_t)k * k + 8);
  if (!work) return -3;
  int64_t c = count_impl(n, k, lam, U, sigma, o, tau, work);
  free(work);
  return c;
}

/* #{mu < lam_p}: the count at a pole, from the limit x -> lam_p^-.  The terms
   whose pole equals lam_p blow up along R = span{u_i : lam_i = lam_p}; the
   remaining inertia is that of M~(lam_p) - Sigma compressed onto R^perp, with
   M~ the sum over the other terms.  Then
     #{mu < lam_p} = #{lam_i < lam_p} + dim R + neg(compression) - k_plus. */
int64_t orc_pole_count(int64_t n, int k, const double* lam, const double* U,
                       const int8_t* sigma, int64_t p) {
  if (n < 1 || k < 1 || p < 0 || p >= n) return -2;
  size_t kk = (size_t)k * k;
  double* G = (double*)calloc(4 * kk + 4 * (size_t)k + 8, sizeof(double));
  if (!G) return -3;
  double* Mt = G + kk;
  double* V = Mt + kk;
  double* C = V + kk;
  double* ev = C + kk;
  int64_t below = 0;
  for (int64_t i = 0; i < n; ++i) {
    double d = lam[p] - lam[i];
    if (d > 0.0) ++below;
    if (d == 0.0) {
      for (int b = 0; b < k; ++b)
        for (int a = 0; a < k; ++a) G[IX(a, b, k)] += U[IX(i, a, n)] * U[IX(i, b, n)];
    } else {
      double r = 1.0 / d;
      for (int b = 0; b < k; ++b)
        for (int a = 0; a < k; ++a) Mt[IX(a, b, k)] += U[IX(i, a, n)] * U[IX(i, b, n)] * r;
    }
  }
  for (int c = 0; c < k; ++c) Mt[IX(c, c, k)] -= (double)sigma[c];
  /* R from the Gram matrix of the pole rows. */
  double gmax = 0.0;
  for (size_t t = 0; t < kk; ++t) gmax = fmax(gmax, fabs(G[t]));
  orc_jacobi(k, G, ev, V, 60);
  double tol = 64.0 * ORC_EPS * (double)k * fmax(gmax, DBL_MIN);
  int dimR = 0;
  for (int c = 0; c < k; ++c) dimR += (ev[c] > tol);
  int m = k - dimR; /* basis of R^perp: eigenvectors 0..m-1 (smallest) */
  int neg = 0;
  if (m > 0) {
    /* C = Vp^T Mt Vp  (m x m) */
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b) {
        double s = 0.0;
        for (int r = 0; r < k; ++r)
          for (int q = 0; q < k; ++q) s += V[IX(r, a, k)] * Mt[IX(r, q, k)] * V[IX(q, b, k)];
        C[IX(a, b, m)] = s;
      }
    orc_jacobi(m, C, ev, NULL, 60);
    for (int c = 0; c < m; ++c) neg += (ev[c] < 0.0);
  }
  free(G);
  return below + dimR + neg - kplus_of(k, sigma);
}

/* ------------------------------------------------------------------------ */
/* Root finder: bisection on the count (Sec. 2.3 with one division point).  */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t n;
  int k;
  const double* lam;
  const double* U;
  const int8_t* sigma;
  int64_t nsel;
  const int64_t* sel;
  int64_t* origin;
  double* tau;
  double* mu;
  int32_t* iters;
  int32_t* flags;
  double lo_sent, hi_sent;
  int kminus, kplus;
  int64_t next; /* shared work counter */
  int status;
} roots_job;

static int64_t nearest_pole(const double* lam, int64_t n, double x) {
  int64_t lo = 0, hi = n - 1;
  while (hi - lo > 1) {
    int64_t mid = lo + (hi - lo) / 2;
    if (lam[mid] <= x) lo = mid; else hi = mid;
  }
  return (fabs(x - lam[lo]) <= fabs(lam[hi] - x)) ? lo : hi;
}

static void solve_one(roots_job* J, int64_t m, double* work, int64_t* o_out, double* tau_out,
                      double* mu_out, int32_t* it_out, int32_t* fl_out) {
  const int64_t n = J->n;
  const double* lam = J->lam;
  int64_t ilo = m - J->kminus, ihi = m + J->kplus;
  double lo = (ilo >= 0) ? lam[ilo] : J->lo_sent;
  double hi = (ihi < n) ? lam[ihi] : J->hi_sent;
  int it = 0, flags = 0;
  const int cap = 400;
  /* Phase 1: absolute coordinates. */
  while (it < cap) {
    if (hi - lo <= 4.0 * ORC_EPS * fmax(fabs(lo), fabs(hi))) break;
    double mid = lo + 0.5 * (hi - lo);
    if (!(mid > lo && mid < hi)) break;
    int64_t c = count_impl(n, J->k, lam, J->U, J->sigma, -1, mid, work);
    if (c < 0) { /* exactly on a pole: step one ulp towards hi */
      mid = nextafter(mid, hi);
      if (!(mid < hi)) break;
      c = count_impl(n, J->k, lam, J->U, J->sigma, -1, mid, work);
      if (c < 0) break;
    }
    ++it;
    if (c <= m) lo = mid; else hi = mid;
  }
  /* Phase 2: coordinates shifted to the nearest pole. */
  double mid0 = lo + 0.5 * (hi - lo);
  int64_t o = nearest_pole(lam, n, mid0);
  double tlo = lo - lam[o], thi = hi - lam[o];
  while (it < cap) {
    if (thi - tlo <= 4.0 * ORC_EPS * fmax(fabs(tlo), fabs(thi))) break;
    double mid = tlo + 0.5 * (thi - tlo);
    if (mid == 0.0) mid = 0.5 * thi;
    if (!(mid > tlo && mid < thi)) break;
    int64_t c = count_impl(n, J->k, lam, J->U, J->sigma, o, mid, work);
    if (c < 0) break;
    ++it;
    if (c <= m) tlo = mid; else thi = mid;
  }
  if (it >= cap) flags |= ORC_FLAG_CAP;
  double t = tlo + 0.5 * (thi - tlo);
  if (tlo <= 0.0 && thi >= 0.0 && fabs(t) <= 4.0 * ORC_EPS * fabs(lam[o])) flags |= ORC_FLAG_AT_POLE;
  *o_out = o;
  *tau_out = t;
  *mu_out = lam[o] + t;
  *it_out = it;
  *fl_out = flags;
}

static void* roots_worker(void* arg) {
  roots_job* J = (roots_job*)arg;
  double* work = (double*)malloc(sizeof(double) * (3 * (size_t)J->k * J->k + 8));
  if (!work) {
    J->status = ORC_ENOMEM;
    return NULL;
  }
  for (;;) {
    int64_t s = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
    if (s >= J->nsel) break;
    int64_t m = J->sel ? J->sel[s] : s;
    solve_one(J, m, work, &J->origin[s], &J->tau[s], &J->mu[s], &J->iters[s], &J->flags[s]);
  }
  free(work);
  return NULL;
}

/* Solve the roots listed in sel[0..nsel) (0-based ascending root indices of
   diag(lam) + U Sigma U^T; sel == NULL means all n).  lam must be ascending.
   Outputs per selected root: origin pole index, tau, mu = lam[origin] + tau,
   bisection steps taken and flags. */
int orc_roots(int64_t n, int k, const double* lam, const double* U, const int8_t* sigma,
              int64_t nsel, const int64_t* sel, int nthreads, int64_t* origin, double* tau,
              double* mu, int32_t* iters, int32_t* flags) {
  if (n < 1 || k < 1 || !lam || !U || !sigma || !origin || !tau || !mu || !iters || !flags)
    return ORC_EINVAL;
  if (!sel) nsel = n;
  for (int64_t i = 1; i < n; ++i)
    if (!(lam[i - 1] <= lam[i])) return ORC_EINVAL;
  for (int64_t s = 0; s < nsel; ++s)
    if (sel && (sel[s] < 0 || sel[s] >= n)) return ORC_EINVAL;
  roots_job J;
  memset(&J, 0, sizeof(J));
  J.n = n; J.k = k; J.lam = lam; J.U = U; J.sigma = sigma; J.nsel = nsel; J.sel = sel;
  J.origin = origin; J.tau = tau; J.mu = mu; J.iters = iters; J.flags = flags;
  double splus = 0.0, sminus = 0.0;
  for (int c = 0; c < k; ++c) {
    double s2 = 0.0;
    for (int64_t i = 0; i < n; ++i) s2 += U[IX(i, c, n)] * U[IX(i, c, n)];
    if (sigma[c] > 0) { splus += s2; J.kplus++; } else { sminus += s2; J.kminus++; }
  }
  /* Weyl: every eigenvalue of diag(lam) + U Sigma U^T lies in
     [lam_min - sum_{sigma<0} |U_c|^2, lam_max + sum_{sigma>0} |U_c|^2];
     the sentinels sit strictly outside that interval. */
  J.lo_sent = lam[0] - 2.0 * sminus - 1e-300 - 4.0 * ORC_EPS * fabs(lam[0]);
  J.hi_sent = lam[n - 1] + 2.0 * splus + 1e-300 + 4.0 * ORC_EPS * fabs(lam[n - 1]);
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  pthread_t th[256];
  int started = 0;
  for (int t = 1; t < nthreads; ++t) {
    if (pthread_create(&th[t], NULL, roots_worker, &J) != 0) break;
    ++started;
  }
  roots_worker(&J);
  for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
  return J.status;
}

/* ------------------------------------------------------------------------ */
/* Eigenvectors of the update in the old eigenbasis, eq. (10).              */
/* For each root s: alpha_0 = eigenvector of the k x k Sigma - M(mu_s) whose */
/* eigenvalue has the rank[s]-th smallest magnitude (rank > 0 only for a    */
/* repeated root); w_i = (u_i^T alpha_0) / (lam_i - mu_s); W[:,s] = w/|w|,   */
/* sign fixed so that the entry of largest magnitude is positive.            */
/* ------------------------------------------------------------------------ */
int orc_vectors(int64_t n, int k, const double* lam, const double* U, const int8_t* sigma,
                int64_t nsel, const int64_t* origin, const double* tau, const int32_t* rank,
                double* W, double* alpha) {
  if (n < 1 || k < 1 || nsel < 0 || !W) return ORC_EINVAL;
  size_t kk = (size_t)k * k;
  double* Mk = (double*)malloc(sizeof(double) * (2 * kk + 2 * (size_t)k + 8));
  if (!Mk) return ORC_ENOMEM;
  double* V = Mk + kk;
  double* ev = V + kk;
  int* order = (int*)malloc(sizeof(int) * (size_t)k);
  if (!order) {
    free(Mk);
    return ORC_ENOMEM;
  }
  for (int64_t s = 0; s < nsel; ++s) {
    int64_t o = origin[s];
    double t = tau[s];
    double* w = W + (size_t)s * (size_t)n;
    if (build_M(n, k, lam, U, o, t, Mk) < 0) {
      for (int64_t i = 0; i < n; ++i) w[i] = (i == o) ? 1.0 : 0.0;
      continue;
    }
    for (int a = 0; a < k; ++a)
      for (int b = 0; b < k; ++b) Mk[IX(a, b, k)] = ((a == b) ? (double)sigma[a] : 0.0) - Mk[IX(a, b, k)];
    orc_jacobi(k, Mk, ev, V, 60);
    for (int c = 0; c < k; ++c) order[c] = c;
    for (int c = 0; c < k; ++c) /* sort by |eigenvalue| */
      for (int d = c + 1; d < k; ++d)
        if (fabs(ev[order[d]]) < fabs(ev[order[c]])) {
          int tmp = order[c];
          order[c] = order[d];
          order[d] = tmp;
        }
    int r = rank ? rank[s] : 0;
    if (r < 0) r = 0;
    if (r >= k) r = k - 1;
    const double* a0 = V + (size_t)order[r] * k;
    if (alpha)
      for (int c = 0; c < k; ++c) alpha[(size_t)s * k + c] = a0[c];
    double nrm = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      double ua = 0.0;
      for (int c = 0; c < k; ++c) ua += U[IX(i, c, n)] * a0[c];
      double d = -diff_at(lam, i, o, t); /* lam_i - mu */
      w[i] = ua / d;
      nrm += w[i] * w[i];
    }
    nrm = sqrt(nrm);
    int64_t imax = 0;
    for (int64_t i = 0; i < n; ++i)
      if (fabs(w[i]) > fabs(w[imax])) imax = i;
    double sc = (w[imax] < 0.0 ? -1.0 : 1.0) / nrm;
    for (int64_t i = 0; i < n; ++i) w[i] *= sc;
  }
  free(order);
  free(Mk);
  return ORC_OK;
}
