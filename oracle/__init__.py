"""CPU FP64 oracle for the rank-k eigen-update of Oh & Hu (arXiv 1706.00773).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package.  The product library
never imports, links or calls it, and it imports nothing from the product.  The
only module both sides share is ``workloads`` (seeded input generators).

Plain and slow on purpose.  The C part (``orc.c``) holds the Jacobi
eigensolver, the root count, the bisection root finder and the eq. (10)
vectors.  This module composes them with numpy library primitives (matmul),
and adds the rank-2 location vector (Algorithms 1a-1c, with the residues of
eq. (3)), the exact-rational Sturm chains of Sec. 2.2 for tiny problems, and
the first-order perturbation estimate of eq. (11) with the Figs. 6-7 panels.
Each function names the passage of the paper it follows.  The paper prints no
worked example, so every pin is a closed form, an invariant, a special case or
a library routine (``tests/test_oracle_pins.py``).

Conventions: Q is n x n with eigenvectors as columns (column-major in memory
when handed to C), lam is ascending, K is n x k, sigma holds +1/-1 per column.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "orc.c")
_SO = os.path.join(_HERE, "_orc.so")
_lock = threading.Lock()
_lib = None

EPS = float(np.finfo(np.float64).eps)
FLAG_CAP = 1
FLAG_AT_POLE = 2


def build(force: bool = False) -> str:
    """Compile orc.c into oracle/_orc.so with gcc (plain -O2, IEEE semantics)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _bind(path: str):
    """Load a compiled oracle library and declare its signatures."""
    lib = ctypes.CDLL(path)
    d, i64, i32, i8 = (ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                       ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int8))
    lib.orc_jacobi.argtypes = [ctypes.c_int, d, d, d, ctypes.c_int]
    lib.orc_jacobi.restype = ctypes.c_int
    lib.orc_count.argtypes = [ctypes.c_int64, ctypes.c_int, d, d, i8, ctypes.c_int64, ctypes.c_double]
    lib.orc_count.restype = ctypes.c_int64
    lib.orc_pole_count.argtypes = [ctypes.c_int64, ctypes.c_int, d, d, i8, ctypes.c_int64]
    lib.orc_pole_count.restype = ctypes.c_int64
    lib.orc_roots.argtypes = [ctypes.c_int64, ctypes.c_int, d, d, i8, ctypes.c_int64, i64,
                              ctypes.c_int, i64, d, d, i32, i32]
    lib.orc_roots.restype = ctypes.c_int
    lib.orc_vectors.argtypes = [ctypes.c_int64, ctypes.c_int, d, d, i8, ctypes.c_int64, i64, d,
                                i32, d, d]
    lib.orc_vectors.restype = ctypes.c_int
    return lib


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(_SO)
        return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _colmajor(A):
    return np.asfortranarray(np.asarray(A, dtype=np.float64))


def _sig(sigma, k):
    if sigma is None:
        return np.ones(k, dtype=np.int8)
    s = np.asarray(sigma).astype(np.int8).reshape(-1)
    if s.shape[0] != k or not np.all(np.abs(s) == 1):
        raise ValueError("sigma must hold k entries of +1/-1")
    return np.ascontiguousarray(s)


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)


# ---------------------------------------------------------------------------
# Plain definitions
# ---------------------------------------------------------------------------
def jacobi_eig(A, vectors: bool = True, max_sweeps: int = 60):
    """Cyclic Jacobi eigendecomposition of a symmetric matrix (textbook definition).

    Returns (w ascending, V with eigenvectors as columns or None)."""
    A = _colmajor(A).copy(order="F")
    n = A.shape[0]
    w = np.zeros(n)
    V = np.zeros((n, n), order="F") if vectors else None
    rc = _L().orc_jacobi(n, _p(A, ctypes.c_double), _p(w, ctypes.c_double),
                         _p(V, ctypes.c_double) if vectors else None, max_sweeps)
    if rc < 0:
        raise ValueError("orc_jacobi failed")
    return w, V


def updated_matrix(Q, lam, K, sigma=None):
    """A' = Q diag(lam) Q^T + K diag(sigma) K^T (Sec. 2.1 problem statement)."""
    Q = np.asarray(Q, dtype=np.float64)
    K = np.asarray(K, dtype=np.float64).reshape(Q.shape[0], -1)
    s = _sig(sigma, K.shape[1]).astype(np.float64)
    A = (Q * np.asarray(lam, dtype=np.float64)[None, :]) @ Q.T + (K * s[None, :]) @ K.T
    return 0.5 * (A + A.T)


def dense_update(Q, lam, K, sigma=None, vectors: bool = True):
    """The direct EVD comparison system (Sec. 3): Jacobi on the dense A'.  n <= ~512."""
    A = updated_matrix(Q, lam, K, sigma)
    return jacobi_eig(A, vectors=vectors)


# ---------------------------------------------------------------------------
# Method steps, in the paper's order
# ---------------------------------------------------------------------------
def project(Q, K):
    """U = Q^T K (Sec. 2.1, below eq. (1)); numpy matmul as the library step."""
    return np.asarray(Q, dtype=np.float64).T @ np.asarray(K, dtype=np.float64).reshape(Q.shape[0], -1)


def rank2_perturbation(n: int, j: int, a):
    """Sec. 2.2 Steps 1-2: e_j a^T + a e_j^T = (x y) [[0,1],[1,0]] (x y)^T with x = e_j, y = a.
    The 2x2 middle matrix is S diag(1,-1) S^T, S = [[1,1],[1,-1]]/sqrt(2), so
    (u1 u2) = (x y) S: K = [(e_j + a)/sqrt2, (e_j - a)/sqrt2], sigma = (+1, -1)."""
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    if a.shape[0] != n or not (0 <= j < n):
        raise ValueError("bad rank-2 arguments")
    e = np.zeros(n)
    e[j] = 1.0
    r = 1.0 / np.sqrt(2.0)
    K = np.stack([(e + a) * r, (e - a) * r], axis=1)
    return K, np.array([1, -1], dtype=np.int8)


def repeated_runs(lam):
    """Maximal runs [g0, g0 + m) of exactly equal lam with m >= 2 (lam ascending)."""
    lam = np.asarray(lam, dtype=np.float64)
    runs = []
    i, n = 0, lam.shape[0]
    while i < n:
        j = i + 1
        while j < n and lam[j] == lam[i]:
            j += 1
        if j - i > 1:
            runs.append((i, j - i))
        i = j
    return runs


def group_rotate(Q, lam, U):
    """Exactly repeated eigenvalues (the paper assumes distinct lam, Sec. 2.1).

    On a run G of m >= 2 equal lam, A = Q diag(lam) Q^T does not change when
    Q_G is replaced by Q_G H for any orthogonal m x m H, and U_G = Q_G^T K then
    becomes H^T U_G.  With the complete QR U_G = H R (numpy, a library step) the
    run's rows of U become R: rows past min(m, k) are zero and rows past
    rank(U_G) are at rounding level, so the row deflation removes them and the
    secular problem keeps the pole lam at most min(m, k) times.  The removed
    pairs are (lam, Q_G H e_j): an orthonormal basis of the part of the
    eigenspace that K does not touch.  Returns (Q~, U~); the inputs when lam
    has no repeats."""
    runs = repeated_runs(lam)
    if not runs:
        return Q, U
    Qt = np.array(Q, dtype=np.float64, copy=True)
    Ut = np.array(U, dtype=np.float64, copy=True)
    k = Ut.shape[1]
    for g0, m in runs:
        H, R = np.linalg.qr(Ut[g0:g0 + m], mode="complete")
        R[min(m, k):] = 0.0
        Ut[g0:g0 + m] = R
        Qt[:, g0:g0 + m] = Qt[:, g0:g0 + m] @ H
    return Qt, Ut


def deflation_mask(lam, U):
    """Rows u_i small enough to drop (the paper assumes all u_i != 0 and
    distinct lam, Sec. 2.1; it is silent on what to do otherwise).
    Row i is deflated when |u_i|_2 |U|_F <= 8 eps (max|lam| + |U|_F^2): zeroing it
    changes A' by at most that much in norm.  Deflated pairs keep mu = lam_i
    and the old eigenvector q_i."""
    lam = np.asarray(lam, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64).reshape(lam.shape[0], -1)
    rown = np.sqrt(np.sum(U * U, axis=1))
    fro2 = float(np.sum(U * U))
    fro = np.sqrt(fro2)
    tol = 8.0 * EPS * (float(np.max(np.abs(lam))) + fro2)
    return rown * fro <= tol


def count(lam, U, sigma, x: float, origin: int = -1) -> int:
    """#{mu < x} for diag(lam) + U Sigma U^T (the root-count sub-problem, Sec. 2.1-2.2).
    With origin >= 0 the point is x = lam[origin] + x."""
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    U = _colmajor(U)
    n, k = U.shape
    s = _sig(sigma, k)
    return int(_L().orc_count(n, k, _p(lam, ctypes.c_double), _p(U, ctypes.c_double),
                              _p(s, ctypes.c_int8), origin, float(x)))


def pole_count(lam, U, sigma, p: int) -> int:
    """#{mu < lam_p}: the count at a pole (limit from the left)."""
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    U = _colmajor(U)
    n, k = U.shape
    s = _sig(sigma, k)
    return int(_L().orc_pole_count(n, k, _p(lam, ctypes.c_double), _p(U, ctypes.c_double),
                                   _p(s, ctypes.c_int8), int(p)))


def roots(lam, U, sigma=None, sel=None, nthreads: int | None = None):
    """Roots of f (Sec. 2.3, bisection on the count inside interlacing brackets)."""
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    U = _colmajor(U)
    n, k = U.shape
    s = _sig(sigma, k)
    if sel is None:
        m = n
        selp = None
    else:
        sel = np.ascontiguousarray(sel, dtype=np.int64)
        m = sel.shape[0]
        selp = _p(sel, ctypes.c_int64)
    origin = np.zeros(m, dtype=np.int64)
    tau = np.zeros(m)
    mu = np.zeros(m)
    iters = np.zeros(m, dtype=np.int32)
    flags = np.zeros(m, dtype=np.int32)
    if m == 0:
        return dict(origin=origin, tau=tau, mu=mu, iters=iters, flags=flags)
    rc = _L().orc_roots(n, k, _p(lam, ctypes.c_double), _p(U, ctypes.c_double), _p(s, ctypes.c_int8),
                        m, selp, int(nthreads or default_threads()), _p(origin, ctypes.c_int64),
                        _p(tau, ctypes.c_double), _p(mu, ctypes.c_double), _p(iters, ctypes.c_int32),
                        _p(flags, ctypes.c_int32))
    if rc != 0:
        raise ValueError("orc_roots failed (%d)" % rc)
    return dict(origin=origin, tau=tau, mu=mu, iters=iters, flags=flags)


def tie_ranks(mu, lam_scale: float):
    """Rank of each root inside a run of numerically equal roots (repeated eigenvalue)."""
    mu = np.asarray(mu)
    rank = np.zeros(mu.shape[0], dtype=np.int32)
    tol = 64.0 * EPS * max(lam_scale, 1e-300)
    for i in range(1, mu.shape[0]):
        if mu[i] - mu[i - 1] <= tol:
            rank[i] = rank[i - 1] + 1
    return rank


def vectors(lam, U, sigma, origin, tau, rank=None):
    """Eq. (10) in the old eigenbasis: columns w_s (unit, largest entry positive)."""
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    U = _colmajor(U)
    n, k = U.shape
    s = _sig(sigma, k)
    origin = np.ascontiguousarray(origin, dtype=np.int64)
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    m = origin.shape[0]
    rk = np.ascontiguousarray(rank if rank is not None else np.zeros(m), dtype=np.int32)
    W = np.zeros((n, m), order="F")
    if m:
        rc = _L().orc_vectors(n, k, _p(lam, ctypes.c_double), _p(U, ctypes.c_double),
                              _p(s, ctypes.c_int8), m, _p(origin, ctypes.c_int64),
                              _p(tau, ctypes.c_double), _p(rk, ctypes.c_int32),
                              _p(W, ctypes.c_double), None)
        if rc != 0:
            raise ValueError("orc_vectors failed")
    # A repeated root gives a multi-dimensional eigenspace; eq. (10) maps an
    # orthonormal basis of the k x k null space onto a basis of it that need not
    # be orthonormal, so orthonormalise inside each run of equal roots.
    i = 0
    while i < m:
        j = i + 1
        while j < m and rk[j] > 0:
            j += 1
        if j - i > 1:
            Qg, _ = np.linalg.qr(W[:, i:j])
            W[:, i:j] = Qg
        i = j
    return W


def update(Q, lam, K, sigma=None, want_vectors: bool = True, sel=None, nthreads: int | None = None):
    """The whole update A' = Q diag(lam) Q^T + K Sigma K^T, by the paper's method
    (with exactly repeated eigenvalues first rotated by ``group_rotate``).

    sel (optional) lists root indices m of the non-deflated sub-problem to solve
    (sampling for large n); then only those roots and vectors are returned.
    Returns a dict with mu (ascending), X (n x len) if want_vectors, and the
    bookkeeping needed to map sampled roots onto output positions."""
    Q = np.asarray(Q, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    n = lam.shape[0]
    K = np.asarray(K, dtype=np.float64).reshape(n, -1)
    k = K.shape[1]
    s = _sig(sigma, k)
    U = project(Q, K)
    Q, U = group_rotate(Q, lam, U)  # no-op unless lam has exact repeats
    defl = deflation_mask(lam, U)
    keep = np.nonzero(~defl)[0]
    lam_p = lam[keep]
    U_p = U[keep]
    out = dict(U=U, deflated=defl, keep=keep, Q=Q)
    if sel is not None:
        r = roots(lam_p, U_p, s, sel=sel, nthreads=nthreads)
        mu = r["mu"]
        dl = np.sort(lam[defl])
        pos = np.asarray(sel, dtype=np.int64) + np.searchsorted(dl, mu, side="left")
        out.update(mu=mu, pos=pos, roots=r)
        if want_vectors:
            Wp = vectors(lam_p, U_p, s, r["origin"], r["tau"])
            Wfull = np.zeros((n, Wp.shape[1]))
            Wfull[keep] = Wp
            out["W"] = Wfull
            out["X"] = Q @ Wfull
        return out
    r = roots(lam_p, U_p, s, nthreads=nthreads) if keep.shape[0] else None
    mu_s = r["mu"] if r is not None else np.zeros(0)
    mu_all = np.concatenate([mu_s, lam[defl]])
    src = np.concatenate([np.arange(mu_s.shape[0]), -1 - np.nonzero(defl)[0]])
    order = np.argsort(mu_all, kind="stable")
    out.update(mu=mu_all[order], roots=r, order_src=src[order])
    if want_vectors:
        W = np.zeros((n, n))
        if r is not None:
            rk = tie_ranks(mu_s, float(np.max(np.abs(lam))) + float(np.sum(U * U)))
            Wp = vectors(lam_p, U_p, s, r["origin"], r["tau"], rk)
        for c, sidx in enumerate(src[order]):
            if sidx >= 0:
                W[keep, c] = Wp[:, sidx]
            else:
                W[-1 - sidx, c] = 1.0
        out["W"] = W
        out["X"] = Q @ W
    return out


# ---------------------------------------------------------------------------
# Result quality (the Sec. 3 accuracy metrics B and C of Figs. 6-7)
# ---------------------------------------------------------------------------
def residuals(Q, lam, K, sigma, mu, X):
    """|A' x_r - mu_r x_r|_2 per column, with A' applied as Q(lam*(Q^T x)) + K Sigma K^T x."""
    Q = np.asarray(Q, dtype=np.float64)
    K = np.asarray(K, dtype=np.float64).reshape(Q.shape[0], -1)
    s = _sig(sigma, K.shape[1]).astype(np.float64)
    X = np.asarray(X, dtype=np.float64)
    AX = Q @ (np.asarray(lam)[:, None] * (Q.T @ X)) + K @ (s[:, None] * (K.T @ X))
    return np.linalg.norm(AX - X * np.asarray(mu)[None, :], axis=0)


def orthogonality(X):
    """max |X^T X - I| entry."""
    X = np.asarray(X, dtype=np.float64)
    G = X.T @ X
    return float(np.max(np.abs(G - np.eye(G.shape[0]))))


# ---------------------------------------------------------------------------
# Location sub-problem, rank 2 (Sec. 2.2, Algorithms 1a-1c)
# ---------------------------------------------------------------------------
def residues(lam, U, sigma=None):
    """alpha_i of eq. (3), f(x) = 1 + sum_i alpha_i/(lam_i - x), for
    f(x) = det(I - Sigma U^T (xI - Lam)^{-1} U): with B_i = I + Sigma U^T D_i U,
    D_i = diag(1/(lam_j - lam_i)) (j != i), alpha_i = u_i^T adj(B_i) Sigma u_i
    (eq. (2) with its sign corrected).  Distinct lam required."""
    lam = np.asarray(lam, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64).reshape(lam.shape[0], -1)
    n, k = U.shape
    S = np.diag(_sig(sigma, k).astype(np.float64))
    out = np.zeros(n)
    for i in range(n):
        d = np.zeros(n)
        m = np.arange(n) != i
        d[m] = 1.0 / (lam[m] - lam[i])
        B = np.eye(k) + S @ U.T @ (U * d[:, None])
        if k == 1:
            adj = np.ones((1, 1))
        elif k == 2:
            adj = np.array([[B[1, 1], -B[0, 1]], [-B[1, 0], B[0, 0]]])
        else:
            adj = np.linalg.det(B) * np.linalg.inv(B)
        out[i] = U[i] @ adj @ S @ U[i]
    return out


def location_vector(lam, U, sigma, printed_1c=False):
    """Algorithms 1a-1c for a rank-2 update: L[0] roots below lam_1, L[i]
    roots in (lam_i, lam_{i+1}), L[n] roots above lam_n (0-based L of length
    n+1).  1a (both sigma > 0) scans up from the left; 1b (both < 0) is its
    mirror from the right (the bound on the roots placed so far is the
    mirrored one of 1a); 1c (opposite signs) starts from the sign of the
    first residue and scans up.  Where the listings read mu_{n+1} or mu_0
    (undefined), the last interval takes the roots not placed yet.

    With opposite signs every new root lies within one pole of its old
    eigenvalue, so at most i+1 roots lie below lam_{i+1}: the 0-or-2 choice
    of 1c compares M+2 with i+1.  printed_1c=True keeps the bound of 1a
    (M+2 > i) as the listing of 1c prints it, which misplaces roots."""
    lam = np.asarray(lam, dtype=np.float64)
    n = lam.shape[0]
    s = _sig(sigma, 2)
    a = residues(lam, U, s)
    L = np.zeros(n + 1, dtype=np.int64)
    if s[0] > 0 and s[1] > 0:
        M = 0
        for i in range(1, n):  # interval (lam_i, lam_{i+1}) in 1-based terms -> L[i]
            if a[i - 1] * a[i] > 0:
                L[i] = 1
                M += 1
            elif M + 2 > i:
                L[i] = 0
            else:
                L[i] = 2
                M += 2
        L[n] = n - M
    elif s[0] < 0 and s[1] < 0:
        M = 0
        for i in range(1, n):  # mirror: interval (lam_{n-i}, lam_{n-i+1}) -> L[n-i]
            j = n - i
            if a[j - 1] * a[j] > 0:
                L[j] = 1
                M += 1
            elif M + 2 > i:
                L[j] = 0
            else:
                L[j] = 2
                M += 2
        L[0] = n - M
    else:
        if a[0] > 0:
            M, L[0] = 0, 0
        else:
            M, L[0] = 1, 1
        bound = 0 if printed_1c else 1
        for i in range(1, n):
            if a[i - 1] * a[i] > 0:
                L[i] = 1
                M += 1
            elif M + 2 > i + bound:
                L[i] = 0
            else:
                L[i] = 2
                M += 2
        L[n] = n - M
    return L


# ---------------------------------------------------------------------------
# The Sturm chain of Sec. 2.2 in exact rational arithmetic (tiny n only)
# ---------------------------------------------------------------------------
def _frac_det(M):
    from fractions import Fraction

    A = [[Fraction(v) for v in row] for row in M]
    n = len(A)
    det = Fraction(1)
    for c in range(n):
        p = next((r for r in range(c, n) if A[r][c] != 0), None)
        if p is None:
            return Fraction(0)
        if p != c:
            A[c], A[p] = A[p], A[c]
            det = -det
        det *= A[c][c]
        for r in range(c + 1, n):
            f = A[r][c] / A[c][c]
            for j in range(c, n):
                A[r][j] -= f * A[c][j]
    return det


def _poly_from_values(xs, ys):
    """Exact interpolation: coefficients (lowest degree first) through (xs, ys)."""
    from fractions import Fraction

    n = len(xs)
    coef = [Fraction(0)] * n
    for i in range(n):
        basis = [Fraction(1)]
        den = Fraction(1)
        for j in range(n):
            if j == i:
                continue
            basis = [Fraction(0)] + basis
            for t in range(len(basis) - 1):
                basis[t] -= xs[j] * basis[t + 1]
            den *= xs[i] - xs[j]
        for t in range(n):
            coef[t] += ys[i] * basis[t] / den
    return coef


def _trim(p):
    while len(p) > 1 and p[-1] == 0:
        p = p[:-1]
    return p


def _polyrem(a, b):
    from fractions import Fraction

    a = list(a)
    b = _trim(list(b))
    while len(_trim(a)) >= len(b) and any(v != 0 for v in a):
        a = _trim(a)
        if len(a) < len(b):
            break
        f = a[-1] / b[-1]
        sh = len(a) - len(b)
        for t in range(len(b)):
            a[sh + t] -= f * b[t]
        a = a[:-1] if a[-1] == 0 else a
    return _trim(a) if a else [Fraction(0)]


def sturm_chain(lam, U, sigma=None):
    """p_0 = prod(x - lam_i) f_0(x) = det(xI - A') (the numerator of the
    secular function, eq. (5)), p_1 = p_0', p_m = -rem(p_{m-2}, p_{m-1}):
    the chain the secular long division of Sec. 2.2 builds, here in exact
    rationals from the exact float inputs."""
    from fractions import Fraction

    lam = np.asarray(lam, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64).reshape(lam.shape[0], -1)
    n, k = U.shape
    S = _sig(sigma, k)
    Uf = [[Fraction(float(U[i, c])) for c in range(k)] for i in range(n)]
    A = [[(Fraction(float(lam[i])) if i == j else Fraction(0)) +
          sum(Uf[i][c] * Uf[j][c] * int(S[c]) for c in range(k)) for j in range(n)] for i in range(n)]
    xs = [Fraction(t) for t in range(n + 1)]
    ys = [_frac_det([[(xs[t] if i == j else 0) - A[i][j] for j in range(n)] for i in range(n)]) for t in range(n + 1)]
    p0 = _poly_from_values(xs, ys)
    p1 = [p0[t] * t for t in range(1, len(p0))]
    chain = [_trim(p0), _trim(p1)]
    while len(chain[-1]) > 1 or chain[-1][0] != 0:
        r = _polyrem(chain[-2], chain[-1])
        if all(v == 0 for v in r):
            break
        chain.append([-v for v in r])
        if len(chain[-1]) == 1:
            break
    return chain


def sturm_count(chain, x) -> int:
    """Number of distinct roots of p_0 below x: V(-inf) - V(x), V = sign changes."""
    from fractions import Fraction

    def sign_changes(vals):
        s = [v for v in vals if v != 0]
        return sum(1 for a, b in zip(s, s[1:]) if (a > 0) != (b > 0))

    X = Fraction(float(x))
    at_x = [sum(c * X ** t for t, c in enumerate(p)) for p in chain]
    at_minf = [c[-1] * (1 if (len(c) - 1) % 2 == 0 else -1) for c in chain]
    return sign_changes(at_minf) - sign_changes(at_x)


# ---------------------------------------------------------------------------
# The modified Sturm chain in secular form (Sec. 2.2, eqs. (4)-(9)), exact
# ---------------------------------------------------------------------------
def _frac_residues(lam, U, sigma):
    """Exact alpha_j^{0} of eq. (4) from p_0 = pi_0 f_0 = det(xI - A'):
    p_0(d_j) = -alpha_j prod_{k != j} (d_j - d_k)."""
    from fractions import Fraction

    lam = np.asarray(lam, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64).reshape(lam.shape[0], -1)
    n, k = U.shape
    S = _sig(sigma, k)
    d = [Fraction(float(v)) for v in lam]
    Uf = [[Fraction(float(U[i, c])) for c in range(k)] for i in range(n)]
    A = [[(d[i] if i == j else Fraction(0)) + sum(Uf[i][c] * Uf[j][c] * int(S[c]) for c in range(k))
          for j in range(n)] for i in range(n)]
    alpha = []
    for j in range(n):
        pj = _frac_det([[(d[j] if r == c else 0) - A[r][c] for c in range(n)] for r in range(n)])
        w = Fraction(1)
        for t in range(n):
            if t != j:
                w *= d[j] - d[t]
        alpha.append(-pj / w)
    return d, alpha


def _top3(c, alpha, poles):
    """Coefficients of x^D, x^(D-1), x^(D-2) of (c - sum alpha_j/(x - d_j)) prod (x - d_k)."""
    e1 = sum(poles)
    e2 = (e1 * e1 - sum(p * p for p in poles)) / 2
    return (c, -c * e1 - sum(alpha), c * e2 + sum(a * (e1 - p) for a, p in zip(alpha, poles)))


def secular_sturm_chain(lam, U, sigma=None):
    """The chain p_m = f_m pi_m, f_m = c_m - sum_{j <= N-m} alpha_j^{m}/(x - d_j),
    pi_m = prod_{j <= N-m} (x - d_j), in exact rationals.

    p_0 is eq. (5) with c_0 = 1; p_1 = p_0' in the form of eq. (6):
    mu_j = 1 - sum_{i != j} (alpha_i + alpha_j)/(d_j - d_i), c_1 = sum mu_j,
    alpha_j^{1} = (d_N - d_j) mu_j.  Then the secular long division:
    p_m = A_m (x - B_m) p_{m-1} - p_{m-2} with A_m = c_{m-2}/c_{m-1} and B_m
    chosen so that the x^(D-1) terms cancel (D = N-m+2 poles in p_{m-2}):
    B_m = d_D + (1/c_{m-2}) sum alpha^{m-2} - (1/c_{m-1}) sum alpha^{m-1}.
    The new residues follow from the values at the poles that remain:
    alpha_j^{m} = A (d_j - B)(d_j - d_{D-1}) alpha_j^{m-1} - (d_j - d_{D-1})(d_j - d_D) alpha_j^{m-2},
    and c_m is the x^(D-2) coefficient.  Returns (d, [(c_m, alpha^{m})]);
    the chain stops early (returned shorter) if some c_m is 0."""
    from fractions import Fraction

    d, a0 = _frac_residues(lam, U, sigma)
    N = len(d)
    chain = [(Fraction(1), a0)]
    if N == 0:
        return d, chain
    mu = [1 - sum((a0[i] + a0[j]) / (d[j] - d[i]) for i in range(N) if i != j) for j in range(N)]
    chain.append((sum(mu), [(d[N - 1] - d[j]) * mu[j] for j in range(N - 1)]))
    for m in range(2, N + 1):
        c2, a2 = chain[m - 2]
        c1, a1 = chain[m - 1]
        if c1 == 0:
            break
        D = N - m + 2
        A = c2 / c1
        B = d[D - 1] + sum(a2) / c2 - sum(a1) / c1
        t2 = _top3(c2, a2, d[:D])
        t1 = _top3(c1, a1, d[:D - 1])
        assert A * t1[0] - t2[0] == 0 and A * t1[1] - A * B * t1[0] - t2[1] == 0
        cm = A * t1[2] - A * B * t1[1] - t2[2]
        am = [A * (d[j] - B) * (d[j] - d[D - 2]) * a1[j] - (d[j] - d[D - 2]) * (d[j] - d[D - 1]) * a2[j]
              for j in range(D - 2)]
        chain.append((cm, am))
    return d, chain


def secular_sturm_values(d, chain, x):
    """p_m(x) for every member of the secular chain (x exact; a pole uses the limit)."""
    from fractions import Fraction

    X = Fraction(float(x)) if not isinstance(x, Fraction) else x
    out = []
    for c, alpha in chain:
        poles = d[:len(alpha)]
        if any(X == p for p in poles):
            j = poles.index(X)
            w = Fraction(1)
            for t, p in enumerate(poles):
                if t != j:
                    w *= X - p
            out.append(-alpha[j] * w)
            continue
        f = c - sum(a / (X - p) for a, p in zip(alpha, poles))
        pi = Fraction(1)
        for p in poles:
            pi *= X - p
        out.append(f * pi)
    return out


def secular_sturm_count(d, chain, x) -> int:
    """Distinct roots of p_0 below x: V(-inf) - V(x).  At -inf, p_m has the sign
    of c_m (-1)^(number of its poles)."""
    def changes(vals):
        s = [v for v in vals if v != 0]
        return sum(1 for a, b in zip(s, s[1:]) if (a > 0) != (b > 0))

    at_minf = [c * (1 if len(a) % 2 == 0 else -1) for c, a in chain]
    return changes(at_minf) - changes(secular_sturm_values(d, chain, x))


def secular_deflate(lam, alpha, xi):
    """Eq. (9): divide the roots xi_1..xi_s (found earlier) out of p_0, pairing
    xi_p with the pole d_p: beta_j = alpha_j prod_p (d_j - d_p)/(d_j - xi_p) for
    the poles j > s that remain, so that
    p_0^1(x) = (1 - sum_{j>s} beta_j/(x - d_j)) prod_{j>s} (x - d_j) = p_0(x) / prod_p (x - xi_p)."""
    lam = np.asarray(lam, dtype=np.float64)
    alpha = np.asarray(alpha, dtype=np.float64)
    xi = np.asarray(xi, dtype=np.float64)
    s = xi.shape[0]
    rest = lam[s:]
    beta = alpha[s:].copy()
    for p in range(s):
        beta *= (rest - lam[p]) / (rest - xi[p])
    return rest, beta


# ---------------------------------------------------------------------------
# The first-order perturbation estimate (Sec. 3, eq. (11)): comparison method
# ---------------------------------------------------------------------------
def perturbation(Q, lam, K, sigma=None, cols=None):
    """mu_j = lam_j + u_j^T Sigma u_j and v_j = q_j + sum_{i != j}
    (u_i^T Sigma u_j)/(lam_j - lam_i) q_i with u = rows of U = Q^T K (eq. (11)
    read as standard first-order perturbation theory: the printed update names
    v_j^0 and lam_i - lam_j where q_i and lam_j - lam_i belong).  Pairs with
    lam_i == lam_j contribute nothing.  mu_j pairs with column j of X; nothing
    is sorted.  With cols, X holds only those columns (in that order)."""
    Q = np.asarray(Q, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    K = np.asarray(K, dtype=np.float64).reshape(lam.shape[0], -1)
    s = _sig(sigma, K.shape[1]).astype(np.float64)
    U = Q.T @ K
    n = lam.shape[0]
    cols = list(range(n)) if cols is None else [int(c) for c in cols]
    W = np.zeros((n, len(cols)))
    for t, j in enumerate(cols):
        e_j = U @ (s * U[j])  # E_ij = u_i^T Sigma u_j for every i
        for i in range(n):
            if i == j:
                W[i, t] = 1.0
            elif lam[j] != lam[i]:
                W[i, t] = e_j[i] / (lam[j] - lam[i])
    mu = lam + np.einsum("ic,c,ic->i", U, s, U)
    return mu, Q @ W


def fig67_metrics(Q, lam, K, sigma, mu, X):
    """The accuracy panels of Figs. 6-7 for an estimate (mu, X) of the updated
    pairs of A' = Q diag(lam) Q^T + K Sigma K^T: (A) 2-norm eigenvalue error
    against the dense decomposition, relative to the 2-norm of the dense
    eigenvalues; (B) 2-norm of A' - X diag(mu) X^T relative to ||A'||_2;
    (C) 2-norm of X^T X - I."""
    A = updated_matrix(Q, lam, K, sigma)
    w = np.linalg.eigvalsh(A)
    mu = np.asarray(mu, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    a = float(np.linalg.norm(np.sort(mu) - w) / np.linalg.norm(w))
    b = float(np.linalg.norm(A - (X * mu[None, :]) @ X.T, 2) / np.linalg.norm(A, 2))
    c = float(np.linalg.norm(X.T @ X - np.eye(X.shape[1]), 2))
    return {"A": a, "B": b, "C": c}
