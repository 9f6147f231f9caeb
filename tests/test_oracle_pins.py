"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these re-types the oracle's own formula: each compares it with a
closed form, an invariant, a special case that reduces to a textbook routine,
or a library routine (numpy LAPACK) used only as an independent check.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

EPS = np.finfo(np.float64).eps


def _problem(n, k, seed, sigma="psd", lam_kind="uniform", kscale=None):
    P = workloads.general(n, k, seed=seed, sigma=sigma, lam_kind=lam_kind, kscale=kscale)
    return P["Q"], P["lam"], P["K"], P["sigma"]


# --------------------------------------------------------------------------
# Jacobi (the direct EVD comparison system, Sec. 3)
# --------------------------------------------------------------------------
def test_jacobi_2x2_closed_form():
    for a, b, c in [(1.0, 2.0, -3.0), (0.5, 1e-9, 0.5), (-2.0, 0.0, 7.0), (1e3, 3.0, -1e-3)]:
        w, V = oracle.jacobi_eig(np.array([[a, b], [b, c]]))
        m, r = 0.5 * (a + c), math.hypot(0.5 * (a - c), b)
        assert abs(w[0] - (m - r)) <= 4 * EPS * (abs(m) + r)
        assert abs(w[1] - (m + r)) <= 4 * EPS * (abs(m) + r)
        A = np.array([[a, b], [b, c]])
        assert np.max(np.abs(A @ V - V * w)) <= 8 * EPS * (abs(m) + r)


def test_jacobi_matches_lapack():
    rng = np.random.default_rng(5)
    for n in (1, 3, 17, 60):
        B = rng.standard_normal((n, n))
        A = B + B.T
        w, V = oracle.jacobi_eig(A)
        ref = np.linalg.eigvalsh(A)
        nrm = np.linalg.norm(A, 2)
        assert np.max(np.abs(w - ref)) <= 50 * EPS * nrm
        assert np.max(np.abs(V.T @ V - np.eye(n))) <= 50 * EPS * n
        assert np.max(np.abs(A @ V - V * w)) <= 50 * EPS * nrm * n


# --------------------------------------------------------------------------
# Root count (Sec. 2.1-2.2): #{mu < x}, by inertia, against dense eigenvalues
# --------------------------------------------------------------------------
@pytest.mark.parametrize("k,sigma", [(1, "psd"), (1, "nsd"), (2, "mixed"), (3, "mixed"), (4, "psd"),
                                     (5, "nsd")])
def test_count_matches_dense_spectrum(k, sigma):
    Q, lam, K, s = _problem(30, k, seed=11 + k, sigma=sigma, kscale=0.7)
    U = oracle.project(Q, K)
    ev = np.linalg.eigvalsh(oracle.updated_matrix(Q, lam, K, s))
    rng = np.random.default_rng(3)
    xs = rng.uniform(ev[0] - 1.0, ev[-1] + 1.0, size=300)
    gap = np.min(np.abs(xs[:, None] - ev[None, :]), axis=1)
    xs = xs[gap > 1e-9]
    for x in xs:
        assert oracle.count(lam, U, s, x) == int(np.sum(ev < x))


def test_count_origin_shift_agrees():
    Q, lam, K, s = _problem(40, 3, seed=4, sigma="mixed")
    U = oracle.project(Q, K)
    ev = np.linalg.eigvalsh(oracle.updated_matrix(Q, lam, K, s))
    for o in (0, 7, 39):
        for t in (-0.05, -1e-6, 1e-7, 0.03):
            x = lam[o] + t
            if np.min(np.abs(ev - x)) < 1e-10:
                continue
            assert oracle.count(lam, U, s, t, origin=o) == int(np.sum(ev < x))


def test_pole_count_matches_dense():
    for k, sg in [(1, "psd"), (2, "mixed"), (4, "psd"), (3, "nsd")]:
        Q, lam, K, s = _problem(25, k, seed=20 + k, sigma=sg)
        U = oracle.project(Q, K)
        ev = np.linalg.eigvalsh(oracle.updated_matrix(Q, lam, K, s))
        for p in range(25):
            assert oracle.pole_count(lam, U, s, p) == int(np.sum(ev < lam[p]))


def test_pole_count_repeated_pole():
    # lam = c I: n - k eigenvalues stay at c, the others move by eig(Sigma K^T K).
    Q, lam, K, s = _problem(20, 3, seed=2, sigma="mixed", lam_kind="constant")
    U = oracle.project(Q, K)
    ev = np.linalg.eigvalsh(oracle.updated_matrix(Q, lam, K, s))
    c = lam[0]
    assert oracle.pole_count(lam, U, s, 5) == int(np.sum(ev < c - 1e-12))


# --------------------------------------------------------------------------
# Eigenvalues (Sec. 2.3)
# --------------------------------------------------------------------------
def _textbook_rank1(lam, z, sigma):
    """Bisection on the rank-1 secular function of eq. (1), f = 1 + sigma sum z_j^2/(lam_j - x):
    for sigma > 0 root i lies in (lam_i, lam_{i+1}), the last in (lam_n, lam_n + |z|^2);
    mirrored for sigma < 0.  f is monotone on each interval."""
    n = lam.shape[0]
    nz = float(z @ z)
    out = np.zeros(n)
    for i in range(n):
        if sigma > 0:
            lo, hi = lam[i], (lam[i + 1] if i + 1 < n else lam[-1] + nz)
        else:
            lo, hi = (lam[i - 1] if i > 0 else lam[0] - nz), lam[i]
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if not (lo < mid < hi):
                break
            f = 1.0 + sigma * np.sum(z * z / (lam - mid))
            # f increases through the root on each interval (f' = sigma*sum z^2/(lam-x)^2 > 0 for sigma>0;
            # for sigma<0 f decreases)
            if (f < 0) == (sigma > 0):
                lo = mid
            else:
                hi = mid
        out[i] = 0.5 * (lo + hi)
    return out


@pytest.mark.parametrize("sigma", [1, -1])
def test_rank1_reduces_to_textbook_secular(sigma):
    Q, lam, K, _ = _problem(80, 1, seed=31, kscale=0.3)
    s = np.array([sigma], dtype=np.int8)
    out = oracle.update(Q, lam, K, s, want_vectors=False)
    z = (Q.T @ K)[:, 0]
    ref = _textbook_rank1(lam, z, sigma)
    assert np.max(np.abs(out["mu"] - ref)) <= 8 * EPS * np.max(np.abs(ref))


@pytest.mark.parametrize("n,k,sigma,kind", [(2, 1, "psd", "uniform"), (5, 2, "mixed", "uniform"),
                                            (9, 3, "nsd", "logspec"), (16, 4, "mixed", "uniform"),
                                            (16, 7, "psd", "clustered"), (12, 12, "mixed", "uniform"),
                                            (3, 6, "psd", "uniform")])
def test_brute_force_small(n, k, sigma, kind):
    Q, lam, K, s = _problem(n, k, seed=n * 10 + k, sigma=sigma, lam_kind=kind, kscale=0.5)
    out = oracle.update(Q, lam, K, s)
    A = oracle.updated_matrix(Q, lam, K, s)
    ref = np.linalg.eigvalsh(A)
    nrm = np.linalg.norm(A, 2)
    assert np.max(np.abs(out["mu"] - ref)) <= 1e-13 * nrm
    res = oracle.residuals(Q, lam, K, s, out["mu"], out["X"])
    assert np.max(res) <= 1e-11 * nrm
    assert oracle.orthogonality(out["X"]) <= 1e-11


@pytest.mark.parametrize("sigma", ["psd", "nsd", "mixed"])
def test_interlacing(sigma):
    k = 4
    Q, lam, K, s = _problem(120, k, seed=77, sigma=sigma, kscale=0.5)
    mu = oracle.update(Q, lam, K, s, want_vectors=False)["mu"]
    kp, km = int(np.sum(s > 0)), int(np.sum(s < 0))
    n = lam.shape[0]
    tol = 1e-14 * np.max(np.abs(lam))
    for m in range(n):
        if m - km >= 0:
            assert mu[m] >= lam[m - km] - tol
        if m + kp < n:
            assert mu[m] <= lam[m + kp] + tol


def test_trace_and_frobenius_identities():
    k = 6
    Q, lam, K, s = _problem(400, k, seed=8, sigma="mixed", lam_kind="logspec", kscale=0.2)
    mu = oracle.update(Q, lam, K, s, want_vectors=False)["mu"]
    S = s.astype(np.float64)
    U = Q.T @ K
    # trace: sum mu - sum lam = tr(Sigma K^T K)
    tr = float(np.sum(S * np.sum(K * K, axis=0)))
    scale = float(np.sum(np.abs(lam))) + float(np.sum(K * K))
    assert abs((np.sum(mu) - np.sum(lam)) - tr) <= 1e-13 * scale
    # Frobenius: sum mu^2 = sum lam^2 + 2 tr(Sigma U^T Lam U) + tr((Sigma U^T U)^2)
    SU = S[:, None] * (U.T @ U)
    fro = float(np.sum(lam * lam)) + 2.0 * float(np.sum(S * np.sum(U * (lam[:, None] * U), axis=0))) \
        + float(np.trace(SU @ SU))
    assert abs(float(np.sum(mu * mu)) - fro) <= 1e-12 * float(np.sum(lam * lam))


def test_characteristic_polynomial_identity():
    """prod(x - mu_i) = prod(x - lam_i) * det(I - Sigma U^T (xI - Lam)^{-1} U): the det form of eq. (1)."""
    k = 3
    Q, lam, K, s = _problem(300, k, seed=9, sigma="mixed", kscale=0.4)
    mu = oracle.update(Q, lam, K, s, want_vectors=False)["mu"]
    U = Q.T @ K
    S = np.diag(s.astype(np.float64))
    rng = np.random.default_rng(1)
    for x in rng.uniform(-2, 2, size=25):
        lhs = np.sum(np.log(np.abs(x - mu))) - np.sum(np.log(np.abs(x - lam)))
        f = np.linalg.det(np.eye(k) - S @ U.T @ (U / (x - lam)[:, None]))
        assert abs(lhs - math.log(abs(f))) <= 1e-9


def test_partial_fraction_form_with_corrected_residues():
    """Eq. (3): f(x) = 1 + sum_i alpha_i/(lam_i - x).  The residue of eq. (2) holds with its sign
    flipped: alpha_i = u_i^T adj(I + Sigma U^T D_i U) Sigma u_i, D_i = diag(1/(lam_j - lam_i)), j != i.
    The oracle's roots are zeros of this form."""
    k = 3
    Q, lam, K, s = _problem(40, k, seed=12, sigma="mixed", kscale=0.6)
    U = Q.T @ K
    S = np.diag(s.astype(np.float64))
    n = lam.shape[0]
    alpha = np.zeros(n)
    for i in range(n):
        d = np.zeros(n)
        msk = np.arange(n) != i
        d[msk] = 1.0 / (lam[msk] - lam[i])
        B = np.eye(k) + S @ U.T @ (U * d[:, None])
        adj = np.linalg.det(B) * np.linalg.inv(B)
        alpha[i] = U[i] @ adj @ S @ U[i]
        # the printed sign: det[[0, u^T],[u, B]] = -u^T adj(B) u  (Sigma = I case check below)

    def f_det(x):
        return np.linalg.det(np.eye(k) - S @ U.T @ (U / (x - lam)[:, None]))

    for x in np.random.default_rng(2).uniform(-1.5, 1.5, size=20):
        pf = 1.0 + np.sum(alpha / (lam - x))
        assert abs(pf - f_det(x)) <= 1e-10 * (1.0 + np.sum(np.abs(alpha / (lam - x))))
    mu = oracle.update(Q, lam, K, s, want_vectors=False)["mu"]
    for m in mu:
        terms = alpha / (lam - m)
        assert abs(1.0 + np.sum(terms)) <= 1e-9 * (1.0 + np.sum(np.abs(terms)))


def test_constant_spectrum_special_case():
    """Lam = c I: mu = c + eig(Sigma K^T K) plus n - k copies of c."""
    n, k = 30, 4
    Q, lam, K, s = _problem(n, k, seed=13, sigma="mixed", lam_kind="constant", kscale=0.5)
    mu = oracle.update(Q, lam, K, s, want_vectors=False)["mu"]
    c = lam[0]
    S = np.diag(s.astype(np.float64))
    G = K.T @ K
    L = np.linalg.cholesky(G)
    small = np.linalg.eigvalsh(L.T @ S @ L)  # same nonzero spectrum as K Sigma K^T
    ref = np.sort(np.concatenate([c + small, np.full(n - k, c)]))
    assert np.max(np.abs(mu - ref)) <= 1e-13 * (abs(c) + np.max(np.abs(small)))


def test_small_perturbation_matches_eq11():
    """Eq. (11): for small |K|, mu_j ~ lam_j + |K^T q_j|^2 with error O(|K|^4 / gap)."""
    n, k = 60, 3
    rng = np.random.default_rng(4)
    lam = np.arange(n, dtype=np.float64) * 0.1
    Q = workloads.haar(n, rng)
    K0 = rng.standard_normal((n, k))
    K0 /= np.linalg.norm(K0, 2)
    errs = []
    for scale in (1e-2, 1e-3):
        K = scale * K0
        mu = oracle.update(Q, lam, K, np.ones(k, np.int8), want_vectors=False)["mu"]
        first = lam + np.sum((Q.T @ K) ** 2, axis=1)
        errs.append(np.max(np.abs(mu - first)))
    # fourth-order: a 10x smaller K cuts the error by ~1e4
    assert errs[0] <= 50 * 1e-8 / 0.1
    assert errs[1] <= errs[0] * 1e-3


def test_rank2_canonicalisation():
    """Sec. 2.2 Steps 1-2: K Sigma K^T == e_j a^T + a e_j^T; trace identity gives 2 a_j."""
    n, j = 50, 17
    a = np.random.default_rng(6).standard_normal(n)
    K, s = oracle.rank2_perturbation(n, j, a)
    E = np.zeros((n, n))
    E[j, :] += a
    E[:, j] += a
    assert np.max(np.abs((K * s.astype(float)) @ K.T - E)) <= 8 * EPS * np.max(np.abs(a))
    assert abs(float(np.sum(s * np.sum(K * K, axis=0))) - 2 * a[j]) <= 16 * EPS * (1 + a @ a)


def test_indefinite_rank2_with_planted_deflation_and_clusters():
    P = workloads.indefinite_rank2(seed=1000, n=500)
    Q, lam = P["Q"], P["lam"]
    K, s = oracle.rank2_perturbation(500, P["j"], P["a"])
    out = oracle.update(Q, lam, K, s)
    assert set(np.nonzero(out["deflated"])[0]) == set(P["planted"].tolist())
    A = oracle.updated_matrix(Q, lam, K, s)
    ref = np.linalg.eigvalsh(A)
    nrm = np.linalg.norm(A, 2)
    assert np.max(np.abs(out["mu"] - ref)) <= 1e-12 * nrm
    res = oracle.residuals(Q, lam, K, s, out["mu"], out["X"])
    assert np.max(res) <= 1e-10 * nrm
    assert oracle.orthogonality(out["X"]) <= 1e-9


def test_eigenvectors_match_lapack_up_to_sign():
    Q, lam, K, s = _problem(150, 4, seed=21, sigma="mixed", kscale=0.5)
    out = oracle.update(Q, lam, K, s)
    w, V = np.linalg.eigh(oracle.updated_matrix(Q, lam, K, s))
    X = out["X"]
    gaps = np.minimum(np.diff(w, prepend=-np.inf), np.diff(w, append=np.inf))
    ok = gaps > 1e-6
    cosines = np.abs(np.sum(X[:, ok] * V[:, ok], axis=0))
    assert np.min(cosines) >= 1 - 1e-10


def test_sampled_roots_match_full_solve():
    Q, lam, K, s = _problem(200, 5, seed=3, sigma="mixed")
    full = oracle.update(Q, lam, K, s)
    sel = np.array([0, 3, 77, 199])
    part = oracle.update(Q, lam, K, s, sel=sel)
    assert np.array_equal(part["pos"], sel)
    assert np.max(np.abs(part["mu"] - full["mu"][sel])) == 0.0
    assert np.max(np.abs(np.abs(part["X"]) - np.abs(full["X"][:, sel]))) <= 1e-13


@pytest.mark.parametrize("seed,sigma", [(91, "mixed"), (92, "psd")])
def test_update_with_a_spiked_perturbation_matches_lapack(seed, sigma):
    """One row of K scaled by 2^61: every row of U carries a component 2^61
    times the rest, and ||U||^2 is ~2^114 times the spread of lambda.  The
    oracle's eigenvalues still match LAPACK's symmetric eigensolver on
    diag(lam) + U Sigma U^T to 1e-14 of |A| = max|lam| + ||U||_F^2 (LAPACK's own
    error is a few units of eps |A|)."""
    P = workloads.general(600, 5, seed=seed, sigma=sigma, lam_kind="uniform")
    K = P["K"].copy()
    K[17, :] *= 2.0 ** 61
    U = P["Q"].T @ K
    ref = np.linalg.eigvalsh(np.diag(P["lam"]) + (U * P["sigma"].astype(float)) @ U.T)
    normA = np.max(np.abs(P["lam"])) + np.sum(U * U)
    r = oracle.update(P["Q"], P["lam"], K, P["sigma"], want_vectors=False)
    assert np.max(np.abs(r["mu"] - ref)) <= 1e-14 * normA
