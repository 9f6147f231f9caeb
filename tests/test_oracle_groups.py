"""Pins of the oracle on exactly repeated eigenvalues.

The paper assumes distinct lam (Sec. 2.1).  The oracle rotates each run of
equal lam inside its eigenspace (``oracle.group_rotate``) before deflation.
These tests pin that step against what the mathematics fixes: A itself is
unchanged, the dense spectrum of A' (numpy LAPACK), the closed form of an
update of the zero matrix, the exact multiplicity that a rank-deficient run
leaves behind, and residual/orthogonality of every returned pair.  A basis of
a repeated eigenvalue's eigenspace is not unique, so eigenvectors of repeated
eigenvalues are compared as subspaces.
"""
import numpy as np
import pytest

import oracle
import workloads

EPS = np.finfo(np.float64).eps


def _clusters(mu, tol):
    """Runs of eigenvalues closer than tol (index ranges)."""
    out, i = [], 0
    while i < len(mu):
        j = i + 1
        while j < len(mu) and mu[j] - mu[j - 1] <= tol:
            j += 1
        out.append((i, j))
        i = j
    return out


def subspace_gap(X, Y):
    """1 - smallest cosine of the principal angles between span X and span Y."""
    s = np.linalg.svd(X.T @ Y, compute_uv=False)
    return 1.0 - float(np.min(s))


def test_repeated_runs_finds_exact_runs_only():
    lam = np.array([-1.0, -1.0, 0.0, np.nextafter(0.0, 1.0), 0.5, 0.5, 0.5, 2.0])
    assert oracle.repeated_runs(lam) == [(0, 2), (4, 3)]
    assert oracle.repeated_runs(np.array([3.0])) == []
    assert oracle.repeated_runs(np.full(5, 7.0)) == [(0, 5)]


@pytest.mark.parametrize("k", [1, 3, 6])
def test_group_rotation_leaves_A_unchanged(k):
    P = workloads.general(80, k, seed=40 + k, sigma="mixed", lam_kind="repeated")
    Q, lam, K = P["Q"], P["lam"], P["K"]
    U = oracle.project(Q, K)
    Qt, Ut = oracle.group_rotate(Q, lam, U)
    runs = oracle.repeated_runs(lam)
    assert any(m > k for _, m in runs)  # the workload has runs longer than k
    A0 = (Q * lam) @ Q.T
    assert np.max(np.abs((Qt * lam) @ Qt.T - A0)) <= 1e-14 * np.max(np.abs(lam)) * 10
    assert np.max(np.abs(Qt.T @ Qt - np.eye(80))) <= 1e-14 * 10
    assert np.max(np.abs(Qt.T @ K - Ut)) <= 1e-14 * 10 * np.max(np.abs(U))  # U~ = Q~^T K
    inrun = np.zeros(80, bool)
    for g0, m in runs:
        inrun[g0:g0 + m] = True
        assert np.all(Ut[g0 + min(m, k):g0 + m] == 0.0)  # rows past min(m, k) vanish
        # the run keeps its Gram matrix (U_G^T U_G = R^T R)
        G = U[g0:g0 + m].T @ U[g0:g0 + m]
        assert np.max(np.abs(Ut[g0:g0 + m].T @ Ut[g0:g0 + m] - G)) <= 1e-14 * 10 * max(1.0, np.max(np.abs(G)))
    assert np.array_equal(Ut[~inrun], U[~inrun])  # other rows untouched, bit for bit
    assert np.array_equal(Qt[:, ~inrun], Q[:, ~inrun])


@pytest.mark.parametrize("n,k,sigma", [(60, 1, "psd"), (90, 3, "mixed"), (120, 5, "nsd"), (70, 8, "mixed")])
def test_repeated_spectrum_matches_dense_eigensolver(n, k, sigma):
    P = workloads.general(n, k, seed=300 + n + k, sigma=sigma, lam_kind="repeated", kscale=0.4)
    Q, lam, K, s = P["Q"], P["lam"], P["K"], P["sigma"]
    A = oracle.updated_matrix(Q, lam, K, s)
    scale = np.linalg.norm(A, 2)
    ref = np.linalg.eigvalsh(A)
    out = oracle.update(Q, lam, K, s)
    mu, X = out["mu"], out["X"]
    assert np.all(np.diff(mu) >= 0)
    assert np.max(np.abs(mu - ref)) <= 1e-13 * scale
    assert np.max(oracle.residuals(Q, lam, K, s, mu, X)) <= 1e-12 * scale
    assert np.max(np.abs(X.T @ X - np.eye(n))) <= 1e-12
    # every run longer than k leaves at least m - k pairs at lam, deflated
    extra = sum(max(0, m - k) for _, m in oracle.repeated_runs(lam))
    assert int(np.sum(out["deflated"])) >= extra
    # eigenspaces against LAPACK's, cluster by cluster
    w, V = np.linalg.eigh(A)
    for i, j in _clusters(ref, 1e-9 * scale):
        assert subspace_gap(X[:, i:j], V[:, i:j]) <= 1e-8


@pytest.mark.parametrize("sigma", ["psd", "mixed"])
def test_update_of_the_zero_matrix(sigma):
    """A = 0 (Q = I, lam = 0): A' = K Sigma K^T, whose nonzero eigenvalues are
    those of Sigma K^T K's symmetric form and whose other n - k are exactly 0."""
    n, k = 50, 4
    P = workloads.general(n, k, seed=77, sigma=sigma, kscale=0.7)
    K, s = P["K"], P["sigma"]
    Q, lam = np.eye(n), np.zeros(n)
    out = oracle.update(Q, lam, K, s)
    S = np.diag(s.astype(np.float64))
    L = np.linalg.cholesky(K.T @ K)
    small = np.linalg.eigvalsh(L.T @ S @ L)
    ref = np.sort(np.concatenate([small, np.zeros(n - k)]))
    mu = out["mu"]
    assert np.max(np.abs(mu - ref)) <= 1e-13 * np.max(np.abs(small))
    assert int(np.sum(mu == 0.0)) == n - k  # the untouched part of the eigenspace is exact
    X = out["X"]
    assert np.max(np.abs(X.T @ X - np.eye(n))) <= 1e-13
    # the zero eigenspace is the orthogonal complement of range(K)
    Z = X[:, mu == 0.0]
    assert np.max(np.abs(K.T @ Z)) <= 1e-13 * np.max(np.abs(K))


def test_rank_deficient_run_keeps_exact_multiplicity():
    """A run of m = 5 equal lam whose rows of U have rank 1 (k = 3): m - 1 = 4
    eigenvalues stay exactly at lam, one moves."""
    n, k, m, g0 = 40, 3, 5, 17
    rng = np.random.default_rng(5)
    Q = workloads.haar(n, rng)
    lam = np.sort(rng.uniform(-1, 1, n))
    lam[g0:g0 + m] = lam[g0]
    lam = np.sort(lam)
    g0 = int(np.nonzero(lam == lam[g0])[0][0])
    U = rng.standard_normal((n, k)) * 0.3
    U[g0:g0 + m] = np.outer(rng.standard_normal(m), rng.standard_normal(k)) * 0.3
    K = Q @ U
    s = np.array([1, -1, 1], np.int8)
    out = oracle.update(Q, lam, K, s)
    assert int(np.sum(out["mu"] == lam[g0])) == m - 1
    A = oracle.updated_matrix(Q, lam, K, s)
    assert np.max(np.abs(out["mu"] - np.linalg.eigvalsh(A))) <= 1e-13 * np.linalg.norm(A, 2)
    assert np.max(oracle.residuals(Q, lam, K, s, out["mu"], out["X"])) <= 1e-12 * np.linalg.norm(A, 2)


def test_runs_not_longer_than_k_need_no_rotation():
    """With every run at most k long and full-rank rows the rotated problem has
    the same roots as the unrotated one (both solved by the oracle)."""
    rng = np.random.default_rng(9)
    n, k = 30, 4
    Q = workloads.haar(n, rng)
    lam = np.repeat(np.sort(rng.uniform(-1, 1, 10)), 3)
    K = rng.standard_normal((n, k)) * 0.3
    s = np.array([1, 1, -1, 1], np.int8)
    U = oracle.project(Q, K)
    mu_plain = oracle.roots(lam, U, s)["mu"]
    mu_rot = oracle.update(Q, lam, K, s, want_vectors=False)["mu"]
    A = oracle.updated_matrix(Q, lam, K, s)
    sc = np.linalg.norm(A, 2)
    assert np.max(np.abs(np.sort(mu_plain) - mu_rot)) <= 1e-13 * sc
    assert np.max(np.abs(mu_rot - np.linalg.eigvalsh(A))) <= 1e-13 * sc


def test_planted_transpose_in_the_rotation_is_caught(monkeypatch):
    """A plausible slip: rotating Q by H^T instead of H.  The dense-spectrum
    pin passes (values depend on U~ only), the residual pin must not."""
    real_qr = np.linalg.qr

    def bad_group_rotate(Q, lam, U):
        Qt, Ut = np.array(Q, copy=True), np.array(U, copy=True)
        k = Ut.shape[1]
        for g0, m in oracle.repeated_runs(lam):
            H, R = real_qr(Ut[g0:g0 + m], mode="complete")
            R[min(m, k):] = 0.0
            Ut[g0:g0 + m] = R
            Qt[:, g0:g0 + m] = Qt[:, g0:g0 + m] @ H.T
        return Qt, Ut

    monkeypatch.setattr(oracle, "group_rotate", bad_group_rotate)
    P = workloads.general(60, 3, seed=11, sigma="mixed", lam_kind="repeated", kscale=0.4)
    Q, lam, K, s = P["Q"], P["lam"], P["K"], P["sigma"]
    out = oracle.update(Q, lam, K, s)
    A = oracle.updated_matrix(Q, lam, K, s)
    assert np.max(oracle.residuals(Q, lam, K, s, out["mu"], out["X"])) > 1e-6 * np.linalg.norm(A, 2)
