"""Pins of the oracle's first-order perturbation estimate (eq. (11)) and the
Figs. 6-7 comparison it serves.

Checked against a 2 x 2 closed form (textbook eigenpairs), an exact special
case (K inside the eigenbasis), the fourth-order error law of first-order
perturbation theory, and dense LAPACK decompositions.
"""
import math

import numpy as np
import pytest

import oracle
import workloads


def _exact_2x2(l1, l2, E):
    """Eigenpairs of diag(l1, l2) + E (E symmetric, l1 < l2) in closed form; the
    eigenvector of the lower eigenvalue from the second row of (A - lo I) v = 0,
    v = (lo - c, b), which has no cancellation."""
    a, b, c = l1 + E[0, 0], E[0, 1], l2 + E[1, 1]
    m, r = 0.5 * (a + c), math.hypot(0.5 * (a - c), b)
    lo, hi = m - r, m + r
    v = np.array([lo - c, b])
    return (lo, hi), v / np.linalg.norm(v)


def test_two_by_two_first_order_error_is_fourth_order_in_K():
    l1, l2 = -0.3, 0.5
    k = np.array([[0.7], [-0.4]])
    errs = []
    for eps in (1e-2, 5e-3, 2.5e-3):
        K = eps * k
        mu, X = oracle.perturbation(np.eye(2), np.array([l1, l2]), K)
        (lo, hi), v = _exact_2x2(l1, l2, K @ K.T)
        x = X[:, 0] / np.linalg.norm(X[:, 0])
        errs.append((abs(mu[0] - lo), min(np.linalg.norm(x - v), np.linalg.norm(x + v))))
    for (e0, v0), (e1, v1) in zip(errs, errs[1:]):
        assert 12 < e0 / e1 < 20  # eigenvalue error ~ |K|^4
        assert 12 < v0 / v1 < 20  # eigenvector error ~ |K|^4 (a wrong sign would give |K|^2)


def test_K_inside_the_eigenbasis_is_exact():
    """K = Q[:, S] D makes U Sigma U^T diagonal: mu_j = lam_j + sigma d_j^2 on S,
    W = I, and the estimate is the exact decomposition."""
    P = workloads.small_k(n=40, k=3, knorm=0.5, seed=5)
    Q, lam = P["Q"], P["lam"]
    S = [3, 17, 31]
    K = Q[:, S] * np.array([0.2, -0.3, 0.1])[None, :]
    sig = np.array([1, -1, 1], dtype=np.int8)
    mu, X = oracle.perturbation(Q, lam, K, sig)
    want = lam.copy()
    want[S] += sig * np.array([0.04, 0.09, 0.01])
    assert np.max(np.abs(mu - want)) <= 1e-15
    assert np.max(np.abs(X - Q)) <= 1e-15
    m = oracle.fig67_metrics(Q, lam, K, sig, mu, X)
    assert m["A"] <= 1e-14 and m["B"] <= 1e-14 and m["C"] <= 1e-13


def test_eigenvalue_error_scales_as_fourth_power():
    errs = []
    for knorm in (0.02, 0.01, 0.005):
        P = workloads.small_k(n=30, k=2, knorm=knorm, seed=8)
        mu, _ = oracle.perturbation(P["Q"], P["lam"], P["K"], P["sigma"])
        w = np.linalg.eigvalsh(oracle.updated_matrix(P["Q"], P["lam"], P["K"], P["sigma"]))
        errs.append(np.max(np.abs(np.sort(mu) - w)))
    assert 12 < errs[0] / errs[1] < 20 and 12 < errs[1] / errs[2] < 20


@pytest.mark.parametrize("k", [1, 2, 5, 10])
def test_figs_6_7_shape(k):
    """N = 100: at |K| = 0.01 the perturbation estimate is close; at 0.3 it
    fails on all three accuracy panels while the method's result does not
    change with |K|."""
    small = workloads.small_k(n=100, k=k, knorm=0.01, seed=600 + k)
    large = workloads.small_k(n=100, k=k, knorm=0.3, seed=600 + k)
    res = {}
    for tag, P in (("0.01", small), ("0.3", large)):
        mu, X = oracle.perturbation(P["Q"], P["lam"], P["K"], P["sigma"])
        res[tag, "pert"] = oracle.fig67_metrics(P["Q"], P["lam"], P["K"], P["sigma"], mu, X)
        out = oracle.update(P["Q"], P["lam"], P["K"], P["sigma"])
        res[tag, "method"] = oracle.fig67_metrics(P["Q"], P["lam"], P["K"], P["sigma"], out["mu"], out["X"])
    for tag in ("0.01", "0.3"):
        assert max(res[tag, "method"].values()) <= 1e-12
    assert max(res["0.01", "pert"].values()) <= 1e-3
    for panel in "ABC":
        assert res["0.3", "pert"][panel] >= 30 * res["0.01", "pert"][panel]
        assert res["0.3", "pert"][panel] >= 1e-4
