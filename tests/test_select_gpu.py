"""GPU parity of the interval query: eigenpairs with eigenvalues in [vl, vu)
(the location sub-problem alone decides which roots, Sec. 2.1; a subset of
eigenvectors, Sec. 3)."""
import numpy as np
import pytest

import oracle
import workloads
from gpu_util import dev_colmajor, dev_vec, host, norm2_A

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eu():
    import paper_1706_00773_gb300 as m

    return m


@pytest.fixture(scope="module")
def handle(eu):
    h = eu.eig_update_init(0, eu.EIG_FP64)
    yield h
    eu.eig_update_destroy(h)


def _select(eu, h, P, vl, vu, max_m=None, vectors=True):
    import torch

    n = P["Q"].shape[0]
    max_m = n if max_m is None else max_m
    Q, lam, K = dev_colmajor(P["Q"]), dev_vec(P["lam"]), dev_colmajor(P["K"])
    mu = torch.full((max(max_m, 1),), np.nan, dtype=torch.float64, device="cuda:0")[:max_m]
    X = torch.empty((max(max_m, 1), n), dtype=torch.float64, device="cuda:0").t()[:, :max_m] if vectors else None
    rc, m = eu.eig_update_select(h, Q, lam, K, P["sigma"], vl, vu, mu, X)
    torch.cuda.synchronize()
    assert np.array_equal(host(lam), P["lam"])  # inputs untouched
    return rc, m, host(mu)[:m], (host(X)[:, :m] if vectors else None)


def _full(eu, h, P):
    import torch

    Q, lam, K = dev_colmajor(P["Q"]), dev_vec(P["lam"]), dev_colmajor(P["K"])
    rc, _ = eu.eig_update_rank_k(h, Q, lam, K, P["sigma"], eu.EIG_VALUES | eu.EIG_VECTORS)
    torch.cuda.synchronize()
    assert rc == 0
    return host(lam), host(Q)


@pytest.mark.parametrize("n,k,sigma,kind", [(200, 2, "mixed", "uniform"), (517, 5, "psd", "logspec"),
                                            (900, 8, "nsd", "clustered"), (1300, 12, "mixed", "uniform")])
def test_select_equals_the_full_update_on_the_interval(eu, handle, n, k, sigma, kind):
    P = workloads.general(n, k, seed=1500 + n, sigma=sigma, lam_kind=kind)
    mu_all, X_all = _full(eu, handle, P)
    rng = np.random.default_rng(n)
    a, b = np.sort(rng.choice(np.arange(1, n), 2, replace=False))

    def mid(i):  # between computed eigenvalues i-1 and i: no count ambiguity
        return 0.5 * (mu_all[i - 1] + mu_all[i])

    cases = [(mid(a), mid(b)), (-np.inf, mid(n // 3)), (mid(2 * n // 3), np.inf), (-np.inf, np.inf)]
    for vl, vu in cases:
        rc, m, mu, X = _select(eu, handle, P, vl, vu)
        assert rc == 0
        sel = np.nonzero((mu_all >= vl) & (mu_all < vu))[0]
        assert m == len(sel)
        assert np.array_equal(mu, mu_all[sel])  # the same zero-finder path, bit for bit
        assert np.max(np.abs(X - X_all[:, sel]), initial=0.0) <= 1e-13


def test_select_against_dense_spectrum_and_deflation(eu, handle):
    """Planted deflated pairs inside the interval are merged in order."""
    P = workloads.general(400, 3, seed=71, sigma="mixed", lam_kind="uniform")
    Q = P["Q"]
    P["K"][:, :] = P["K"] - Q[:, 50:60] @ (Q[:, 50:60].T @ P["K"])  # rows 50..59 of U vanish
    w = np.linalg.eigvalsh(oracle.updated_matrix(Q, P["lam"], P["K"], P["sigma"]))
    vl, vu = P["lam"][48], P["lam"][65]
    rc, m, mu, X = _select(eu, handle, P, vl, vu)
    assert rc == 0
    ref = w[(w >= vl) & (w < vu)]
    assert m == len(ref)
    assert np.max(np.abs(mu - ref)) <= 1e-13 * norm2_A(P["lam"], P["K"])
    assert np.all(np.diff(mu) >= 0)
    res = oracle.residuals(Q, P["lam"], P["K"], P["sigma"], mu, X)
    assert np.max(res) <= 1e-12 * norm2_A(P["lam"], P["K"])
    assert np.max(np.abs(X.T @ X - np.eye(m))) <= 1e-12


def test_select_capacity_values_only_and_empty(eu, handle):
    P = workloads.general(300, 4, seed=9, sigma="psd")
    rc, m, _, _ = _select(eu, handle, P, -0.5, 0.5, max_m=3)
    assert rc == eu.EIG_ETOOBIG and m > 3
    rc2, m2, mu, X = _select(eu, handle, P, -0.5, 0.5, max_m=m, vectors=False)
    assert rc2 == 0 and m2 == m and X is None
    w = np.linalg.eigvalsh(oracle.updated_matrix(P["Q"], P["lam"], P["K"], P["sigma"]))
    assert np.max(np.abs(mu - w[(w >= -0.5) & (w < 0.5)])) <= 1e-13
    gap_lo = 10.0  # beyond every eigenvalue: nothing selected
    rc3, m3, _, _ = _select(eu, handle, P, gap_lo, gap_lo + 1.0)
    assert rc3 == 0 and m3 == 0
    with pytest.raises(eu.EigError):
        _select(eu, handle, P, 0.5, -0.5)  # vl >= vu


def test_select_full_size_sampled(eu, handle):
    """n = 8192, k = 8: about a hundred eigenpairs in the middle of the
    spectrum against the oracle."""
    P = workloads.general_rank_k(k=8, seed=2000, n=8192, device="cuda:0")
    U = oracle.project(P["Q"], P["K"])
    lam = P["lam"]
    assert not np.any(oracle.deflation_mask(lam, U))  # root indices are spectrum indices
    vl, vu = lam[4000], lam[4100]
    rc, m, mu, X = _select(eu, handle, P, vl, vu)
    assert rc == 0 and m > 10
    i0 = oracle.pole_count(lam, U, P["sigma"], 4000)  # the interval ends are poles
    assert oracle.pole_count(lam, U, P["sigma"], 4100) - i0 == m
    sel = np.arange(i0, i0 + m)
    ref = oracle.update(P["Q"], lam, P["K"], P["sigma"], sel=sel)
    scale = norm2_A(lam, P["K"])
    assert np.max(np.abs(mu - ref["mu"])) <= 1e-13 * scale
    cos = np.abs(np.sum(X * ref["X"], axis=0))
    assert np.min(cos) >= 1 - 1e-9


def test_select_mixed_mode_equals_the_full_mixed_update(eu):
    """Mixed mode: the interval's zero finder runs the FP32 coarse phase and the
    certified FP32 pole counts exactly like the full update, so the selected
    eigenvalues are the full update's, bit for bit; X_sel comes from the same
    split-BF16 tensor-core GEMM as X.  The full update splits each W entry
    straight from its unnormalised value, the interval query from the stored
    unit column, so a digit may round once more: at most 2^-39 per entry of
    W, a few units of 1e-12 in X."""
    import torch

    h = eu.eig_update_init(0, eu.EIG_MIXED)
    try:
        for n, k, sigma, kind in [(900, 8, "psd", "logspec"), (1300, 5, "mixed", "clustered")]:
            P = workloads.general(n, k, seed=1600 + n, sigma=sigma, lam_kind=kind)
            mu_all, X_all = _full(eu, h, P)
            mid = lambda i: 0.5 * (mu_all[i - 1] + mu_all[i])  # noqa: E731
            for vl, vu in [(mid(n // 4), mid(n // 4 + 60)), (-np.inf, mid(40))]:
                rc, m, mu, X = _select(eu, h, P, vl, vu)
                assert rc == 0
                sel = np.nonzero((mu_all >= vl) & (mu_all < vu))[0]
                assert m == len(sel)
                assert np.array_equal(mu, mu_all[sel])
                assert np.max(np.abs(X - X_all[:, sel])) <= 1e-11
    finally:
        eu.eig_update_destroy(h)
