"""GPU parity on exactly repeated eigenvalues (runs of equal lam, some longer
than k), through the C ABI, in both precision modes and every entry point that
deflates: the full update (in place and with Q_out), the batch, the interval
query, and the two eigenvalue-only calls.

Eigenvalues are compared with the oracle; a repeated eigenvalue's eigenvectors
are not unique, so eigenvectors are compared as subspaces per cluster of equal
eigenvalues, and every pair is checked for residual and orthogonality.
"""
import numpy as np
import pytest

import oracle
import workloads
from gpu_util import dev_colmajor, dev_vec, host, norm2_A

pytestmark = pytest.mark.gpu

MU_TOL = 1e-13   # x ||A'||: the secular problem after the rotation is an ordinary one
RES_TOL = {0: 1e-12, 1: 1e-10}   # mode -> residual / orthogonality bound (split-BF16 GEMM in mode 1)
SUB_TOL = {0: 1e-9, 1: 1e-8}


@pytest.fixture(scope="module")
def eu():
    import paper_1706_00773_gb300 as m

    return m


@pytest.fixture(scope="module", params=[0, 1], ids=["fp64", "mixed"])
def mode_handle(eu, request):
    h = eu.eig_update_init(0, request.param)
    yield request.param, h
    eu.eig_update_destroy(h)


def _clusters(mu, tol):
    out, i = [], 0
    while i < len(mu):
        j = i + 1
        while j < len(mu) and mu[j] - mu[j - 1] <= tol:
            j += 1
        out.append((i, j))
        i = j
    return out


def _check(P, mu, X, mode, ref=None):
    ref = ref or oracle.update(P["Q"], P["lam"], P["K"], P["sigma"])
    scale = norm2_A(P["lam"], P["K"])
    assert np.all(np.diff(mu) >= 0)
    assert np.max(np.abs(mu - ref["mu"])) <= MU_TOL * scale
    n = len(mu)
    if X is not None:
        res = oracle.residuals(P["Q"], P["lam"], P["K"], P["sigma"], mu, X)
        assert np.max(res) <= RES_TOL[mode] * scale
        assert np.max(np.abs(X.T @ X - np.eye(n))) <= RES_TOL[mode]
        for i, j in _clusters(ref["mu"], 1e-9 * scale):
            s = np.linalg.svd(X[:, i:j].T @ ref["X"][:, i:j], compute_uv=False)
            assert 1.0 - np.min(s) <= SUB_TOL[mode]
    return ref


def _run(eu, h, P, Q_out=False):
    import torch

    Q, lam, K = dev_colmajor(P["Q"]), dev_vec(P["lam"]), dev_colmajor(P["K"])
    Qo = torch.empty_like(Q) if Q_out else None
    rc, rep = eu.eig_update_rank_k(h, Q, lam, K, P["sigma"], eu.EIG_VALUES | eu.EIG_VECTORS | eu.EIG_REPORT,
                                   Q_out=Qo)
    torch.cuda.synchronize()
    if Q_out:
        assert np.array_equal(host(Q), P["Q"])  # input untouched, bit for bit
        return rc, rep, host(lam), host(Qo)
    return rc, rep, host(lam), host(Q)


@pytest.mark.parametrize("n,k,sigma", [(257, 1, "psd"), (300, 3, "mixed"), (700, 8, "nsd"), (1100, 5, "mixed")])
def test_repeated_spectrum_full_update(eu, mode_handle, n, k, sigma):
    mode, h = mode_handle
    P = workloads.general(n, k, seed=900 + n + k, sigma=sigma, lam_kind="repeated", kscale=0.3)
    runs = oracle.repeated_runs(P["lam"])
    assert any(m > k for _, m in runs)
    rc, rep, mu, X = _run(eu, h, P)
    assert rc == 0 and rep["n_notconv"] == 0
    assert rep["n_runs"] == len(runs)
    assert rep["n_deflated"] >= sum(max(0, m - k) for _, m in runs)
    _check(P, mu, X, mode)


@pytest.mark.parametrize("sigma", ["psd", "mixed"])
@pytest.mark.parametrize("q_out", [False, True], ids=["inplace", "q_out"])
def test_update_of_the_zero_matrix(eu, mode_handle, sigma, q_out):
    """A = 0 (Q = I, lam = 0), one run of length n: A' = K Sigma K^T, whose
    other n - k eigenvalues are exactly 0 with eigenvectors orthogonal to K."""
    mode, h = mode_handle
    n, k = 600, 6
    P = workloads.general(n, k, seed=31, sigma=sigma, kscale=0.5)
    P["Q"], P["lam"] = np.eye(n), np.zeros(n)
    rc, rep, mu, X = _run(eu, h, P, Q_out=q_out)
    assert rc == 0 and rep["n_runs"] == 1 and rep["n_deflated"] == n - k
    assert int(np.sum(mu == 0.0)) == n - k
    _check(P, mu, X, mode)
    Z = X[:, mu == 0.0]
    assert np.max(np.abs(P["K"].T @ Z)) <= RES_TOL[mode] * np.max(np.abs(P["K"])) * 10


def test_rank_deficient_run_keeps_exact_multiplicity(eu, mode_handle):
    mode, h = mode_handle
    n, k, m = 400, 4, 9
    rng = np.random.default_rng(17)
    Q = workloads.haar(n, rng)
    lam = np.sort(rng.uniform(-1, 1, n))
    g0 = 150
    lam[g0:g0 + m] = lam[g0]
    U = rng.standard_normal((n, k)) * 0.05
    U[g0:g0 + m] = np.outer(rng.standard_normal(m), rng.standard_normal(k)) * 0.05  # rank 1
    P = dict(Q=Q, lam=lam, K=Q @ U, sigma=np.array([1, -1, 1, 1], np.int8))
    rc, rep, mu, X = _run(eu, h, P)
    assert rc == 0
    assert int(np.sum(mu == lam[g0])) == m - 1
    _check(P, mu, X, mode)


def test_batch_mixes_runs_and_distinct(eu, mode_handle):
    import torch

    mode, h = mode_handle
    Ps = [workloads.general(n, k, seed=70 + n, sigma="mixed", lam_kind=kind, kscale=0.3)
          for n, k, kind in [(200, 2, "repeated"), (333, 4, "uniform"), (450, 7, "repeated"), (128, 1, "constant")]]
    devs = [dict(Q=dev_colmajor(P["Q"]), lam=dev_vec(P["lam"]), K=dev_colmajor(P["K"]), sigma=P["sigma"])
            for P in Ps]
    tickets = eu.eig_update_batch(h, devs)
    torch.cuda.synchronize()
    for t, P, d in zip(tickets, Ps, devs):
        assert eu.eig_update_query(h, eu.EIG_Q_STATUS, t) == 0
        _check(P, host(d["lam"]), host(d["Q"]), mode)


def test_select_on_a_repeated_spectrum(eu, mode_handle):
    import torch

    mode, h = mode_handle
    P = workloads.general(500, 3, seed=5, sigma="mixed", lam_kind="repeated", kscale=0.3)
    ref = oracle.update(P["Q"], P["lam"], P["K"], P["sigma"])
    runs = [(g0, m) for g0, m in oracle.repeated_runs(P["lam"]) if m > 3]
    g0, m = runs[len(runs) // 2]
    vl = 0.5 * (P["lam"][g0 - 1] + P["lam"][g0]) if g0 > 0 else -np.inf
    j = min(g0 + m + 20, 499)
    while P["lam"][j - 1] == P["lam"][j]:
        j -= 1
    vu = 0.5 * (P["lam"][j - 1] + P["lam"][j])  # between two distinct poles
    sel = np.nonzero((ref["mu"] >= vl) & (ref["mu"] < vu))[0]
    n = 500
    mu = torch.full((n,), np.nan, dtype=torch.float64, device="cuda:0")
    X = torch.empty((n, n), dtype=torch.float64, device="cuda:0").t()
    rc, cnt = eu.eig_update_select(h, dev_colmajor(P["Q"]), dev_vec(P["lam"]), dev_colmajor(P["K"]), P["sigma"],
                                   vl, vu, mu, X)
    torch.cuda.synchronize()
    assert rc == 0 and cnt == len(sel)
    mu_s, X_s = host(mu)[:cnt], host(X)[:, :cnt]
    scale = norm2_A(P["lam"], P["K"])
    assert np.max(np.abs(mu_s - ref["mu"][sel])) <= MU_TOL * scale
    res = oracle.residuals(P["Q"], P["lam"], P["K"], P["sigma"], mu_s, X_s)
    assert np.max(res) <= RES_TOL[mode] * scale
    assert np.max(np.abs(X_s.T @ X_s - np.eye(cnt))) <= RES_TOL[mode]
    for i, j in _clusters(ref["mu"][sel], 1e-9 * scale):
        s = np.linalg.svd(X_s[:, i:j].T @ ref["X"][:, sel[i:j]], compute_uv=False)
        assert 1.0 - np.min(s) <= SUB_TOL[mode]


def test_eigenvalue_only_calls_on_runs(eu, mode_handle):
    """eig_secular_values and eig_secular_values_static rotate a copy of U and
    leave the caller's U as it was."""
    import torch

    mode, h = mode_handle
    P = workloads.general(640, 5, seed=12, sigma="mixed", lam_kind="repeated", kscale=0.3)
    U = oracle.project(P["Q"], P["K"])
    ref = oracle.update(P["Q"], P["lam"], P["K"], P["sigma"], want_vectors=False)["mu"]
    scale = norm2_A(P["lam"], P["K"])
    Ud = dev_colmajor(U)
    mu = torch.empty(640, dtype=torch.float64, device="cuda:0")
    assert eu.eig_secular_values(h, dev_vec(P["lam"]), Ud, P["sigma"], mu) == 0
    torch.cuda.synchronize()
    assert np.max(np.abs(host(mu) - ref)) <= MU_TOL * scale
    assert np.array_equal(host(Ud), U)
    mu2 = torch.empty(640, dtype=torch.float64, device="cuda:0")
    assert eu.eig_secular_values_static(dev_vec(P["lam"]), Ud, P["sigma"], mu2) == 0
    torch.cuda.synchronize()
    assert np.array_equal(host(mu2), host(mu))
    assert np.array_equal(host(Ud), U)
