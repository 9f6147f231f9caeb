"""GPU parity of the first-order perturbation estimate (eq. (11)), the
comparison method of Figs. 6-7, in both arithmetic modes."""
import numpy as np
import pytest

import oracle
import workloads
from gpu_util import dev_colmajor, dev_vec, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eu():
    import paper_1706_00773_gb300 as m

    return m


@pytest.fixture(scope="module", params=["fp64", "mixed"])
def handle(eu, request):
    h = eu.eig_update_init(0, eu.EIG_MIXED if request.param == "mixed" else eu.EIG_FP64)
    yield h
    eu.eig_update_destroy(h)


def _run(eu, h, P, alias=False):
    import torch

    n = P["Q"].shape[0]
    Q, lam, K = dev_colmajor(P["Q"]), dev_vec(P["lam"]), dev_colmajor(P["K"])
    mu = lam if alias else torch.empty(n, dtype=torch.float64, device="cuda:0")
    X = torch.empty((n, n), dtype=torch.float64, device="cuda:0").t()
    eu.eig_perturbation(h, Q, lam, K, P["sigma"], mu, X)
    torch.cuda.synchronize()
    return host(mu), host(X)


# FP64: the GEMM's rounding, n eps |Q| |W|; mixed: 5 BF16 slices keep ~2^-40 of
# each row / column scale.  Both well under 1e-10 of max |W| at these sizes.
X_TOL = 1e-10


@pytest.mark.parametrize("k", [1, 2, 5, 10])
@pytest.mark.parametrize("knorm", [0.01, 0.3])
def test_perturbation_matches_oracle_and_reproduces_figs_6_7(eu, handle, k, knorm):
    P = workloads.small_k(n=100, k=k, knorm=knorm, seed=600 + k)
    mu, X = _run(eu, handle, P)
    mu_ref, X_ref = oracle.perturbation(P["Q"], P["lam"], P["K"], P["sigma"])
    assert np.max(np.abs(mu - mu_ref)) <= 1e-14
    Wmax = np.max(np.abs(P["Q"].T @ X_ref))
    assert np.max(np.abs(X - X_ref)) <= X_TOL * max(1.0, Wmax)
    m = oracle.fig67_metrics(P["Q"], P["lam"], P["K"], P["sigma"], mu, X)
    m_ref = oracle.fig67_metrics(P["Q"], P["lam"], P["K"], P["sigma"], mu_ref, X_ref)
    # B and C are quadratic in X: they move by at most 2 |X| |dX| (+ |dX|^2) per
    # unit of max |mu|, with |dX|_2 <= n max |dX|
    dX = X.shape[0] * np.max(np.abs(X - X_ref))
    nx = np.linalg.norm(X_ref, 2)
    slack = 4 * dX * (1 + nx) ** 2 * max(1.0, np.max(np.abs(mu_ref)))
    for panel in "ABC":
        assert abs(m[panel] - m_ref[panel]) <= 1e-6 * m_ref[panel] + slack + 1e-14


def test_perturbation_sigma_repeated_eigenvalues_and_aliasing(eu, handle):
    P = workloads.general(150, 6, seed=77, sigma="mixed", lam_kind="uniform", kscale=0.02)
    P["lam"][40] = P["lam"][41]  # a repeated eigenvalue: its pair contributes 0
    mu, X = _run(eu, handle, P)
    mu_ref, X_ref = oracle.perturbation(P["Q"], P["lam"], P["K"], P["sigma"])
    assert np.max(np.abs(mu - mu_ref)) <= 1e-14
    assert np.max(np.abs(X - X_ref)) <= X_TOL * max(1.0, np.max(np.abs(P["Q"].T @ X_ref)))
    mu2, X2 = _run(eu, handle, P, alias=True)  # mu written over lambda
    assert np.array_equal(mu2, mu) and np.array_equal(X2, X)


def test_perturbation_full_size_sampled(eu, handle):
    """n = 8192, k = 8 (the update's headline workload), sampled columns."""
    P = workloads.general_rank_k(k=8, seed=2000, n=8192, device="cuda:0")
    mu, X = _run(eu, handle, P)
    n = 8192
    cols = np.unique(np.concatenate([[0, 1, n // 2, n - 1], np.random.default_rng(4).choice(n, 12, replace=False)]))
    mu_ref, Xc = oracle.perturbation(P["Q"], P["lam"], P["K"], P["sigma"], cols=cols)
    scale = np.max(np.abs(P["lam"]))
    assert np.max(np.abs(mu - mu_ref)) <= 1e-14 * scale
    Wmax = np.max(np.abs(P["Q"].T @ Xc))
    assert np.max(np.abs(X[:, cols] - Xc)) <= X_TOL * max(1.0, Wmax)


def test_perturbation_invalid_inputs(eu, handle):
    import torch

    P = workloads.small_k(n=20, k=2, knorm=0.1, seed=1)
    Q, lam, K = dev_colmajor(P["Q"]), dev_vec(P["lam"]), dev_colmajor(P["K"])
    mu = torch.empty(20, dtype=torch.float64, device="cuda:0")
    with pytest.raises(eu.EigError):
        eu.eig_perturbation(handle, Q, lam, K, None, mu, Q)  # X must not be Q
    X = torch.empty((20, 20), dtype=torch.float64, device="cuda:0").t()
    with pytest.raises(eu.EigError):
        eu.eig_perturbation(handle, Q, lam, K, [1, 2], mu, X)
