"""Per-eigenpair error report (eig_problem.errors) against the oracle.

Column 0 is the residual of the FP64 eq. (10) vector in the old eigenbasis;
X = Q W only adds the GEMM's error, so it must match oracle.residuals of the
returned X to within that error, pair by pair.  Column 1 (Rayleigh shift) is at
rounding level, column 2 is the gap of the returned spectrum, column 3 the dot
with the next root's vector, which must match the returned X's columns.
"""
import numpy as np
import pytest

import oracle
import workloads
from gpu_util import dev_colmajor, dev_vec, host, norm2_A

pytestmark = pytest.mark.gpu

EPS = np.finfo(float).eps


@pytest.fixture(scope="module")
def eu():
    import paper_1706_00773_gb300 as m

    return m


@pytest.fixture(scope="module")
def handles(eu):
    hs = {"fp64": eu.eig_update_init(0, eu.EIG_FP64), "mixed": eu.eig_update_init(0, eu.EIG_MIXED)}
    yield hs
    for h in hs.values():
        eu.eig_update_destroy(h)


def _errors_buf(n):
    import torch

    return torch.full((4, n), -1.0, dtype=torch.float64, device="cuda:0").t()


def _run(eu, h, P, want=None):
    import torch

    n = P["lam"].shape[0]
    Q = dev_colmajor(P["Q"])
    lam = dev_vec(P["lam"])
    X = torch.empty((n, n), dtype=torch.float64, device="cuda:0").t()
    E = _errors_buf(n)
    want = want if want is not None else eu.EIG_VALUES | eu.EIG_VECTORS
    rc, rep = eu.eig_update_rank_k(h, Q, lam, dev_colmajor(P["K"]), P["sigma"], want, Q_out=X, errors=E)
    torch.cuda.synchronize()
    assert rc == 0
    return rep, host(lam), host(X), host(E)


def _gap(mu):
    return np.minimum(np.diff(mu, prepend=-np.inf), np.diff(mu, append=np.inf))


def _gemm_err(X, X64):
    """Column norms of the mixed-mode X's departure from the FP64 GEMM's X: what
    the split-BF16 product adds to each pair's residual (times |A' - mu|)."""
    return np.linalg.norm(X - X64, axis=0)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("n,k,sigma,kind", [(2100, 8, "psd", "logspec"), (900, 3, "mixed", "clustered"),
                                            (700, 16, "nsd", "uniform")])
def test_pair_errors_match_oracle(eu, handles, mode, n, k, sigma, kind):
    P = workloads.general(n, k, seed=6100 + n + k, sigma=sigma, lam_kind=kind)
    rep, mu, X, E = _run(eu, handles[mode], P)
    normA = rep["norm_A"]
    assert abs(normA - norm2_A(P["lam"], oracle.project(P["Q"], P["K"]))) <= 1e-12 * normA
    assert np.all(E >= 0.0)
    # (0) eigenbasis residual at rounding level; the returned X's residual
    #     (oracle, FP64 in real space) agrees pair by pair up to the GEMM's own
    #     error: |(A' - mu)(X - X64)| <= 2 |A| |X - X64| column by column
    assert np.max(E[:, 0]) <= 1e-13
    res = oracle.residuals(P["Q"], P["lam"], P["K"], P["sigma"], mu, X) / normA
    if mode == "fp64":
        X64 = X
        gemm = np.full(n, 1e-13)
    else:
        _, mu64, X64, _ = _run(eu, handles["fp64"], P)
        assert np.max(np.abs(mu64 - mu)) <= 1e-13 * normA
        gemm = 2.0 * _gemm_err(X, X64) + 1e-13
        assert np.max(_gemm_err(X, X64)) <= 1e-9
        # the report needs the FP64 entries: every secular column takes that path
        assert rep["asm_fp64_cols"] == n - rep["n_deflated"]
    assert np.all(np.abs(res - E[:, 0]) <= gemm), np.max(np.abs(res - E[:, 0]) - gemm)
    # (1) Rayleigh quotient of the FP64 vector agrees with mu
    assert np.max(E[:, 1]) <= 1e-13
    # (2) the gap of the returned spectrum, exactly
    assert np.allclose(E[:, 2], _gap(mu) / normA, rtol=1e-15, atol=0.0)
    # (3) dot with the next secular root's vector where the gap < 1e-6 |A|
    close = np.nonzero(E[:, 3] > 0.0)[0]
    for r in close:
        dots = abs(float(X64[:, r] @ X64[:, r + 1]))
        assert abs(dots - E[r, 3]) <= 1e-12
    assert np.max(E[:, 3]) <= 1e-9
    assert rep["max_pair_residual"] == np.max(E[:, 0])
    assert rep["max_pair_rayleigh"] == np.max(E[:, 1])
    assert rep["max_pair_orth"] == np.max(E[:, 3])


@pytest.mark.parametrize("seed", [1001, 1002])
def test_mixed_projection_keeps_planted_deflation(eu, handles, seed):
    """Mixed mode forms U = Q^T K in double-float arithmetic; its error on the
    planted rows (|u_i| ~ 1e-15) must stay below the deflation threshold, so
    the same rows deflate as in FP64 mode."""
    W = workloads.indefinite_rank2(seed=seed, n=4096)
    K, s = oracle.rank2_perturbation(4096, W["j"], W["a"])
    P = dict(Q=W["Q"], lam=W["lam"], K=K, sigma=s)
    reps = {mode: _run(eu, h, P)[0] for mode, h in handles.items()}
    assert reps["mixed"]["n_deflated"] == reps["fp64"]["n_deflated"] == len(W["planted"])


def test_pair_errors_deflated_pairs(eu, handles):
    """Planted deflation (one-row-one-column workload, n = 4096): deflated pairs
    report the deflation bound |U|_F |u_i| / |A| <= 8 eps."""
    import torch

    W = workloads.indefinite_rank2(seed=1000, n=4096)
    n = 4096
    K, s = oracle.rank2_perturbation(n, W["j"], W["a"])
    P = dict(Q=W["Q"], lam=W["lam"], K=K, sigma=s)
    for mode, h in handles.items():
        rep, mu, X, E = _run(eu, h, P)
        assert rep["n_deflated"] == len(W["planted"])
        U = oracle.project(W["Q"], K)
        defl = oracle.deflation_mask(W["lam"], U)
        pos = np.searchsorted(mu, W["lam"][defl])  # deflated eigenvalues are kept exactly
        assert np.all(mu[pos] == W["lam"][defl])
        assert np.max(E[pos, 0]) <= 8 * EPS
        assert np.all(E[pos, 3] == 0.0)
        assert np.max(E[:, 0]) <= 1e-13
        res = oracle.residuals(P["Q"], P["lam"], P["K"], P["sigma"], mu, X) / rep["norm_A"]
        if mode == "fp64":
            X64 = X
            assert np.max(np.abs(res - E[:, 0])) <= 1e-13
        else:
            assert np.all(np.abs(res - E[:, 0]) <= 2.0 * _gemm_err(X, X64) + 1e-13)
        del X, E
        torch.cuda.empty_cache()


def test_pair_errors_full_size_sampled(eu, handles):
    """n = 8192, k = 8 (the benchmark workload), mixed mode: every pair's
    eigenbasis residual at rounding level; 256 sampled columns' real-space
    residuals (oracle) agree with it pair by pair."""
    P = workloads.general_rank_k(k=8, seed=2000, n=8192, device="cuda:0")
    rep, mu, X, E = _run(eu, handles["mixed"], P)
    assert np.max(E[:, 0]) <= 1e-13 and np.max(E[:, 1]) <= 1e-13
    sel = np.random.default_rng(12).choice(8192, 256, replace=False)
    Xs = X[:, sel].copy()
    del X
    _, mu64, X64, E64 = _run(eu, handles["fp64"], P)
    res = oracle.residuals(P["Q"], P["lam"], P["K"], P["sigma"], mu[sel], Xs) / rep["norm_A"]
    assert np.all(np.abs(res - E[sel, 0]) <= 2.0 * _gemm_err(Xs, X64[:, sel]) + 1e-13)
    res64 = oracle.residuals(P["Q"], P["lam"], P["K"], P["sigma"], mu64[sel], X64[:, sel]) / rep["norm_A"]
    assert np.max(np.abs(res64 - E64[sel, 0])) <= 1e-13
    ref = oracle.update(P["Q"], P["lam"], P["K"], P["sigma"], sel=np.sort(sel), want_vectors=False)
    assert np.max(np.abs(mu[ref["pos"]] - ref["mu"])) <= 1e-10 * rep["norm_A"]


def test_pair_errors_in_a_batch_equal_solo(eu, handles):
    import torch

    probs = [workloads.general(n, k, seed=6200 + n, sigma="mixed" if k > 1 else "psd")
             for n, k in [(300, 2), (129, 9), (511, 5)]]
    devs, bufs = [], []
    for P in probs:
        n = P["lam"].shape[0]
        E = _errors_buf(n)
        bufs.append(E)
        devs.append(dict(Q=dev_colmajor(P["Q"]), lam=dev_vec(P["lam"]), K=dev_colmajor(P["K"]),
                         sigma=P["sigma"], want=eu.EIG_VALUES | eu.EIG_VECTORS, errors=E))
    h = handles["mixed"]
    tickets = eu.eig_update_batch(h, devs)
    torch.cuda.synchronize()
    for P, t, E in zip(probs, tickets, bufs):
        assert eu.eig_update_query(h, eu.EIG_Q_STATUS, t) == 0
        _, _, _, E1 = _run(eu, h, P)
        assert np.array_equal(host(E), E1)
