"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Tolerances: |mu - mu_oracle| <= 1e-10 ||A||_2; |A'x - mu x| <= 1e-9 ||A||_2;
root counts bit-exact at points away from the eigenvalues.
"""
import numpy as np
import pytest

import oracle
import workloads
from gpu_util import cos_match, dev_colmajor, dev_vec, host, norm2_A

pytestmark = pytest.mark.gpu

MU_TOL = 1e-10
RES_TOL = 1e-9


@pytest.fixture(scope="module")
def eu():
    import paper_1706_00773_gb300 as m

    return m


@pytest.fixture(scope="module")
def handle(eu):
    h = eu.eig_update_init(0, eu.EIG_FP64)
    yield h
    eu.eig_update_destroy(h)


def _run_update(eu, h, P, want=None, sigma=None):
    import torch

    Q = dev_colmajor(P["Q"])
    lam = dev_vec(P["lam"])
    K = dev_colmajor(P["K"])
    s = P["sigma"] if sigma is None else sigma
    want = want if want is not None else (eu.EIG_VALUES | eu.EIG_VECTORS | eu.EIG_REPORT)
    rc, rep = eu.eig_update_rank_k(h, Q, lam, K, s, want)
    torch.cuda.synchronize()
    return rc, rep, host(lam), host(Q)


def _check_full(P, mu, X, tol_mu=MU_TOL, tol_res=RES_TOL, ref=None):
    ref = ref or oracle.update(P["Q"], P["lam"], P["K"], P["sigma"])
    scale = norm2_A(P["lam"], P["K"])
    assert np.all(np.diff(mu) >= 0)
    err = np.max(np.abs(mu - ref["mu"]))
    assert err <= tol_mu * scale, err
    res = oracle.residuals(P["Q"], P["lam"], P["K"], P["sigma"], mu, X)
    assert np.max(res) <= tol_res * scale, np.max(res)
    # eigenvectors agree with the oracle's up to sign where the eigenvalue is isolated
    gaps = np.minimum(np.diff(ref["mu"], prepend=-np.inf), np.diff(ref["mu"], append=np.inf))
    iso = gaps > 1e-6 * scale
    if np.any(iso):
        assert np.min(cos_match(X[:, iso], ref["X"][:, iso])) >= 1 - 1e-9
    return ref


# ---------------------------------------------------------------------------
def test_project_matches_oracle(eu, handle):
    import torch

    for n, k in [(1, 1), (37, 3), (300, 8), (513, 16)]:
        P = workloads.general(n, k, seed=n + k)
        U = torch.empty((k, n), dtype=torch.float64, device="cuda:0").t()
        eu.eig_project(handle, dev_colmajor(P["Q"]), dev_colmajor(P["K"]), U)
        torch.cuda.synchronize()
        ref = oracle.project(P["Q"], P["K"])
        assert np.max(np.abs(host(U) - ref)) <= 1e-14 * max(1.0, np.max(np.abs(ref))) * np.sqrt(n)


def test_make_rank2_matches_oracle(eu):
    import torch

    n, j = 1000, 123
    a = np.random.default_rng(0).standard_normal(n)
    K = torch.empty((2, n), dtype=torch.float64, device="cuda:0").t()
    sig = eu.eig_make_rank2(n, j, dev_vec(a), K)
    torch.cuda.synchronize()
    Kr, sr = oracle.rank2_perturbation(n, j, a)
    assert sig == [1, -1] and list(sr) == [1, -1]
    assert np.max(np.abs(host(K) - Kr)) <= 2 * np.finfo(float).eps * np.max(np.abs(Kr))


@pytest.mark.parametrize("k,sigma", [(1, "psd"), (1, "nsd"), (2, "mixed"), (3, "mixed"), (4, "psd"),
                                     (5, "nsd"), (8, "mixed"), (9, "psd"), (12, "mixed"), (16, "mixed")])
def test_counts_bit_exact(eu, handle, k, sigma):
    import torch

    n = 150
    P = workloads.general(n, k, seed=100 + k, sigma=sigma, kscale=0.4)
    U = oracle.project(P["Q"], P["K"])
    ev = np.linalg.eigvalsh(oracle.updated_matrix(P["Q"], P["lam"], P["K"], P["sigma"]))
    scale = norm2_A(P["lam"], P["K"])
    mids = 0.5 * (ev[1:] + ev[:-1])
    gaps = np.diff(ev)
    pts = list(mids[gaps > 1e-6 * scale]) + [ev[0] - 1.0, ev[-1] + 1.0]
    pts += list(P["lam"][::7])  # exactly at poles (limit from the left)
    pts = np.array(pts)
    expect = []
    for x in pts:
        if np.any(P["lam"] == x):
            expect.append(oracle.pole_count(P["lam"], U, P["sigma"], int(np.nonzero(P["lam"] == x)[0][0])))
        else:
            expect.append(oracle.count(P["lam"], U, P["sigma"], x))
    expect = np.array(expect)
    # where the dense spectrum is unambiguous, the oracle's count is that index
    far = np.min(np.abs(pts[:, None] - ev[None, :]), axis=1) > 1e-9 * scale
    assert np.array_equal(expect[far], np.sum(ev[None, :] < pts[far, None], axis=1))
    counts = torch.zeros(pts.shape[0], dtype=torch.int32, device="cuda:0")
    eu.eig_count(handle, dev_vec(P["lam"]), dev_colmajor(U), P["sigma"], dev_vec(pts), counts)
    got = host(counts)
    assert np.array_equal(got, expect), (got - expect)


@pytest.mark.parametrize("n,k,sigma,kind", [(64, 1, "psd", "uniform"), (200, 2, "mixed", "uniform"),
                                            (333, 4, "nsd", "logspec"), (257, 7, "mixed", "clustered"),
                                            (300, 8, "psd", "logspec"), (129, 11, "mixed", "uniform"),
                                            (96, 16, "psd", "uniform")])
def test_secular_values(eu, handle, n, k, sigma, kind):
    import torch

    P = workloads.general(n, k, seed=7 * n + k, sigma=sigma, lam_kind=kind)
    U = oracle.project(P["Q"], P["K"])
    mu = torch.empty(n, dtype=torch.float64, device="cuda:0")
    iters = torch.zeros(n, dtype=torch.int32, device="cuda:0")
    rc = eu.eig_secular_values(handle, dev_vec(P["lam"]), dev_colmajor(U), P["sigma"], mu, iters)
    assert rc == 0
    ref = oracle.update(P["Q"], P["lam"], P["K"], P["sigma"], want_vectors=False)
    assert np.max(np.abs(host(mu) - ref["mu"])) <= MU_TOL * norm2_A(P["lam"], P["K"])
    assert int(host(iters).max()) < 128


def test_rank2_basic_workload(eu, handle):
    P = workloads.rank2_basic(seed=0, n=256, k=2)
    rc, rep, mu, X = _run_update(eu, handle, P)
    assert rc == 0 and rep["status"] == 0
    _check_full(P, mu, X)
    assert rep["max_residual"] <= RES_TOL * norm2_A(P["lam"], P["K"])
    assert rep["max_orth"] <= 1e-12


@pytest.mark.parametrize("n,k,sigma", [(1, 1, "psd"), (2, 1, "nsd"), (3, 5, "mixed"), (31, 3, "psd"),
                                       (33, 2, "mixed"), (100, 9, "nsd"), (257, 13, "mixed"),
                                       (130, 15, "psd"), (64, 16, "mixed")])
def test_update_ragged_and_padded(eu, handle, n, k, sigma):
    P = workloads.general(n, k, seed=n * 31 + k, sigma=sigma, kscale=0.5)
    rc, rep, mu, X = _run_update(eu, handle, P)
    assert rc == 0
    _check_full(P, mu, X)


def test_indefinite_rank2_full_size(eu, handle):
    """One-row-one-column update at n=4096 with 1e-8 clusters and planted deflation."""
    import torch

    P = workloads.indefinite_rank2(seed=1000, n=4096)
    n = 4096
    Q = dev_colmajor(P["Q"])
    lam = dev_vec(P["lam"])
    a = dev_vec(P["a"])
    K = torch.empty((2, n), dtype=torch.float64, device="cuda:0").t()
    sig = eu.eig_make_rank2(n, P["j"], a, K)
    rc, rep = eu.eig_update_rank_k(handle, Q, lam, K, sig, eu.EIG_VALUES | eu.EIG_VECTORS | eu.EIG_REPORT)
    torch.cuda.synchronize()
    assert rc == 0
    Kh, sh = oracle.rank2_perturbation(n, P["j"], P["a"])
    PP = dict(Q=P["Q"], lam=P["lam"], K=Kh, sigma=sh)
    assert rep["n_deflated"] == len(P["planted"])
    _check_full(PP, host(lam), host(Q))
    assert oracle.orthogonality(host(Q)) <= 1e-9


def test_general_rank_k_full_size_sampled(eu, handle):
    """n=8192, k=8: sampled roots and vectors against the oracle, computed one by one."""
    import torch

    P = workloads.general_rank_k(k=8, seed=2000, n=8192, device="cuda:0")
    rc, rep, mu, X = _run_update(eu, handle, P)
    assert rc == 0
    n = 8192
    sel = np.unique(np.concatenate([[0, 1, n // 2, n - 2, n - 1],
                                    np.random.default_rng(5).choice(n, 59, replace=False)]))
    ref = oracle.update(P["Q"], P["lam"], P["K"], P["sigma"], sel=sel)
    scale = norm2_A(P["lam"], P["K"])
    pos = ref["pos"]
    assert np.max(np.abs(mu[pos] - ref["mu"])) <= MU_TOL * scale
    assert np.min(cos_match(X[:, pos], ref["X"])) >= 1 - 1e-9
    res = oracle.residuals(P["Q"], P["lam"], P["K"], P["sigma"], mu[pos], X[:, pos])
    assert np.max(res) <= RES_TOL * scale
    assert rep["max_residual"] <= RES_TOL * scale


def test_everything_deflates(eu, handle):
    P = workloads.general(50, 3, seed=1)
    P["K"] = np.zeros_like(P["K"])
    rc, rep, mu, X = _run_update(eu, handle, P)
    assert rc == 0 and rep["n_deflated"] == 50
    assert np.array_equal(mu, P["lam"])
    assert np.array_equal(X, P["Q"])


def test_invalid_inputs_are_rejected(eu, handle):
    import torch

    P = workloads.general(40, 2, seed=3)
    lam_bad = P["lam"].copy()[::-1].copy()
    Q = dev_colmajor(P["Q"])
    Qcopy = Q.clone()
    lam = dev_vec(lam_bad)
    rc, _ = eu.eig_update_rank_k(handle, Q, lam, dev_colmajor(P["K"]), None,
                                 eu.EIG_VALUES | eu.EIG_VECTORS, raise_on_error=False)
    assert rc == eu.EIG_EINVAL
    assert torch.equal(Q, Qcopy) and np.array_equal(host(lam), lam_bad)
    lam_nan = P["lam"].copy()
    lam_nan[5] = np.nan
    rc, _ = eu.eig_update_rank_k(handle, dev_colmajor(P["Q"]), dev_vec(lam_nan), dev_colmajor(P["K"]),
                                 None, eu.EIG_VALUES, raise_on_error=False)
    assert rc == eu.EIG_EINVAL
    with pytest.raises(eu.EigError):
        eu.eig_update_rank_k(handle, dev_colmajor(P["Q"]), dev_vec(P["lam"]), dev_colmajor(P["K"]), [1, 2])
    K17 = dev_colmajor(np.zeros((40, 17)))
    with pytest.raises(eu.EigError):
        eu.eig_update_rank_k(handle, dev_colmajor(P["Q"]), dev_vec(P["lam"]), K17)


def test_q_out_keeps_input(eu, handle):
    import torch

    P = workloads.general(120, 4, seed=9, sigma="mixed")
    Q = dev_colmajor(P["Q"])
    Qo = torch.empty((120, 120), dtype=torch.float64, device="cuda:0").t()
    lam = dev_vec(P["lam"])
    rc, rep = eu.eig_update_rank_k(handle, Q, lam, dev_colmajor(P["K"]), P["sigma"],
                                   eu.EIG_VALUES | eu.EIG_VECTORS, Q_out=Qo)
    torch.cuda.synchronize()
    assert rc == 0
    assert np.array_equal(host(Q), P["Q"])
    _check_full(P, host(lam), host(Qo))


def test_batch_matches_solo(eu, handle):
    import torch

    probs, devs = [], []
    for t, (n, k) in enumerate([(64, 1), (200, 3), (129, 8), (300, 5)]):
        P = workloads.general(n, k, seed=500 + t, sigma="mixed" if k > 1 else "psd")
        d = dict(Q=dev_colmajor(P["Q"]), lam=dev_vec(P["lam"]), K=dev_colmajor(P["K"]), sigma=P["sigma"],
                 want=eu.EIG_VALUES | eu.EIG_VECTORS)
        probs.append(P)
        devs.append(d)
    tickets = eu.eig_update_batch(handle, devs)
    torch.cuda.synchronize()
    for P, d, t in zip(probs, devs, tickets):
        assert eu.eig_update_query(handle, eu.EIG_Q_STATUS, t) == 0
        rc, rep = eu.eig_update_query(handle, eu.EIG_Q_REPORT, t)
        assert rc == 0 and rep["n"] == P["lam"].shape[0]
        solo_rc, _, mu_s, X_s = _run_update(eu, handle, P, want=eu.EIG_VALUES | eu.EIG_VECTORS)
        assert np.array_equal(host(d["lam"]), mu_s)
        assert np.array_equal(host(d["Q"]), X_s)


# ---------------------------------------------------------------------------
# Mixed mode: X = Q W as split-BF16 tensor-core products (5 slices, 15 pairs)
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def handle_mixed(eu):
    h = eu.eig_update_init(0, eu.EIG_MIXED)
    yield h
    eu.eig_update_destroy(h)


@pytest.mark.parametrize("n,k,sigma", [(1, 1, "psd"), (100, 2, "mixed"), (256, 8, "psd"), (333, 16, "mixed"),
                                       (1000, 5, "nsd"), (2100, 8, "mixed")])
def test_mixed_matches_fp64_and_oracle(eu, handle, handle_mixed, n, k, sigma):
    P = workloads.general(n, k, seed=900 + n + k, sigma=sigma, lam_kind="logspec" if n > 500 else "uniform")
    rc, rep, mu64, X64 = _run_update(eu, handle, P, want=eu.EIG_VALUES | eu.EIG_VECTORS)
    assert rc == 0
    rc, rep, mum, Xm = _run_update(eu, handle_mixed, P)
    assert rc == 0 and rep["status"] == 0
    # Mixed mode runs the zero finder's coarse steps on FP32 sums (bracket moved
    # only by certified counts) and finishes every root in FP64: the roots agree
    # with the FP64 mode's to rounding.
    assert np.max(np.abs(mum - mu64)) <= 1e-13 * norm2_A(P["lam"], P["K"])
    if n > 1:
        assert rep["iters32_total"] > 0
    assert 0 <= rep["gj32_total"] <= rep["iters32_total"]
    # X from the tensor cores vs the FP64 GEMM: 5 slices keep ~2^-40 of the scale
    assert np.max(np.abs(Xm - X64)) <= 1e-10
    _check_full(P, mum, Xm)
    assert rep["max_orth"] <= 1e-10


def _pair_products_full(n):
    t = (n + 127) // 128
    return 15 * t * t * ((n + 31) // 32)


def test_mixed_gemm_pair_products_issued(eu, handle, handle_mixed):
    """report.tc_pair_tiles: the split GEMM issues 15 slice-pair products per
    128 x 128 output tile and 32-deep step, less 5 where W's slice 0 is all zero
    in that tile and 4 where slice 1 is; 0 where the split GEMM does not run."""
    # W = I (every pole deflates): slice 0 holds one entry per column (the
    # unit), slice 1 none.  In tile column tn only the step holding a column's
    # diagonal has slice 0 non-zero: 11 pairs there, 6 in every other step.
    n = 1000
    P = workloads.general(n, 3, seed=11)
    P["K"] = np.zeros_like(P["K"])
    rc, rep, mu, X = _run_update(eu, handle_mixed, P)
    assert rc == 0 and rep["n_deflated"] == n
    assert np.array_equal(mu, P["lam"])
    assert np.max(np.abs(X - P["Q"])) <= 1e-11  # Q through its 5 BF16 slices
    t, nch = (n + 127) // 128, (n + 31) // 32
    assert rep["tc_pair_tiles"] == t * (6 * t * nch + 5 * nch)
    # a secular update: between the 6 pairs never skipped (q >= 2) and all 15
    P = workloads.general(2100, 8, seed=3008, sigma="mixed", lam_kind="logspec")
    rc, rep, mu, X = _run_update(eu, handle_mixed, P)
    assert rc == 0
    full = _pair_products_full(2100)
    assert 6 * full // 15 <= rep["tc_pair_tiles"] <= full
    assert rep["asm_fp64_cols"] == 0  # every column of W from the double-float path
    _check_full(P, mu, X)
    # no split GEMM: FP64 mode, eigenvalues only
    rc, rep, _, _ = _run_update(eu, handle, P)
    assert rc == 0 and rep["tc_pair_tiles"] == 0
    rc, rep, _, _ = _run_update(eu, handle_mixed, P, want=eu.EIG_VALUES | eu.EIG_REPORT)
    assert rc == 0 and rep["tc_pair_tiles"] == 0


def test_mixed_projection_fallbacks(eu, handle, handle_mixed):
    """Mixed mode forms U = Q^T K in double-float arithmetic (pairs of FP32,
    K's columns scaled by powers of 2).  A K whose row 17 is 2^20 times the
    others (a wide dynamic range in every column of U) still gives the
    eigenvalues of diag(lam) + U Sigma U^T to 1e-13 |A| (numpy's symmetric
    eigensolver as the reference).  A column of Q holding an Inf or a NaN takes
    the FP64 projection, so the non-finite input reaches the deflation check
    (EIG_EINVAL) instead of being flushed; a non-finite K likewise."""
    P = workloads.general(600, 5, seed=91, sigma="mixed", lam_kind="uniform")
    K = P["K"].copy()
    K[17, :] *= 2.0 ** 20
    U = P["Q"].T @ K
    ref = np.linalg.eigvalsh(np.diag(P["lam"]) + (U * P["sigma"].astype(float)) @ U.T)
    normA = np.max(np.abs(P["lam"])) + np.sum(U * U)
    for h in (handle, handle_mixed):
        rc, rep, mu, _ = _run_update(eu, h, dict(P, K=K), want=eu.EIG_VALUES | eu.EIG_REPORT)
        assert rc == 0
        assert np.max(np.abs(mu - ref)) <= 1e-13 * normA
    for bad in ("Q_inf", "Q_nan", "K_nan"):
        Pn = dict(P, Q=P["Q"].copy(), K=P["K"].copy())
        if bad == "Q_inf":
            Pn["Q"][5, 9] = np.inf
        elif bad == "Q_nan":
            Pn["Q"][5, 9] = np.nan
        else:
            Pn["K"][40, 2] = np.nan
        rc, _ = eu.eig_update_rank_k(handle_mixed, dev_colmajor(Pn["Q"]), dev_vec(Pn["lam"]),
                                     dev_colmajor(Pn["K"]), Pn["sigma"], eu.EIG_VALUES | eu.EIG_VECTORS,
                                     raise_on_error=False)
        assert rc == eu.EIG_EINVAL, bad


def test_mixed_full_size_sampled(eu, handle_mixed):
    P = workloads.general_rank_k(k=8, seed=2000, n=8192, device="cuda:0")
    rc, rep, mu, X = _run_update(eu, handle_mixed, P)
    assert rc == 0
    n = 8192
    sel = np.unique(np.concatenate([[0, n // 3, n - 1], np.random.default_rng(6).choice(n, 29, replace=False)]))
    ref = oracle.update(P["Q"], P["lam"], P["K"], P["sigma"], sel=sel)
    scale = norm2_A(P["lam"], P["K"])
    pos = ref["pos"]
    assert np.max(np.abs(mu[pos] - ref["mu"])) <= MU_TOL * scale
    assert np.min(cos_match(X[:, pos], ref["X"])) >= 1 - 1e-9
    res = oracle.residuals(P["Q"], P["lam"], P["K"], P["sigma"], mu[pos], X[:, pos])
    assert np.max(res) <= RES_TOL * scale
    assert rep["max_residual"] <= RES_TOL * scale and rep["max_orth"] <= 1e-10


# ---------------------------------------------------------------------------
# Batches: every stage of every update in one grouped launch (per padded rank)
# ---------------------------------------------------------------------------
def _batch_problems(count, seed, nmin=64, nmax=700):
    rng = np.random.default_rng(seed)
    out = []
    for t in range(count):
        n = int(np.exp(rng.uniform(np.log(nmin), np.log(nmax))))
        k = int(rng.integers(1, 17))
        sg = ["psd", "nsd", "mixed"][t % 3] if k > 1 else "psd"
        out.append(workloads.general(n, k, seed=seed * 100 + t, sigma=sg, lam_kind=["uniform", "logspec"][t % 2]))
    return out


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_batch_uneven_sizes_match_solo_and_oracle(eu, handle, handle_mixed, mode):
    import torch

    h = handle if mode == "fp64" else handle_mixed
    probs = _batch_problems(24, seed=41 if mode == "fp64" else 42)
    devs = [dict(Q=dev_colmajor(P["Q"]), lam=dev_vec(P["lam"]), K=dev_colmajor(P["K"]), sigma=P["sigma"],
                 want=eu.EIG_VALUES | eu.EIG_VECTORS) for P in probs]
    tickets = eu.eig_update_batch(h, devs)
    torch.cuda.synchronize()
    for P, d, t in zip(probs, devs, tickets):
        assert eu.eig_update_query(h, eu.EIG_Q_STATUS, t) == 0
        rc, _, mu_s, X_s = _run_update(eu, h, P, want=eu.EIG_VALUES | eu.EIG_VECTORS)
        assert rc == 0
        assert np.array_equal(host(d["lam"]), mu_s)       # alone and in the batch: identical
        assert np.array_equal(host(d["Q"]), X_s)
        _check_full(P, mu_s, X_s)


def test_batch_mixes_values_only_and_invalid(eu, handle):
    import torch

    probs = _batch_problems(6, seed=7)
    devs = []
    for i, P in enumerate(probs):
        lam = P["lam"].copy()
        if i == 3:
            lam = lam[::-1].copy()  # unsorted: rejected on the device, outputs untouched
        devs.append(dict(Q=dev_colmajor(P["Q"]), lam=dev_vec(lam), K=dev_colmajor(P["K"]), sigma=P["sigma"],
                         want=eu.EIG_VALUES if i % 2 else eu.EIG_VALUES | eu.EIG_VECTORS))
    tickets = eu.eig_update_batch(handle, devs)
    torch.cuda.synchronize()
    for i, (P, d, t) in enumerate(zip(probs, devs, tickets)):
        st = eu.eig_update_query(handle, eu.EIG_Q_STATUS, t)
        if i == 3:
            assert st == eu.EIG_EINVAL
            assert np.array_equal(host(d["lam"]), P["lam"][::-1])
            continue
        assert st == 0
        ref = oracle.update(P["Q"], P["lam"], P["K"], P["sigma"], want_vectors=False)
        assert np.max(np.abs(host(d["lam"]) - ref["mu"])) <= MU_TOL * norm2_A(P["lam"], P["K"])
        if i % 2:
            assert np.array_equal(host(d["Q"]), P["Q"])  # values only: Q untouched


def test_residuals_at_rounding_level(eu, handle):
    """The null vector is taken at the accepted root, not at the last evaluated
    point (a Newton step away), so eq. (10) vectors reach rounding-level
    residuals like the oracle's; includes a problem with planted deflation."""
    import torch

    P = workloads.general(400, 3, seed=71, sigma="mixed", lam_kind="uniform")
    Q = P["Q"]
    P["K"] = P["K"] - Q[:, 50:60] @ (Q[:, 50:60].T @ P["K"])
    for prob in (P, workloads.general(700, 8, seed=72, sigma="psd", lam_kind="logspec")):
        rc, rep, mu, X = _run_update(eu, handle, prob, want=eu.EIG_VALUES | eu.EIG_VECTORS)
        assert rc == 0
        res = oracle.residuals(prob["Q"], prob["lam"], prob["K"], prob["sigma"], mu, X)
        assert np.max(res) <= 1e-13 * norm2_A(prob["lam"], prob["K"])


# ---------------------------------------------------------------------------
# Mixed mode: the zero finder's FP32 coarse phase and the FP32 pole counts
# (certified, with FP64 fallbacks) against the oracle on hard spectra
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind,sigma,k", [("clustered", "mixed", 3), ("clustered", "psd", 8), ("logspec", "nsd", 5),
                                          ("logspec", "mixed", 12), ("uniform", "mixed", 16)])
def test_mixed_coarse_phase_on_hard_spectra(eu, handle, handle_mixed, kind, sigma, k):
    n = 700
    P = workloads.general(n, k, seed=4100 + k, sigma=sigma, lam_kind=kind)
    rc, rep, mum, Xm = _run_update(eu, handle_mixed, P)
    assert rc == 0 and rep["n_notconv"] == 0
    rc64, _, mu64, _ = _run_update(eu, handle, P, want=eu.EIG_VALUES | eu.EIG_VECTORS)
    assert rc64 == 0
    assert np.max(np.abs(mum - mu64)) <= 1e-12 * norm2_A(P["lam"], P["K"])
    _check_full(P, mum, Xm)


def test_mixed_repeated_poles_and_planted_deflation(eu, handle_mixed):
    """Exactly repeated eigenvalues (FP32 differences of zero: the FP64 paths take
    over) and rows of U that deflate."""
    P = workloads.general(500, 4, seed=77, sigma="mixed", lam_kind="uniform")
    lam = P["lam"].copy()
    lam[100:104] = lam[100]          # a four-fold pole
    lam[300] = lam[301] = lam[300]   # and a double one
    P["lam"] = lam
    Q = P["Q"]
    P["K"] = P["K"] - Q[:, 200:210] @ (Q[:, 200:210].T @ P["K"])
    rc, rep, mu, X = _run_update(eu, handle_mixed, P, want=eu.EIG_VALUES | eu.EIG_VECTORS | eu.EIG_REPORT)
    assert rc == 0 and rep["n_notconv"] == 0
    w = np.linalg.eigvalsh(oracle.updated_matrix(P["Q"], P["lam"], P["K"], P["sigma"]))
    scale = norm2_A(P["lam"], P["K"])
    assert np.max(np.abs(mu - w)) <= 1e-12 * scale
    res = oracle.residuals(P["Q"], P["lam"], P["K"], P["sigma"], mu, X)
    assert np.max(res) <= 1e-9 * scale


def test_mixed_indefinite_workload_matches_oracle(eu, handle_mixed):
    """The one-row-one-column workload (1e-8 clusters, planted deflation) in
    mixed mode, sampled against the oracle."""
    import torch

    W = workloads.indefinite_rank2(seed=1000, n=4096)
    n = W["lam"].shape[0]
    a = torch.from_numpy(W["a"].copy()).to("cuda:0")
    K = torch.empty((2, n), dtype=torch.float64, device="cuda:0").t()
    sig = eu.eig_make_rank2(n, W["j"], a, K)
    P = dict(Q=W["Q"], lam=W["lam"], K=host(K), sigma=np.array(sig, dtype=np.int8))
    rc, rep, mu, X = _run_update(eu, handle_mixed, P)
    assert rc == 0 and rep["n_notconv"] == 0 and rep["iters32_total"] > 0
    nk = n - int(rep["n_deflated"])  # roots of the sub-problem
    sel = np.unique(np.concatenate([[0, nk // 2, nk - 1], np.random.default_rng(9).choice(nk, 40, replace=False)]))
    ref = oracle.update(P["Q"], P["lam"], P["K"], P["sigma"], sel=sel)
    scale = norm2_A(P["lam"], P["K"])
    assert np.max(np.abs(mu[ref["pos"]] - ref["mu"])) <= MU_TOL * scale
    res = oracle.residuals(P["Q"], P["lam"], P["K"], P["sigma"], mu[ref["pos"]], X[:, ref["pos"]])
    assert np.max(res) <= RES_TOL * scale
