"""Root counts the update takes, pinned bit-exactly against the oracle.

The zero finder places every root from the count #{mu < lam'_q} at each kept
pole q (Sec. 2.2, the location sub-problem).  In mixed mode that count comes
from a certified FP32 pass, with an FP64 recount wherever the FP32 error bound
cannot certify it.  eig_pole_counts returns both the final counts and the FP32
pass's own (-1 where it gave up); both are compared here, element by element,
with oracle.pole_count on the oracle's own deflated sub-problem, at full size
(n = 8192 log-spectrum, n = 4096 one-row-one-column) and on spectra built to
defeat the FP32 bound.  Points inside 1e-8 clusters check eig_count there.
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


def _oracle_pole_counts(lam, U, sigma):
    """The oracle's deflation rule and its pole-limit count at every kept pole."""
    assert not oracle.repeated_runs(lam)  # no rotation of equal poles in these cases
    keep = np.nonzero(~oracle.deflation_mask(lam, U))[0]
    lp, Up = lam[keep], np.asfortranarray(U[keep])
    return keep, np.array([oracle.pole_count(lp, Up, sigma, q) for q in range(keep.shape[0])], dtype=np.int64)


def _gpu_pole_counts(eu, h, lam, U, sigma):
    import torch

    n = lam.shape[0]
    cnt = torch.full((n,), -7, dtype=torch.int32, device="cuda:0")
    c32 = torch.full((n,), -7, dtype=torch.int32, device="cuda:0")
    idx = torch.full((n,), -7, dtype=torch.int32, device="cuda:0")
    rc, nk = eu.eig_pole_counts(h, dev_vec(lam), dev_colmajor(U), sigma, cnt, c32, idx)
    assert rc == 0
    return nk, host(cnt)[:nk].astype(np.int64), host(c32)[:nk].astype(np.int64), host(idx)[:nk]


def _compare(eu, handles, lam, U, sigma, expect_uncertified=False):
    keep, want = _oracle_pole_counts(lam, U, sigma)
    out = {}
    for mode, h in handles.items():
        nk, cnt, c32, idx = _gpu_pole_counts(eu, h, lam, U, sigma)
        assert nk == keep.shape[0], (mode, nk, keep.shape[0])
        assert np.array_equal(idx, keep), mode                     # same rows deflate
        bad = np.nonzero(cnt != want)[0]
        assert bad.size == 0, (mode, bad[:10], cnt[bad[:10]], want[bad[:10]])
        if mode == "fp64":
            assert np.all(c32 == -1)
        else:
            cert = c32 >= 0
            # every count the FP32 bound certified is the exact count
            assert np.array_equal(c32[cert], want[cert])
            assert np.all(c32[~cert] == -1)
            assert cert.sum() > 0
            if expect_uncertified:
                assert (~cert).sum() > 0          # the FP64 recount fired and was right
            out["uncertified"] = int((~cert).sum())
    return out


def test_pole_counts_general_rank_k_full_size(eu, handles):
    """n = 8192, k = 8, lam = +-10^U[-3,3] (dense poles: M~ ~ 1e4 against pole gaps)."""
    P = workloads.general_rank_k(k=8, seed=2000, n=8192, device="cuda:0")
    U = oracle.project(P["Q"], P["K"])
    _compare(eu, handles, P["lam"], U, P["sigma"])


def test_pole_counts_indefinite_full_size(eu, handles):
    """n = 4096 one-row-one-column update: 1e-8 clusters and planted deflation."""
    W = workloads.indefinite_rank2(seed=1000, n=4096)
    K, s = oracle.rank2_perturbation(4096, W["j"], W["a"])
    U = oracle.project(W["Q"], K)
    _compare(eu, handles, W["lam"], U, s)


@pytest.mark.parametrize("k,sigma", [(2, "mixed"), (5, "psd"), (8, "mixed"), (12, "nsd"), (16, "mixed")])
def test_pole_counts_defeat_the_fp32_bound(eu, handles, k, sigma):
    """Clustered spectrum with some pole pairs 1e-13 apart (relative): the FP32
    pair differences there carry errors far above the pole gap, so the bound
    refuses those counts and the FP64 recount must supply them, bit-exactly."""
    P = workloads.general(700, k, seed=5100 + k, sigma=sigma, lam_kind="clustered")
    lam = P["lam"].copy()
    rng = np.random.default_rng(k)
    for i in rng.choice(np.arange(1, 699, 3), 20, replace=False):
        lam[i + 1] = lam[i] + 1e-13 * max(1.0, abs(lam[i]))
    lam = np.sort(lam)
    assert np.all(np.diff(lam) > 0)
    U = oracle.project(P["Q"], P["K"])
    _compare(eu, handles, lam, U, P["sigma"], expect_uncertified=True)


@pytest.mark.parametrize("k,sigma", [(2, "mixed"), (3, "psd"), (8, "mixed"), (16, "nsd")])
def test_counts_inside_clusters(eu, handles, k, sigma):
    """Counts at points inside 1e-8 clusters, farther than 1e3 eps |A| from every
    eigenvalue, in both modes: equal to the dense spectrum's and the oracle's."""
    import torch

    P = workloads.general(600, k, seed=5200 + k, sigma=sigma, lam_kind="clustered")
    U = oracle.project(P["Q"], P["K"])
    lam = P["lam"]
    ev = np.linalg.eigvalsh(oracle.updated_matrix(P["Q"], lam, P["K"], P["sigma"]))
    scale = norm2_A(lam, P["K"])
    margin = 1e3 * EPS * scale
    gaps = np.diff(lam)
    cl = np.nonzero(gaps < 1e-7)[0]
    assert cl.size >= 30
    cand = []
    for i in cl:  # points spread over the 1e-8 interval of each cluster and just outside it
        for t in (-0.5, 0.1, 0.25, 0.5, 0.75, 0.9, 1.5):
            cand.append(lam[i] + t * gaps[i])
    mids = 0.5 * (ev[1:] + ev[:-1])
    cand += list(mids[(np.diff(ev) < 1e-6) & (np.diff(ev) > 2 * margin)])
    pts = np.array([x for x in cand if np.min(np.abs(ev - x)) > margin and not np.any(lam == x)])
    assert pts.size >= 100
    want = np.array([oracle.count(lam, U, P["sigma"], x) for x in pts])
    assert np.array_equal(want, np.sum(ev[None, :] < pts[:, None], axis=1))  # the oracle, pinned
    for mode, h in handles.items():
        counts = torch.zeros(pts.shape[0], dtype=torch.int32, device="cuda:0")
        eu.eig_count(h, dev_vec(lam), dev_colmajor(U), P["sigma"], dev_vec(pts), counts)
        got = host(counts)
        assert np.array_equal(got, want), (mode, np.nonzero(got != want)[0][:10])


def test_pole_counts_rejects_bad_input(eu, handles):
    import torch

    lam = np.array([3.0, 1.0, 2.0])
    U = np.ones((3, 2))
    cnt = torch.zeros(3, dtype=torch.int32, device="cuda:0")
    with pytest.raises(eu.EigError) as ei:
        eu.eig_pole_counts(handles["mixed"], dev_vec(lam), dev_colmajor(U), None, cnt)
    assert ei.value.code == eu.EIG_EINVAL
