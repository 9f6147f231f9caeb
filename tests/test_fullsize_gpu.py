"""The general rank-k workload at full size (n = 8192, k in {4, 8, 16}), both
modes, against the CPU oracle: EVERY eigenvalue at |mu - mu_oracle| <= 1e-10 |A|,
and 256 sampled eigenvectors (cos to the oracle's, residual |A'x - mu x|).

k = 16 runs the padded-rank path with four warps per root (named barriers
between them) and the loosest FP32 certificates; k = 4 the one-warp path with
the fewest accumulators.  The oracle solves each k once (about 10-40 s on the
host cores) and the result is shared by the two modes.
"""
import numpy as np
import pytest

import oracle
import workloads
from gpu_util import cos_match, dev_colmajor, dev_vec, host, norm2_A

pytestmark = pytest.mark.gpu

N = 8192
MU_TOL = 1e-10
RES_TOL = 1e-9
NSAMPLE = 256

_cache = {}


def _case(k):
    if k not in _cache:
        P = workloads.general_rank_k(k=k, seed=2000, n=N, device="cuda:0")
        ref = oracle.update(P["Q"], P["lam"], P["K"], P["sigma"], want_vectors=False)
        assert not ref["deflated"].any()
        rng = np.random.default_rng(100 + k)
        sel = np.unique(np.concatenate([[0, 1, N // 2, N - 2, N - 1], rng.choice(N, NSAMPLE, replace=False)]))[:NSAMPLE]
        refv = oracle.update(P["Q"], P["lam"], P["K"], P["sigma"], sel=sel)
        _cache[k] = (P, ref, refv)
    return _cache[k]


@pytest.fixture(scope="module")
def eu():
    import paper_1706_00773_gb300 as m

    return m


@pytest.mark.parametrize("k", [4, 8, 16])
@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_general_rank_k_every_eigenvalue(eu, mode, k):
    import torch

    P, ref, refv = _case(k)
    h = eu.eig_update_init(0, eu.EIG_MIXED if mode == "mixed" else eu.EIG_FP64)
    try:
        Q = dev_colmajor(P["Q"])
        lam = dev_vec(P["lam"])
        X = torch.empty((N, N), dtype=torch.float64, device="cuda:0").t()
        rc, rep = eu.eig_update_rank_k(h, Q, lam, dev_colmajor(P["K"]), P["sigma"],
                                       eu.EIG_VALUES | eu.EIG_VECTORS | eu.EIG_REPORT, Q_out=X)
        torch.cuda.synchronize()
    finally:
        eu.eig_update_destroy(h)
    assert rc == 0 and rep["n_notconv"] == 0
    scale = norm2_A(P["lam"], P["K"])
    mu = host(lam)
    assert np.all(np.diff(mu) >= 0)
    err = np.abs(mu - ref["mu"])
    assert np.max(err) <= MU_TOL * scale, (np.argmax(err), np.max(err) / scale)
    # trace identity at full size: sum mu - sum lam = tr(Sigma K^T K)
    tr = float(np.sum(P["K"] ** 2 * P["sigma"].astype(float)[None, :]))
    assert abs(np.sum(mu) - np.sum(P["lam"]) - tr) <= 1e-9 * scale
    pos = refv["pos"]
    Xs = host(X[:, torch.from_numpy(pos).to("cuda:0")])
    gaps = np.minimum(np.diff(ref["mu"], prepend=-np.inf), np.diff(ref["mu"], append=np.inf))[pos]
    iso = gaps > 1e-6 * scale
    assert iso.sum() >= 64  # the log-spectrum packs many eigenvalues closer than 1e-6 |A|
    assert np.min(cos_match(Xs[:, iso], refv["X"][:, iso])) >= 1 - 1e-9
    res = oracle.residuals(P["Q"], P["lam"], P["K"], P["sigma"], mu[pos], Xs)
    assert np.max(res) <= RES_TOL * scale
    assert rep["max_residual"] <= RES_TOL * scale
    assert rep["max_orth"] <= (1e-10 if mode == "mixed" else 1e-12)
    if mode == "mixed":
        assert rep["iters32_total"] > 0
