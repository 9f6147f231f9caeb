"""Serving: chained updates of resident decompositions under continuous batching.

Each request's result must be the same whether it ran alone or in a mixed
batch; after a chain the eigenvalues must match a fresh eigendecomposition of
the accumulated matrix, and admission must respect the workspace budget.
"""
import numpy as np
import pytest

import oracle
import workloads
from gpu_util import dev_colmajor, dev_vec, host

pytestmark = pytest.mark.gpu


def _residents(sizes, seed):
    return [workloads.rank2_basic(seed=seed + i, n=n, k=2) for i, n in enumerate(sizes)]


def _chain(n, steps, seed):
    rng = np.random.default_rng(seed)
    out = []
    for t in range(steps):
        k = int(rng.integers(2, 9))
        K = rng.standard_normal((n, k)) / np.sqrt(n)
        sig = np.ones(k, dtype=np.int8)
        if t % 3 == 2:
            sig[rng.permutation(k)[: k // 2]] = -1
        out.append((K, sig))
    return out


@pytest.mark.parametrize("mode_name", ["fp64", "mixed"])
def test_served_results_equal_alone_and_match_fresh_decomposition(mode_name):
    import torch

    import paper_1706_00773_gb300 as eu

    mode = eu.EIG_MIXED if mode_name == "mixed" else eu.EIG_FP64
    sizes = [90, 150, 257, 300]
    res = _residents(sizes, seed=60)
    chains = [_chain(n, 5, seed=700 + i) for i, n in enumerate(sizes)]
    srv = eu.Server(mode=mode, slots=2, max_batch=8)
    devs = []
    for P in res:
        Q, lam = dev_colmajor(P["Q"]), dev_vec(P["lam"])
        devs.append((Q, lam, srv.add_resident(Q, lam)))
    tickets = []
    for t in range(5):  # interleaved arrivals: every resident's t-th update
        for i in range(len(sizes)):
            K, sig = chains[i][t]
            tickets.append((i, srv.submit(devs[i][2], K, sig)))
    srv.drain()
    torch.cuda.synchronize()
    infos = [srv.query(tk) for _, tk in tickets]
    assert all(inf["status"] == 0 for inf in infos)
    assert max(inf["batch_size"] for inf in infos) > 1  # requests really shared batches
    srv.close()
    h = eu.eig_update_init(0, mode)
    try:
        for i, P in enumerate(res):
            Q, lam = dev_colmajor(P["Q"]), dev_vec(P["lam"])
            for K, sig in chains[i]:
                rc, _ = eu.eig_update_rank_k(h, Q, lam, dev_colmajor(K), sig)
                assert rc == 0
            torch.cuda.synchronize()
            assert np.array_equal(host(devs[i][1]), host(lam))
            assert np.array_equal(host(devs[i][0]), host(Q))
            # drift after the chain versus a fresh decomposition of the accumulated matrix
            A = oracle.updated_matrix(P["Q"], P["lam"], np.zeros((sizes[i], 1)))
            for K, sig in chains[i]:
                A = A + (K * sig.astype(float)[None, :]) @ K.T
            w, _ = oracle.jacobi_eig(A, vectors=False)
            scale = np.linalg.norm(A, 2)
            assert np.max(np.abs(host(lam) - w)) <= 1e-10 * scale * len(chains[i])
            X = host(Q)
            assert np.max(np.linalg.norm(A @ X - X * host(lam)[None, :], axis=0)) <= 1e-9 * scale * len(chains[i])
    finally:
        eu.eig_update_destroy(h)


def test_admission_respects_the_workspace_budget():
    import torch

    import paper_1706_00773_gb300 as eu

    sizes = [200, 220, 240]
    res = _residents(sizes, seed=80)
    # One slot holds 1.5x the largest single request: every batch carries one request.
    h = eu.eig_update_init(0, eu.EIG_MIXED)
    per = max(eu.workspace_bytes(h, n, 3) + 8 * n * 3 + 8192 for n in sizes)
    eu.eig_update_destroy(h)
    srv = eu.Server(mode=eu.EIG_MIXED, slots=2, max_batch=16, hbm_budget=2 * int(1.5 * per))
    ids = []
    for P in res:
        Q, lam = dev_colmajor(P["Q"]), dev_vec(P["lam"])
        ids.append((Q, lam, srv.add_resident(Q, lam)))
    big = workloads.rank2_basic(seed=99, n=1500, k=2)
    Qb, lb = dev_colmajor(big["Q"]), dev_vec(big["lam"])
    bid = srv.add_resident(Qb, lb)
    tks = []
    for t in range(3):
        for i, n in enumerate(sizes):
            K = np.random.default_rng(10 * t + i).standard_normal((n, 3)) / np.sqrt(n)
            tks.append(srv.submit(ids[i][2], K))
    tbig = srv.submit(bid, np.random.default_rng(5).standard_normal((1500, 4)) / 40.0)
    srv.drain()
    torch.cuda.synchronize()
    infos = [srv.query(tk) for tk in tks]
    assert all(inf["status"] == 0 for inf in infos)
    assert max(inf["batch_size"] for inf in infos) == 1  # only what fits one slot's workspace
    assert srv.query(tbig)["status"] == eu.EIG_ENOMEM  # can never fit: rejected, not hung
    assert np.array_equal(host(lb), big["lam"])
    srv.close()


def test_chained_updates_converge_everywhere():
    """Regression: two chains of the serving workload where a root once hit the
    evaluation cap (a model step kept aiming at a neighbouring root)."""
    import torch

    import paper_1706_00773_gb300 as eu

    ns, reqs = workloads.serving_plan(seed=4000, residents=12, nmin=1024, nmax=4096, chain=6)
    h = eu.eig_update_init(0, eu.EIG_MIXED)
    try:
        for r in (9, 10):
            P = workloads.rank2_basic(seed=40000 + r, n=ns[r], k=2, device="cuda:0", min_device_n=256)
            Q, lam = dev_colmajor(P["Q"]), dev_vec(P["lam"])
            for rr, k, sd in reqs:
                if rr != r:
                    continue
                K = dev_colmajor(workloads.chained_K(ns[r], k, sd))
                rc, rep = eu.eig_update_rank_k(h, Q, lam, K, None, eu.EIG_VALUES | eu.EIG_VECTORS | eu.EIG_REPORT)
                assert rc == 0 and rep["n_notconv"] == 0 and rep["iters_max"] < 128
                assert rep["max_residual"] <= 1e-9 * rep["norm_A"]
            torch.cuda.synchronize()
    finally:
        eu.eig_update_destroy(h)
