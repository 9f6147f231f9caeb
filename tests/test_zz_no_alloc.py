"""eig_secular_values_static: the eigenvalue stage without any device allocation.

Some callers cannot allocate device memory (their HBM belongs to another memory
manager, or an allocation's device synchronisation is not acceptable in their
loop).  This entry point keeps every temporary in a fixed library-owned device
array.  The test calls it through the C ABI twice in a row, on two different
problems, and checks each result against eig_secular_values, which allocates
its workspace through a handle.  It lives in its own file, collected last.
"""
import numpy as np
import pytest

import oracle
import workloads
from gpu_util import dev_colmajor, dev_vec, host, norm2_A

pytestmark = pytest.mark.gpu

MU_TOL = 1e-10


def _both(eu, h, P):
    import torch

    n = P["lam"].shape[0]
    U = dev_colmajor(oracle.project(P["Q"], P["K"]))
    lam = dev_vec(P["lam"])
    mu_ref = torch.empty(n, dtype=torch.float64, device="cuda:0")
    it_ref = torch.zeros(n, dtype=torch.int32, device="cuda:0")
    assert eu.eig_secular_values(h, lam, U, P["sigma"], mu_ref, it_ref) == 0
    mu = torch.full((n,), np.nan, dtype=torch.float64, device="cuda:0")
    it = torch.full((n,), -1, dtype=torch.int32, device="cuda:0")
    rc = eu.eig_secular_values_static(lam, U, P["sigma"], mu, it)
    torch.cuda.synchronize()
    return rc, host(mu_ref), host(it_ref), host(mu), host(it)


def test_static_scratch_matches_allocating_entry_point():
    import paper_1706_00773_gb300 as eu

    h = eu.eig_update_init(0)
    try:
        first = workloads.general(3000, 5, seed=71, sigma="mixed", lam_kind="logspec")
        second = workloads.general(777, 12, seed=72, sigma="psd", lam_kind="clustered")
        for P in (first, second):  # two calls in a row share the one scratch array
            rc, mu_ref, it_ref, mu, it = _both(eu, h, P)
            assert rc == 0
            scale = norm2_A(P["lam"], P["K"])
            assert np.all(np.isfinite(mu))
            assert np.max(np.abs(mu - mu_ref)) <= MU_TOL * scale
            assert np.array_equal(it, it_ref)
            ref = oracle.update(P["Q"], P["lam"], P["K"], P["sigma"], want_vectors=False)
            assert np.max(np.abs(mu - ref["mu"])) <= MU_TOL * scale
        n = eu.EIG_STATIC_MAX_N + 1
        big = dev_vec(np.arange(n, dtype=np.float64))
        Ub = dev_colmajor(np.zeros((n, 1)))
        import torch

        out = torch.empty(n, dtype=torch.float64, device="cuda:0")
        assert eu.eig_secular_values_static(big, Ub, None, out) == eu.EIG_ETOOBIG
    finally:
        eu.eig_update_destroy(h)
