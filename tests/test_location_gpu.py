"""GPU parity of the rank-2 location vector (Algorithms 1a-1c) and its residues.

The location vector is integer work: it must equal the oracle's bit for bit,
and (where every residue is well away from zero) the true interval counts.
"""
import numpy as np
import pytest

import oracle
import workloads
from gpu_util import dev_colmajor, dev_vec, host

pytestmark = pytest.mark.gpu

SIGNS = {"1a": (1, 1), "1b": (-1, -1), "1c": (1, -1), "1c'": (-1, 1)}


@pytest.fixture(scope="module")
def eu():
    import paper_1706_00773_gb300 as m

    return m


def _run(eu, lam, U, s):
    import torch

    n = len(lam)
    alpha = torch.empty(n, dtype=torch.float64, device="cuda:0")
    L = torch.full((n + 1,), -7, dtype=torch.int32, device="cuda:0")
    eu.eig_location_rank2(dev_vec(lam), dev_colmajor(U), s, alpha, L)
    torch.cuda.synchronize()
    return host(alpha), host(L).astype(np.int64)


def _pole_truth(lam, U, s):
    n = len(lam)
    below = [0] + [oracle.pole_count(lam, U, s, p) for p in range(n)]
    below.append(n)
    return np.diff(np.array(below))


def _rank2(n, seed):
    rng = np.random.default_rng(seed)
    return np.sort(rng.standard_normal(n)), rng.standard_normal((n, 2)) * 0.6


@pytest.mark.parametrize("case", list(SIGNS))
@pytest.mark.parametrize("n", [2, 3, 37, 1000, 1025, 4097])
def test_location_matches_oracle_and_counts(eu, case, n):
    s = np.array(SIGNS[case], dtype=np.int8)
    lam, U = _rank2(n, 31 * n + len(case))
    a_gpu, L_gpu = _run(eu, lam, U, s)
    a_ref = oracle.residues(lam, U, s)
    scale = np.abs(a_ref) + 1e-300
    # both sides sum n-1 reciprocal terms in different orders; against extended
    # precision the oracle is within 3e-12 at n = 4097
    assert np.max(np.abs(a_gpu - a_ref) / scale) <= 1e-9
    same_signs = np.array_equal(np.sign(a_gpu), np.sign(a_ref))
    assert same_signs
    assert np.array_equal(L_gpu, oracle.location_vector(lam, U, s))
    assert L_gpu.sum() == n
    if n <= 1025:
        assert np.array_equal(L_gpu, _pole_truth(lam, U, s))


def test_location_of_the_indefinite_workload(eu):
    """e_j a^T + a e_j^T on a Haar basis, n = 4096 (Sec. 2.2 Steps 1-2, 1c)."""
    import torch

    P = workloads.rank2_basic(seed=17, n=4096, k=2, device="cuda:0", min_device_n=256)
    n = P["Q"].shape[0]
    rng = np.random.default_rng(3)
    a = rng.standard_normal(n) / np.sqrt(n)
    K = torch.empty((2, n), dtype=torch.float64, device="cuda:0").t()  # column-major n x 2
    s = eu.eig_make_rank2(n, 123, dev_vec(a), K)
    U = oracle.project(P["Q"], host(K))
    lam = P["lam"]
    a_gpu, L_gpu = _run(eu, lam, U, np.array(s, dtype=np.int8))
    s8 = np.array(s, dtype=np.int8)
    a_ref = oracle.residues(lam, U, s8)
    assert np.min(np.abs(a_ref)) > 1e-10 * np.max(np.abs(a_ref))  # signs are meaningful here
    assert np.array_equal(np.sign(a_gpu), np.sign(a_ref))
    assert np.array_equal(L_gpu, oracle.location_vector(lam, U, s8))
    assert np.array_equal(L_gpu, _pole_truth(lam, U, s8))


def test_zero_residue_follows_the_listing(eu):
    """A zero row of U gives alpha_p = 0: the sign test fails on both sides of
    it, exactly as the oracle's greedy scan reads it."""
    for case in SIGNS:
        s = np.array(SIGNS[case], dtype=np.int8)
        lam, U = _rank2(50, 5)
        U[[7, 20, 21]] = 0.0
        a_gpu, L_gpu = _run(eu, lam, U, s)
        assert a_gpu[7] == 0.0 and a_gpu[20] == 0.0
        assert np.array_equal(L_gpu, oracle.location_vector(lam, U, s)), case


def test_location_invalid_inputs(eu):
    import torch

    lam, U = _rank2(8, 1)
    alpha = torch.empty(8, dtype=torch.float64, device="cuda:0")
    L = torch.zeros(9, dtype=torch.int32, device="cuda:0")
    with pytest.raises(eu.EigError):
        eu.eig_location_rank2(dev_vec(lam[:1]), dev_colmajor(U[:1]), None, alpha, L)
    with pytest.raises(eu.EigError):
        eu.eig_location_rank2(dev_vec(lam), dev_colmajor(U), [1, 3], alpha, L)
    # sigma None reads as (+1, +1)
    eu.eig_location_rank2(dev_vec(lam), dev_colmajor(U), None, alpha, L)
    torch.cuda.synchronize()
    assert np.array_equal(host(L).astype(np.int64), oracle.location_vector(lam, U, np.array([1, 1], np.int8)))
