"""Pins of the oracle's rank-2 location vector (Algorithms 1a-1c), its
residues (eq. (3)) and the exact Sturm chain (Sec. 2.2).

The residues are checked against a determinant evaluated directly (numpy
LAPACK), the location vectors against interval counts of the dense updated
spectrum, and the Sturm count against both the dense spectrum and the inertia
count.  None of them re-types the oracle's formulas.
"""
import numpy as np
import pytest

import oracle

SIGNS = {"1a": (1, 1), "1b": (-1, -1), "1c": (1, -1), "1c'": (-1, 1)}


def _rank2(n, seed, spread=1.0, scale=0.6):
    rng = np.random.default_rng(seed)
    lam = np.sort(rng.standard_normal(n) * spread)
    U = rng.standard_normal((n, 2)) * scale
    return lam, U


def _dense_intervals(lam, U, s):
    A = np.diag(lam) + (U * np.asarray(s, dtype=float)[None, :]) @ U.T
    w = np.linalg.eigvalsh(A)
    edges = np.concatenate([[-np.inf], lam, [np.inf]])
    return np.array([np.sum((w > edges[i]) & (w < edges[i + 1])) for i in range(len(lam) + 1)]), w


def _well_posed(lam, U, s, w):
    """Residues and roots away from zero / the poles, so float signs are safe."""
    a = oracle.residues(lam, U, s)
    sep = np.min(np.abs(w[:, None] - lam[None, :]))
    return np.min(np.abs(a)) > 1e-8 * np.max(np.abs(a)) and sep > 1e-9


@pytest.mark.parametrize("k", [1, 2, 3])
def test_residues_reproduce_the_determinant(k):
    """f(x) = det(I - Sigma U^T (xI - Lam)^{-1} U) = 1 + sum alpha_i/(lam_i - x)."""
    rng = np.random.default_rng(40 + k)
    n = 9
    lam = np.sort(rng.standard_normal(n))
    U = rng.standard_normal((n, k)) * 0.7
    s = np.array([1, -1, 1][:k], dtype=np.int8)
    a = oracle.residues(lam, U, s)
    for x in rng.uniform(lam[0] - 1, lam[-1] + 1, size=25):
        d = 1.0 / (x - lam)
        F = np.eye(k) - np.diag(s.astype(float)) @ U.T @ (U * d[:, None])
        lhs = np.linalg.det(F)
        rhs = 1.0 + np.sum(a / (lam - x))
        scale = 1.0 + np.sum(np.abs(a / (lam - x)))
        assert abs(lhs - rhs) <= 1e-12 * scale


@pytest.mark.parametrize("case", ["1a", "1b", "1c", "1c'"])
@pytest.mark.parametrize("n", [2, 3, 5, 12, 40])
def test_location_vector_matches_dense_intervals(case, n):
    s = np.array(SIGNS[case], dtype=np.int8)
    done = 0
    for seed in range(60):
        lam, U = _rank2(n, 1000 * n + seed)
        ref, w = _dense_intervals(lam, U, s)
        if not _well_posed(lam, U, s, w):
            continue
        L = oracle.location_vector(lam, U, s)
        assert L.sum() == n
        assert np.array_equal(L, ref), (seed, L, ref)
        done += 1
        if done == 20:
            break
    assert done >= 10


def test_location_vector_agrees_with_inertia_counts():
    """L[i] = #{mu < lam_{i+1}} - #{mu < lam_i}, both from the pole-limit inertia count."""
    for case in SIGNS:
        s = np.array(SIGNS[case], dtype=np.int8)
        lam, U = _rank2(16, 77 + len(case))
        L = oracle.location_vector(lam, U, s)
        below = [0] + [oracle.pole_count(lam, U, s, p) for p in range(len(lam))]
        below.append(oracle.count(lam, U, s, float(lam[-1] + 1e3)))
        assert np.array_equal(L, np.diff(below)), case


def test_printed_1c_bound_misplaces_roots():
    """With opposite signs a root may lie one pole below its old eigenvalue,
    so #{mu < lam_{i+1}} reaches i+1; the 1a bound (M+2 > i) as printed for 1c
    then puts 0 where 2 roots lie.  The corrected bound is exact on the same
    problems."""
    s = np.array([1, -1], dtype=np.int8)
    wrong = 0
    for seed in range(30):
        lam, U = _rank2(12, 500 + seed)
        ref, w = _dense_intervals(lam, U, s)
        if not _well_posed(lam, U, s, w):
            continue
        assert np.array_equal(oracle.location_vector(lam, U, s), ref)
        if not np.array_equal(oracle.location_vector(lam, U, s, printed_1c=True), ref):
            wrong += 1
    assert wrong >= 10


def test_location_vector_interlacing_bounds():
    """1a: each L[i] <= 2 and at most i roots below lam_{i+1}; 1c: at most i+1."""
    for case, (lo_off, hi_off) in {"1a": (-1, 0), "1c": (0, 1)}.items():
        s = np.array(SIGNS[case], dtype=np.int8)
        lam, U = _rank2(30, 91)
        L = oracle.location_vector(lam, U, s)
        C = np.cumsum(L)[:-1]  # C[i] = roots below lam_{i+1} (0-based i)
        i = np.arange(len(lam))
        assert np.all(L <= 2)
        assert np.all(C <= i + hi_off) and np.all(C >= i + lo_off)


# --------------------------------------------------------------------------
# Sturm chain (Sec. 2.2) in exact rationals
# --------------------------------------------------------------------------
@pytest.mark.parametrize("k,s", [(1, (1,)), (1, (-1,)), (2, (1, 1)), (2, (1, -1)), (3, (1, -1, -1))])
def test_sturm_count_equals_inertia_and_dense_counts(k, s):
    rng = np.random.default_rng(7 + 3 * k + (s[-1] > 0))
    n = 5
    lam = np.sort(np.round(rng.standard_normal(n), 3))
    U = np.round(rng.standard_normal((n, k)) * 0.5, 3)
    sig = np.array(s, dtype=np.int8)
    chain = oracle.sturm_chain(lam, U, sig)
    assert len(chain[0]) == n + 1  # p_0 = det(xI - A') has degree n
    w = np.linalg.eigvalsh(np.diag(lam) + (U * sig.astype(float)[None, :]) @ U.T)
    xs = np.concatenate([rng.uniform(w[0] - 1, w[-1] + 1, size=12), lam + 1e-3])
    for x in xs:
        if np.min(np.abs(w - x)) < 1e-9:
            continue
        ref = int(np.sum(w < x))
        assert oracle.sturm_count(chain, x) == ref
        assert oracle.count(lam, U, sig, float(x)) == ref


def test_sturm_chain_of_a_known_polynomial():
    """lam = (0, 1), u = (1, 0), sigma = +1: the updated matrix is diag(1, 1),
    so p_0 = (x-1)^2 with one distinct root; the chain ends at p_0' and the
    count of distinct roots jumps by one at x = 1."""
    chain = oracle.sturm_chain(np.array([0.0, 1.0]), np.array([[1.0], [0.0]]), np.array([1], dtype=np.int8))
    assert [float(c) for c in chain[0]] == [1.0, -2.0, 1.0]
    assert oracle.sturm_count(chain, 0.5) == 0
    assert oracle.sturm_count(chain, 1.5) == 1  # distinct roots only


# --------------------------------------------------------------------------
# The secular-form Sturm chain (eqs. (4)-(9))
# --------------------------------------------------------------------------
def _tiny(n, k, s, seed):
    rng = np.random.default_rng(seed)
    lam = np.sort(np.round(rng.standard_normal(n), 3))
    U = np.round(rng.standard_normal((n, k)) * 0.5, 3)
    return lam, U, np.array(s, dtype=np.int8)


@pytest.mark.parametrize("n,k,s", [(4, 1, (1,)), (5, 2, (1, -1)), (6, 2, (-1, -1)), (6, 3, (1, 1, -1))])
def test_secular_chain_equals_the_polynomial_remainder_chain(n, k, s):
    """Secular long division yields -rem(p_{m-2}, p_{m-1}): every member equals
    the polynomial Sturm chain's member exactly, at exact rational points."""
    from fractions import Fraction

    lam, U, sig = _tiny(n, k, s, 100 + n + k)
    d, chain = oracle.secular_sturm_chain(lam, U, sig)
    poly = oracle.sturm_chain(lam, U, sig)
    assert len(chain) == n + 1 == len(poly)
    for x in [Fraction(-7, 3), Fraction(1, 7), Fraction(22, 5), d[1] + Fraction(1, 1000)]:
        vs = oracle.secular_sturm_values(d, chain, x)
        vp = [sum(c * x ** t for t, c in enumerate(p)) for p in poly]
        assert vs == vp


@pytest.mark.parametrize("n,k,s", [(5, 1, (-1,)), (6, 2, (1, -1)), (7, 2, (1, 1)), (7, 4, (1, -1, 1, -1))])
def test_secular_chain_counts_and_positive_leading_terms(n, k, s):
    """A symmetric matrix has n real roots, so on a simple spectrum every c_m is
    positive (the paper's test for a complete chain) and the chain's count
    equals the dense and the inertia counts."""
    lam, U, sig = _tiny(n, k, s, 300 + n * k)
    d, chain = oracle.secular_sturm_chain(lam, U, sig)
    w = np.linalg.eigvalsh(np.diag(lam) + (U * sig.astype(float)[None, :]) @ U.T)
    assert np.min(np.diff(w)) > 1e-6  # simple spectrum
    assert all(c > 0 for c, _ in chain)
    rng = np.random.default_rng(n)
    for x in np.concatenate([rng.uniform(w[0] - 1, w[-1] + 1, size=15), lam]):
        if np.min(np.abs(w - x)) < 1e-9:
            continue
        ref = int(np.sum(w < x))
        assert oracle.secular_sturm_count(d, chain, x) == ref
        if not np.any(lam == x):
            assert oracle.count(lam, U, sig, float(x)) == ref


def test_exact_residues_agree_with_the_float_residues():
    lam, U, sig = _tiny(7, 2, (1, -1), 9)
    _, a_exact = oracle._frac_residues(lam, U, sig)
    a = oracle.residues(lam, U, sig)
    ref = np.array([float(v) for v in a_exact])
    assert np.max(np.abs(a - ref) / np.abs(ref)) <= 1e-12


def test_root_deflation_eq9():
    """p_0^1(x) prod_p (x - xi_p) = p_0(x), and p_0^1 keeps the other roots."""
    rng = np.random.default_rng(12)
    n, k = 12, 2
    lam = np.sort(rng.standard_normal(n))
    U = rng.standard_normal((n, k)) * 0.5
    sig = np.array([1, -1], dtype=np.int8)
    A = np.diag(lam) + (U * sig.astype(float)[None, :]) @ U.T
    w = np.linalg.eigvalsh(A)
    alpha = oracle.residues(lam, U, sig)
    for s in (1, 3, 5):
        xi = w[:s]
        rest, beta = oracle.secular_deflate(lam, alpha, xi)

        def p01(x):
            return (1.0 - np.sum(beta / (x - rest))) * np.prod(x - rest)

        for x in rng.uniform(w[0] - 0.5, w[-1] + 0.5, size=10):
            p0 = np.linalg.det(x * np.eye(n) - A)
            scale = np.prod(np.abs(x - lam)) * (1 + np.sum(np.abs(alpha / (x - lam))))
            assert abs(p01(x) * np.prod(x - xi) - p0) <= 1e-10 * scale
        for r in w[s:]:
            terms = np.abs(beta / (r - rest))
            assert abs(1.0 - np.sum(beta / (r - rest))) <= 1e-9 * (1 + np.sum(terms))
