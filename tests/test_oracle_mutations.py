"""Planted mistakes in the oracle must be caught by its pins.

Each case compiles a copy of oracle/orc.c with one plausible slip (a sign, a
dropped term, an index off by one, the wrong null vector), swaps it in for the
real library on the CPU, and checks that the pin battery rejects it.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
import workloads

MUTATIONS = {
    "sigma_sign_in_count": ("Mk[IX(c, c, k)] -= (double)sigma[c];", "Mk[IX(c, c, k)] += (double)sigma[c];"),
    "dropped_reciprocal": ("    double r = 1.0 / d;\n    for (int b = 0; b < k; ++b) {",
                           "    double r = d;\n    for (int b = 0; b < k; ++b) {"),
    "k_plus_off_by_one": ("return below + neg - kplus_of(k, sigma);\n}\n\nint64_t orc_count",
                          "return below + neg - kplus_of(k, sigma) + 1;\n}\n\nint64_t orc_count"),
    "bracket_index": ("int64_t ilo = m - J->kminus, ihi = m + J->kplus;",
                      "int64_t ilo = m - J->kminus, ihi = m + J->kplus - 1;"),
    "wrong_null_vector": ("const double* a0 = V + (size_t)order[r] * k;",
                          "const double* a0 = V + (size_t)order[k - 1 - r] * k;"),
    "eq10_inverse_dropped": ("w[i] = ua / d;", "w[i] = ua * d;"),
    "transposed_U_in_M": ("Mk[IX(a, b, k)] += U[IX(i, a, n)] * ub;", "Mk[IX(a, b, k)] += U[IX(i, b, n)] * ub;"),
}


def _pins_pass() -> bool:
    """A compact battery of the pins in test_oracle_pins.py."""
    try:
        for n, k, sg in [(14, 3, "mixed"), (12, 1, "psd"), (10, 2, "psd")]:
            P = workloads.general(n, k, seed=n + k, sigma=sg, kscale=0.6)
            Q, lam, K, s = P["Q"], P["lam"], P["K"], P["sigma"]
            A = oracle.updated_matrix(Q, lam, K, s)
            ref = np.linalg.eigvalsh(A)
            out = oracle.update(Q, lam, K, s)
            if np.max(np.abs(out["mu"] - ref)) > 1e-12 * np.linalg.norm(A, 2):
                return False
            if np.max(oracle.residuals(Q, lam, K, s, out["mu"], out["X"])) > 1e-10 * np.linalg.norm(A, 2):
                return False
            U = oracle.project(Q, K)
            for x in np.linspace(ref[0] - 0.5, ref[-1] + 0.5, 37):
                if np.min(np.abs(ref - x)) > 1e-9 and oracle.count(lam, U, s, x) != int(np.sum(ref < x)):
                    return False
        return True
    except Exception:
        return False


@pytest.fixture(scope="module")
def src():
    with open(oracle._SRC) as f:
        return f.read()


def test_unmutated_oracle_passes_battery():
    assert _pins_pass()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name, src, tmp_path, monkeypatch):
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, "mutation anchor drifted: %s" % name
    c = tmp_path / "orc_mut.c"
    c.write_text(src.replace(old, new))
    so = tmp_path / "orc_mut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", str(so), str(c), "-lm"])
    monkeypatch.setattr(oracle, "_lib", oracle._bind(str(so)))
    assert not _pins_pass(), "planted mistake %s went unnoticed" % name
