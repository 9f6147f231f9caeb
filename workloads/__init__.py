"""Seeded synthetic inputs for the rank-k eigen-update.

This module is shared by the CUDA path's tests and bench and by the CPU oracle.
It only draws random numbers and builds orthogonal matrices: it holds none of
the update method's arithmetic (no projection, no secular function, no count).

Every generator takes a seed and returns plain numpy arrays (FP64):
    Q      n x n orthogonal, eigenvectors as columns
    lam    n, ascending
    K      n x k  (or (j, a) for the one-row-one-column form)
    sigma  k int8 entries of +1/-1

Recipes follow the paper's settings (random rank-2 and rank-k updates, Sec. 3)
at the sizes of the five workloads described in the project's design notes:
    small / rank2_basic   n=256,  k=2,  lam ~ U[-1,1], K ~ N(0,1)/sqrt(n), PSD
    indefinite_rank2      n=4096, e_j a^T + a e_j^T, lam ~ U[-10,10] with 5%
                          clustered pairs (gap 1e-8), 1% planted tiny rows of U
    general_rank_k        n=8192, k in {4,8,16}, lam = +-10^U[-3,3], K ~ N(0,1)/sqrt(n)
    batched               512 instances, n log-uniform [128,2048], k ~ U{1..8}
    serving               48 residents, n log-uniform [1024,8192], k ~ U{2..8}
"""
from __future__ import annotations

import math

import numpy as np


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def haar(n: int, rng: np.random.Generator, device=None, min_device_n: int = 1024) -> np.ndarray:
    """Haar-distributed orthogonal matrix: QR of a Gaussian matrix with the
    signs of diag(R) folded into Q (Mezzadri's recipe).  With a CUDA device the
    QR runs there for n >= min_device_n (input construction only), otherwise numpy."""
    G = rng.standard_normal((n, n))
    if device is not None and n >= min_device_n:
        import torch

        Gt = torch.from_numpy(G).to(device)
        Qt, Rt = torch.linalg.qr(Gt)
        d = torch.sign(torch.diagonal(Rt))
        d[d == 0] = 1.0
        Qt = Qt * d[None, :]
        Q = Qt.cpu().numpy()
        del Gt, Qt, Rt
    else:
        Qn, R = np.linalg.qr(G)
        d = np.sign(np.diag(R))
        d[d == 0] = 1.0
        Q = Qn * d[None, :]
    return np.ascontiguousarray(Q)


def _sorted_distinct_uniform(n: int, lo: float, hi: float, rng) -> np.ndarray:
    lam = np.sort(rng.uniform(lo, hi, size=n))
    # Uniform draws are distinct with probability one; enforce it anyway.
    for i in range(1, n):
        if lam[i] <= lam[i - 1]:
            lam[i] = np.nextafter(lam[i - 1], np.inf)
    return lam


def rank2_basic(seed: int = 0, n: int = 256, k: int = 2, device=None, min_device_n: int = 1024) -> dict:
    """Plain PSD rank-k update: lam ~ U[-1,1] sorted, Q Haar, K ~ N(0,1)/sqrt(n)."""
    rng = rng_for(seed)
    lam = _sorted_distinct_uniform(n, -1.0, 1.0, rng)
    Q = haar(n, rng, device, min_device_n)
    K = rng.standard_normal((n, k)) / math.sqrt(n)
    return dict(name="rank%d_psd_n%d" % (k, n), Q=Q, lam=lam, K=K,
                sigma=np.ones(k, dtype=np.int8))


def indefinite_rank2(seed: int = 1000, n: int = 4096, cluster_frac: float = 0.05,
                     cluster_gap: float = 1e-8, planted_frac: float = 0.01, device=None) -> dict:
    """One-row-one-column update e_j a^T + a e_j^T (Sec. 1 and 2.2).

    lam mixes U[-10,10] values with clustered pairs (base, base + gap); for a set
    P of planted indices the eigenvector column q_i is rotated (Givens, against
    a non-planted partner) so that Q[j,i] = 0, and a = Q z with z_i = 1e-15 g_i on
    P, so rows i in P of U = Q^T K are ~1e-14: the paper's nonzero-component
    condition fails there and those pairs must deflate.  Returns (j, a); the
    caller forms K and sigma with its own canonicalisation."""
    rng = rng_for(seed)
    npairs = int(math.floor(cluster_frac * n / 2))
    base = rng.uniform(-10.0, 10.0, size=n - npairs)
    bidx = rng.choice(n - npairs, size=npairs, replace=False)
    lam = np.sort(np.concatenate([base, base[bidx] + cluster_gap]))
    for i in range(1, n):
        if lam[i] <= lam[i - 1]:
            lam[i] = np.nextafter(lam[i - 1], np.inf)
    Q = haar(n, rng, device)
    j = int(rng.integers(0, n))
    nplant = int(round(planted_frac * n))
    perm = rng.permutation(n)
    planted = np.sort(perm[:nplant])
    partners = perm[nplant:2 * nplant]
    for i, p in zip(planted, partners):
        qi, qp = Q[j, i], Q[j, p]
        r = math.hypot(qi, qp)
        if r == 0.0:
            continue
        c, s = qp / r, qi / r
        ci, cp = Q[:, i].copy(), Q[:, p].copy()
        Q[:, i] = c * ci - s * cp
        Q[:, p] = s * ci + c * cp
        Q[j, i] = 0.0
    z = rng.standard_normal(n)
    z[planted] = 1e-15 * rng.standard_normal(nplant)
    a = Q @ z
    return dict(name="indefinite_rank2_n%d" % n, Q=np.ascontiguousarray(Q), lam=lam, j=j, a=a,
                planted=planted)


def general_rank_k(k: int = 8, seed: int = 2000, n: int = 8192, device=None) -> dict:
    """lam = s * 10^U[-3,3] with random sign s, Q Haar, K ~ N(0,1)/sqrt(n), PSD."""
    rng = rng_for(seed + k)
    mag = 10.0 ** rng.uniform(-3.0, 3.0, size=n)
    sgn = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    lam = np.sort(sgn * mag)
    for i in range(1, n):
        if lam[i] <= lam[i - 1]:
            lam[i] = np.nextafter(lam[i - 1], np.inf)
    Q = haar(n, rng, device)
    K = rng.standard_normal((n, k)) / math.sqrt(n)
    return dict(name="rank%d_logspec_n%d" % (k, n), Q=Q, lam=lam, K=K,
                sigma=np.ones(k, dtype=np.int8))


def batched_sizes(seed: int = 3000, count: int = 512, nmin: int = 128, nmax: int = 2048,
                  kmax: int = 8):
    """(n, k) per instance: n = round(exp U[ln nmin, ln nmax]), k ~ U{1..kmax}."""
    rng = rng_for(seed)
    ns = np.rint(np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=count))).astype(np.int64)
    ks = rng.integers(1, kmax + 1, size=count)
    return [(int(a), int(b)) for a, b in zip(ns, ks)]


def batched(seed: int = 3000, count: int = 512, nmin: int = 128, nmax: int = 2048,
            kmax: int = 8, device=None) -> list:
    """Independent instances, each drawn with the rank2_basic recipe."""
    out = []
    for t, (n, k) in enumerate(batched_sizes(seed, count, nmin, nmax, kmax)):
        out.append(rank2_basic(seed=seed * 1000 + t, n=n, k=k, device=device, min_device_n=256))
    return out


def random_sigma(k: int, rng, kminus: int | None = None) -> np.ndarray:
    s = np.ones(k, dtype=np.int8)
    if kminus is None:
        kminus = int(rng.integers(0, k + 1))
    s[rng.permutation(k)[:kminus]] = -1
    return s


def general(n: int, k: int, seed: int, sigma="psd", lam_kind: str = "uniform",
            kscale: float | None = None) -> dict:
    """Small general problems for tests: any n, k, sign pattern and spectrum."""
    rng = rng_for(seed)
    if lam_kind == "uniform":
        lam = _sorted_distinct_uniform(n, -1.0, 1.0, rng)
    elif lam_kind == "logspec":
        lam = np.sort(np.where(rng.random(n) < 0.5, -1.0, 1.0) * 10.0 ** rng.uniform(-3, 3, size=n))
    elif lam_kind == "clustered":
        npairs = max(1, n // 10)
        base = rng.uniform(-10.0, 10.0, size=n - npairs)
        lam = np.sort(np.concatenate([base, base[rng.choice(n - npairs, npairs, replace=False)] + 1e-8]))
    elif lam_kind == "constant":
        lam = np.full(n, 0.375)
    elif lam_kind == "repeated":
        # runs of exactly equal values: singles, pairs, and runs longer than k
        sizes = []
        while sum(sizes) < n:
            sizes.append(int(rng.choice([1, 1, 1, 2, 3, k + 1, 2 * k + 3])))
        sizes[-1] -= sum(sizes) - n
        lam = np.repeat(_sorted_distinct_uniform(len(sizes), -1.0, 1.0, rng), sizes)
    else:
        raise ValueError(lam_kind)
    Q = haar(n, rng)
    K = rng.standard_normal((n, k)) * (kscale if kscale is not None else 1.0 / math.sqrt(n))
    if isinstance(sigma, str):
        if sigma == "psd":
            s = np.ones(k, dtype=np.int8)
        elif sigma == "nsd":
            s = -np.ones(k, dtype=np.int8)
        elif sigma == "mixed":
            s = random_sigma(k, rng, kminus=max(1, k // 2) if k > 1 else 0)
        else:
            raise ValueError(sigma)
    else:
        s = np.asarray(sigma, dtype=np.int8)
    return dict(name="general_n%d_k%d" % (n, k), Q=Q, lam=lam, K=K, sigma=s)


def serving_plan(seed: int = 4000, residents: int = 48, nmin: int = 1024, nmax: int = 8192,
                 chain: int = 100, kmin: int = 2, kmax: int = 8):
    """Resident sizes and the chained request list (resident id, k, seed) in arrival order."""
    rng = rng_for(seed)
    ns = np.rint(np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=residents))).astype(np.int64)
    reqs = []
    for step in range(chain):
        for r in rng.permutation(residents):
            reqs.append((int(r), int(rng.integers(kmin, kmax + 1)), int(seed * 100000 + step * 1000 + r)))
    return [int(x) for x in ns], reqs


def poisson_arrivals(rate_per_s: float, count: int, seed: int) -> np.ndarray:
    """Arrival offsets (s) of a Poisson stream."""
    rng = rng_for(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


def chained_K(n: int, k: int, seed: int) -> np.ndarray:
    rng = rng_for(seed)
    return rng.standard_normal((n, k)) / math.sqrt(n)


def small_k(n: int = 100, k: int = 2, knorm: float = 0.01, seed: int = 5000, sigma="psd") -> dict:
    """The Figs. 6-7 shape: N = 100 (by default), lam ~ U[-1,1] sorted, Q Haar,
    K Gaussian rescaled to the 2-norm knorm (0.01 and 0.3 in the figures)."""
    rng = rng_for(seed)
    lam = _sorted_distinct_uniform(n, -1.0, 1.0, rng)
    Q = haar(n, rng)
    K = rng.standard_normal((n, k))
    K *= knorm / np.linalg.norm(K, 2)
    s = np.ones(k, dtype=np.int8) if sigma == "psd" else np.asarray(
        random_sigma(k, rng, kminus=max(1, k // 2) if k > 1 else 0) if sigma == "mixed" else sigma, dtype=np.int8)
    return dict(name="small_k_n%d_k%d" % (n, k), Q=Q, lam=lam, K=K, sigma=s)
