"""Helpers shared by the GPU tests: device copies in the library's layout."""
import numpy as np


def dev_colmajor(a):
    import torch

    return torch.from_numpy(np.asfortranarray(np.asarray(a, dtype=np.float64))).to("cuda:0")


def dev_vec(a, dtype=None):
    import torch

    a = np.ascontiguousarray(a)
    return torch.from_numpy(a).to("cuda:0")


def host(t):
    return t.detach().cpu().numpy()


def norm2_A(lam, K, sigma=None):
    """||A'||_2 upper bound used as the tolerance scale: max|lam| + sum |K_c|^2."""
    return float(np.max(np.abs(lam))) + float(np.sum(np.asarray(K) ** 2))


def cos_match(X, Y):
    """|cos| between matching columns (eigenvectors are defined up to sign)."""
    nx = np.linalg.norm(X, axis=0)
    ny = np.linalg.norm(Y, axis=0)
    return np.abs(np.sum(X * Y, axis=0)) / (nx * ny)
