"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generation only -- none of the factorization's
arithmetic -- so that the CUDA path and the CPU oracle can be fed the very same
bytes.  Families (paper Sec. 1.4 and Sec. 6):

* ``gaussian``: iid N(0,1) entries (the paper's performance matrices);
* ``spectrum``: U diag(sigma) V^T with U, V orthonormal from the QR of seeded
  N(0,1) matrices (used for pivot-quality and rank checks);
* ``c1_matrix``: the 2000 x 1000 matrix with sigma_k = 10^(-10(k-1)/999),
  U, V from numpy PCG64 seed 0;
* ``kahan``: the Kahan matrix of Sec. 6 (alpha = sin(theta), beta = -cos(theta),
  plus eps*p*diag(n, ..., 1));
* ``low_rank``: exact rank-r products of two Gaussian factors.

Large matrices are generated on the GPU with torch (untimed test tooling).
"""
from __future__ import annotations

import numpy as np


def _orthonormal(rng, rows, cols):
    q, r = np.linalg.qr(rng.standard_normal((rows, cols)))
    return q * np.sign(np.diag(r))[None, :]


def gaussian(m, n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.asfortranarray(rng.standard_normal((m, n)))


def spectrum(m, n, sigma, seed):
    """U diag(sigma) V^T with min(m, n) singular values ``sigma``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = min(m, n)
    sigma = np.asarray(sigma, dtype=np.float64)
    assert sigma.shape == (k,)
    U = _orthonormal(rng, m, k)
    V = _orthonormal(rng, n, k)
    return np.asfortranarray((U * sigma[None, :]) @ V.T)


def geometric_sigma(k, lo_exp):
    """sigma_j = 10^(lo_exp * j / (k-1)), j = 0..k-1 (1 down to 10^lo_exp)."""
    if k == 1:
        return np.ones(1)
    return 10.0 ** (lo_exp * np.arange(k) / (k - 1))


def c1_matrix():
    """2000 x 1000, sigma_k = 10^(-10(k-1)/999), U and V from PCG64 seed 0."""
    return spectrum(2000, 1000, geometric_sigma(1000, -10.0), 0)


def low_rank(m, n, r, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.asfortranarray(rng.standard_normal((m, r)) @ rng.standard_normal((r, n)))


def kahan(n, p=1000.0, theta=1.2):
    """Kahan matrix (Sec. 6): diag(1, a, ..., a^{n-1}) * (upper triangle with
    beta on the diagonal and 1 above) + eps * p * diag(n, ..., 1)."""
    a = np.sin(theta)
    beta = -np.cos(theta)
    U = np.triu(np.ones((n, n)), 1) + beta * np.eye(n)
    D = a ** np.arange(n)
    eps = np.finfo(np.float64).eps
    return np.asfortranarray(D[:, None] * U + eps * p * np.diag(np.arange(n, 0, -1, dtype=np.float64)))


# --------------------------- device generators ---------------------------

def gaussian_torch(m, n, seed, device="cuda"):
    """iid N(0,1), column-major m x n float64 tensor (storage n x m transposed view)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return torch.randn((n, m), generator=g, dtype=torch.float64, device=device).t()


def spectrum_torch(m, n, sigma, seed, device="cuda"):
    """U diag(sigma) V^T on the device, U and V from torch QR of N(0,1) blocks."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    k = min(m, n)
    sig = torch.as_tensor(np.asarray(sigma, dtype=np.float64), device=device)
    U, _ = torch.linalg.qr(torch.randn((m, k), generator=g, dtype=torch.float64, device=device))
    V, _ = torch.linalg.qr(torch.randn((n, k), generator=g, dtype=torch.float64, device=device))
    A = (U * sig[None, :]) @ V.t()
    del U, V
    return A.t().contiguous().t()
