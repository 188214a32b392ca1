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
* ``low_rank``: exact rank-r products of two Gaussian factors;
* ``batched_shapes`` / ``batched_matrix``: the many-small-matrices workload
  (m log-uniform in [64, 1024], n log-uniform in [32, m],
  sigma_k = 10^(-8(k-1)/(n-1))), and ``batch_offsets`` for its packed layout.

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


def batched_shapes(count, seed, m_lo=64, m_hi=1024, n_lo=32):
    """``count`` shapes: m log-uniform in [m_lo, m_hi], then n log-uniform in
    [n_lo, m] (both rounded down to integers, n clamped to [n_lo, m])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = np.floor(np.exp(rng.uniform(np.log(m_lo), np.log(m_hi), count))).astype(np.int64)
    m = np.clip(m, m_lo, m_hi)
    u = rng.uniform(0.0, 1.0, count)
    n = np.floor(np.exp(np.log(n_lo) + u * (np.log(m) - np.log(n_lo)))).astype(np.int64)
    n = np.clip(n, n_lo, m)
    return m, n


def batched_sigma(n, decades=8.0):
    """sigma_k = 10^(-decades (k-1)/(n-1)), k = 1..n."""
    return geometric_sigma(n, -decades)


def batched_matrix(m, n, seed, decades=8.0):
    """One matrix of the batched workload: U diag(sigma) V^T, sigma geometric
    over ``decades`` decades."""
    return spectrum(m, n, batched_sigma(n, decades), seed)


def batch_offsets(m, n):
    """Packed layout of a batch: matrix i (column-major, lda = m_i) starts at
    element offset sum_{j<i} m_j n_j of A; its jpvt and tau start at
    sum_{j<i} n_j.  Returns (offA, offJ, totalA, totalJ)."""
    m = np.asarray(m, dtype=np.int64)
    n = np.asarray(n, dtype=np.int64)
    sizes = m * n
    offA = np.concatenate([[0], np.cumsum(sizes)[:-1]]) if len(m) else np.zeros(0, np.int64)
    offJ = np.concatenate([[0], np.cumsum(n)[:-1]]) if len(m) else np.zeros(0, np.int64)
    return offA.astype(np.int64), offJ.astype(np.int64), int(sizes.sum()), int(n.sum())


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


def batched_torch(m, n, seed, decades=8.0, device="cuda"):
    """The batched workload packed on the device (``batch_offsets`` layout):
    matrix i is U diag(sigma) V^T with U, V from torch QR of N(0,1) blocks drawn
    from a generator seeded with seed + i.  Returns a 1-D float64 tensor."""
    import torch
    offA, _, total, _ = batch_offsets(m, n)
    out = torch.empty(max(total, 1), dtype=torch.float64, device=device)
    g = torch.Generator(device=device)
    for i, (mi, ni) in enumerate(zip(m.tolist(), n.tolist())):
        g.manual_seed(int(seed) + i)
        sig = torch.as_tensor(batched_sigma(ni, decades), device=device)
        U, _ = torch.linalg.qr(torch.randn((mi, ni), generator=g, dtype=torch.float64, device=device))
        V, _ = torch.linalg.qr(torch.randn((ni, ni), generator=g, dtype=torch.float64, device=device))
        Ai = (U * sig[None, :]) @ V.t()
        out[offA[i]:offA[i] + mi * ni].copy_(Ai.t().reshape(-1))
    return out
