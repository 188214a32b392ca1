"""Numpy checkers for GEQP3-format factorizations (test code only).

Everything here is written from the output-format definition of Sec. 1.3:
Q = H_1 H_2 ... H_l with H_i = I - tau_i v_i v_i^T, v_i(i) = 1, v_i(:i) = 0 and
v_i(i+1:) stored below the diagonal; R in the upper trapezoid; J 1-based.
"""
from __future__ import annotations

import numpy as np


def form_q_slow(F, tau, ell):
    """Explicit m x m Q, one reflector at a time (small inputs)."""
    m = F.shape[0]
    Q = np.eye(m)
    for i in reversed(range(ell)):
        v = np.zeros(m)
        v[i] = 1.0
        v[i + 1:] = F[i + 1:, i]
        Q -= tau[i] * np.outer(v, v @ Q)
    return Q


def form_q(F, tau, ell):
    """Explicit m x m Q through LAPACK dorgqr (a library cross-check)."""
    from scipy.linalg import lapack
    m, n = F.shape
    if ell == 0:
        return np.eye(m)
    W = np.zeros((m, m), order="F")
    W[:, :ell] = F[:, :ell]
    t = np.zeros(m)
    t[:ell] = tau[:ell]
    Q, _work, info = lapack.dorgqr(W, t)
    assert info == 0
    return Q


def upper_r(F, ell):
    """R: rows 0..ell-1 of the upper trapezoid of F (zeros elsewhere)."""
    m, n = F.shape
    R = np.triu(F)[:m, :]
    R[ell:, :] = 0.0
    return R


def metrics(A, F, jpvt, tau, ell):
    """Relative residual ||AP - QR||_F/||A||_F, orthogonality ||Q^TQ-I||_F,
    and whether jpvt is a 1-based permutation."""
    A = np.asarray(A)
    m, n = A.shape
    Q = form_q(F, tau, ell)
    R = upper_r(F, ell)
    AP = A[:, np.asarray(jpvt) - 1]
    nrm = np.linalg.norm(A)
    res = np.linalg.norm(AP - Q @ R) / (nrm if nrm > 0 else 1.0)
    orth = np.linalg.norm(Q.T @ Q - np.eye(m))
    perm_ok = sorted(np.asarray(jpvt).tolist()) == list(range(1, n + 1))
    return res, orth, perm_ok


def trailing_norms(F, ell, cols=None):
    """||R(i:, i:)||_F for i in ``cols`` (default 0..n-1) with R from F."""
    R = upper_r(F, ell)
    m, n = F.shape
    if cols is None:
        cols = range(n)
    out = []
    for i in cols:
        out.append(np.linalg.norm(R[i:, i:]))
    return np.array(out)
