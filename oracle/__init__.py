"""Plain FP64 CPU oracle for BQRRP -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
library never loads it and it never loads the CUDA library.

The arithmetic lives in ``bqrrp_oracle.c`` (plain loops, no BLAS); this module
only compiles it with gcc on first use and marshals numpy arrays through
ctypes.  Function names follow the paper's notation (Alg. 1-3, Alg. 5).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bqrrp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int64)
_u32p = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (plain -O2, IEEE
    arithmetic: no fast-math and no FMA contraction; OpenMP for the loops over
    independent columns, which leaves every result bit for bit unchanged)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-fopenmp", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.bqrrp_ref_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
            L.bqrrp_ref_sketch_dense.argtypes = [_i64, _i64, _u64, _dp]
            L.bqrrp_ref_sketch_sparse.argtypes = [_i64, _i64, _u64, _i64, _dp]
            L.bqrrp_ref_sketch_sparse.restype = ctypes.c_int
            L.bqrrp_ref_sketch_apply.argtypes = [_i64, _i64, _i64, _dp, _dp, _i64, _dp, _i64]
            L.bqrrp_ref_geqrf.argtypes = [_i64, _i64, _dp, _i64, _dp]
            L.bqrrp_ref_qrcp_bg.argtypes = [_i64, _i64, _dp, _i64, _ip, _dp]
            L.bqrrp_ref_lupp.argtypes = [_i64, _i64, _dp, _i64, _ip, _dp]
            L.bqrrp_ref_lupp.restype = _i64
            L.bqrrp_ref_piv_transform.argtypes = [_i64, _i64, _ip, _ip]
            L.bqrrp_ref_orhr_col.argtypes = [_i64, _i64, _dp, _i64, _dp, _i64, _dp]
            L.bqrrp_ref_cholqr_panel.argtypes = [_i64, _i64, _i64, _dp, _i64, _dp, _i64, _dp, _i64, _dp]
            L.bqrrp_ref_cholqr_panel.restype = _i64
            L.bqrrp_ref_factor.argtypes = [_i64, _i64, _dp, _i64, _i64, _i64, _u64, ctypes.c_int, _i64,
                                           ctypes.c_int, _ip, _dp, _ip, _dp, _i64, _i64, _dp]
            L.bqrrp_ref_factor.restype = ctypes.c_int
            L.bqrrp_ref_trunc_rank.argtypes = [_i64, _i64, _dp, _i64, _i64, ctypes.c_double, ctypes.c_double]
            L.bqrrp_ref_trunc_rank.restype = _i64
            L.bqrrp_ref_fro_norm.argtypes = [_i64, _i64, _dp, _i64]
            L.bqrrp_ref_fro_norm.restype = ctypes.c_double
            L.bqrrp_ref_set_threads.argtypes = [ctypes.c_int]
            L.bqrrp_ref_get_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def set_threads(t):
    """Threads of the oracle's parallel loops (1, the default, runs serially).
    The results are identical for every thread count."""
    lib().bqrrp_ref_set_threads(int(t))


def get_threads():
    return int(lib().bqrrp_ref_get_threads())


def _f(a):
    """Fortran-ordered float64 copy."""
    return np.array(a, dtype=np.float64, order="F", copy=True)


def _p(a, t=_dp):
    return a.ctypes.data_as(t)


def philox4x32_10(ctr, key):
    """One Philox4x32-10 block (Salmon et al., SC'11): 4 counter words, 2 key words."""
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().bqrrp_ref_philox4x32_10(_p(c, _u32p), _p(k, _u32p), _p(out, _u32p))
    return out


def sketch_operator(d, m, seed, kind=0, nnz=8):
    """The d x m sketching operator S (Alg. 1 sample step): kind 0 dense +-1,
    kind 1 sparse sign with ``nnz`` nonzeros per column."""
    S = np.zeros((d, m), dtype=np.float64, order="F")
    if kind == 0:
        lib().bqrrp_ref_sketch_dense(d, m, seed, _p(S))
    else:
        rc = lib().bqrrp_ref_sketch_sparse(d, m, seed, nnz, _p(S))
        if rc != 0:
            raise ValueError(f"sketch_sparse failed: {rc}")
    return S


def sketch_apply(S, A):
    """Msk = S @ A with a plain triple loop."""
    S = _f(S); A = _f(A)
    d, m = S.shape
    m2, n = A.shape
    assert m == m2
    out = np.zeros((d, n), dtype=np.float64, order="F")
    lib().bqrrp_ref_sketch_apply(d, m, n, _p(S), _p(A), max(m, 1), _p(out), max(d, 1))
    return out


def geqrf(A):
    """Unpivoted Householder QR; returns (A overwritten GEQRF-style, tau)."""
    A = _f(A)
    m, n = A.shape
    tau = np.zeros(min(m, n), dtype=np.float64)
    lib().bqrrp_ref_geqrf(m, n, _p(A), max(m, 1), _p(tau))
    return A, tau


def qrcp_bg(A):
    """Businger-Golub QRCP; returns (A overwritten GEQP3-style, jpvt 1-based, tau)."""
    A = _f(A)
    m, n = A.shape
    jpvt = np.zeros(n, dtype=np.int64)
    tau = np.zeros(n, dtype=np.float64)
    lib().bqrrp_ref_qrcp_bg(m, n, _p(A), max(m, 1), _p(jpvt, _ip), _p(tau))
    return A, jpvt, tau[: min(m, n)]


def lupp(X):
    """Row-pivoted LU (GETRF rule): returns (LU in place, ipiv 0-based swap sequence, margin)."""
    X = _f(X)
    N, d = X.shape
    ipiv = np.zeros(max(min(N, d), 1), dtype=np.int64)
    margin = ctypes.c_double(0.0)
    steps = lib().bqrrp_ref_lupp(N, d, _p(X), max(N, 1), _p(ipiv, _ip), ctypes.byref(margin))
    return X, ipiv[:steps], margin.value


def piv_transform(N, ipiv):
    """Swap-sequence pivots -> permutation format (0-based), Alg. 2."""
    ipiv = np.ascontiguousarray(ipiv, dtype=np.int64)
    J = np.zeros(max(N, 1), dtype=np.int64)
    lib().bqrrp_ref_piv_transform(N, len(ipiv), _p(ipiv, _ip), _p(J, _ip))
    return J[:N]


def orhr_col(Q):
    """Householder reconstruction of an explicit orthonormal Q (rows x k):
    returns (Y unit-lower trapezoidal, T k x k upper, D signs)."""
    Y = _f(Q)
    rows, k = Y.shape
    T = np.zeros((k, k), dtype=np.float64, order="F")
    D = np.zeros(k, dtype=np.float64)
    lib().bqrrp_ref_orhr_col(rows, k, _p(Y), max(rows, 1), _p(T), max(k, 1), _p(D))
    return Y, T, D


def cholqr_panel(M, Rsk, k):
    """Alg. 3 on one panel: returns (panel with R11 and reflectors, T (k x k),
    tau, k kept)."""
    M = _f(M)
    Rsk = _f(Rsk)
    rows, w = M.shape
    T = np.zeros((max(k, 1), max(k, 1)), dtype=np.float64, order="F")
    tau = np.zeros(max(k, 1), dtype=np.float64)
    kc = lib().bqrrp_ref_cholqr_panel(rows, w, k, _p(M), max(rows, 1), _p(Rsk), max(Rsk.shape[0], 1),
                                      _p(T), max(k, 1), _p(tau))
    return M, T[:k, :k], tau[:k], kc


class Factorization:
    """GEQP3-format result: ``A`` (R above the diagonal, reflectors below),
    ``jpvt`` (1-based), ``tau``, ``rank`` and the per-iteration ``trace``
    (k, min LU pivot margin, non-finite-sketch flag, w)."""

    def __init__(self, A, jpvt, tau, rank, trace):
        self.A, self.jpvt, self.tau, self.rank, self.trace = A, jpvt, tau, rank, trace


def bqrrp(A, b, d, seed, sketch_kind=0, nnz=8, panel="cholqr", max_iters=0, want_sketch=False):
    """BQRRP (Alg. 1) with Alg. 2 on the sketch and the Alg. 3 CholQR panel
    (``panel='cholqr'``) or a Householder panel (``panel='hqr'``).
    ``max_iters``/``want_sketch`` are test hooks: stop after that many
    iterations and return the sketch buffer as ``.sketch``."""
    A = _f(A)
    m, n = A.shape
    jpvt = np.zeros(max(n, 1), dtype=np.int64)
    tau = np.zeros(max(n, 1), dtype=np.float64)
    rank = ctypes.c_int64(0)
    iters = max(1, -(-n // b)) if b > 0 else 1
    trace = np.zeros(4 * iters, dtype=np.float64)
    sk = np.zeros((d, max(n, 1)), dtype=np.float64, order="F") if want_sketch else None
    rc = lib().bqrrp_ref_factor(m, n, _p(A), max(m, 1), b, d, seed, int(sketch_kind), nnz,
                                0 if panel == "cholqr" else 1, _p(jpvt, _ip), _p(tau),
                                ctypes.byref(rank), _p(trace), iters, int(max_iters),
                                _p(sk) if sk is not None else None)
    if rc != 0:
        raise RuntimeError(f"bqrrp_ref_factor returned {rc}")
    r = rank.value
    used = 0
    tr = []
    for i in range(iters):
        if trace[4 * i + 3] == 0:
            break
        tr.append(dict(k=int(trace[4 * i]), margin=float(trace[4 * i + 1]),
                       nonfinite=bool(trace[4 * i + 2]), w=int(trace[4 * i + 3])))
        used += 1
    f = Factorization(A, jpvt[:n], tau[:n], r, tr)
    f.sketch = sk
    return f


def bqrrp_status(A, b, d, seed=0, sketch_kind=0, nnz=8, lda=None):
    """Return code of the oracle's argument checks (for edge-case tests)."""
    A = _f(A) if A is not None else np.zeros((1, 1), order="F")
    m, n = A.shape
    jpvt = np.zeros(max(n, 1), dtype=np.int64)
    tau = np.zeros(max(n, 1), dtype=np.float64)
    rank = ctypes.c_int64(0)
    return lib().bqrrp_ref_factor(m, n, _p(A), lda if lda is not None else max(m, 1), b, d, seed,
                                  int(sketch_kind), nnz, 0, _p(jpvt, _ip), _p(tau), ctypes.byref(rank),
                                  None, 0, 0, None)


def fro_norm(A):
    """||A||_F as a plain sum of squares."""
    A = _f(A)
    m, n = A.shape
    return lib().bqrrp_ref_fro_norm(m, n, _p(A), max(m, 1))


def trunc_rank(F, rank, anorm, tol):
    """Rank-revealing truncation on a factored A (GEQP3 storage): the smallest i
    with ||R(i:rank, i:n)||_F <= tol * anorm (the Sec. 6 residual measure as a
    rule; rows at and below ``rank`` count as zero)."""
    F = _f(F)
    m, n = F.shape
    return int(lib().bqrrp_ref_trunc_rank(m, n, _p(F), max(m, 1), int(rank), float(anorm), float(tol)))


class BatchedResult:
    """Per-matrix results of ``bqrrp_batched``: lists ``F``, ``jpvt``, ``tau``,
    ``rank``, ``trunc_rank`` and ``trace`` (each entry as for ``bqrrp``)."""

    def __init__(self):
        self.F, self.jpvt, self.tau, self.rank, self.trunc_rank, self.trace = [], [], [], [], [], []


def bqrrp_batched(mats, bs, ds, seeds, tol):
    """Many independent BQRRP factorizations (Alg. 1 with the Alg. 3 panel),
    each with its own block size, sketch size and seed, followed by the
    truncation rule.  A plain loop over ``bqrrp``: the batched workload has no
    arithmetic of its own beyond the truncation post-pass."""
    out = BatchedResult()
    for A, b, d, sd in zip(mats, bs, ds, seeds):
        f = bqrrp(A, int(b), int(d), int(sd))
        out.F.append(f.A)
        out.jpvt.append(f.jpvt)
        out.tau.append(f.tau)
        out.rank.append(f.rank)
        out.trace.append(f.trace)
        out.trunc_rank.append(trunc_rank(f.A, f.rank, fro_norm(A), tol))
    return out
