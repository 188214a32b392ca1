"""ctypes binding of ``libbqrrp.so`` (argument marshalling only).

Each function mirrors one entry point of ``include/bqrrp.h`` under the same
name; every step of the computation runs in the library's CUDA kernels.
Matrices are torch float64 tensors in column-major layout (``stride(0) == 1``,
``stride(1)`` = leading dimension), on the current CUDA device; the current
torch stream is passed to the library.  ``colmajor_empty``/``to_colmajor``
build such tensors.

There is no fallback: if the shared library is missing or fails to load, the
first call raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbqrrp.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "bqrrp.h")

OK, ENOMEM, ECUDA, ENUMERIC, ETIMEOUT, EUNSUPPORTED = 0, 1, 2, 3, 4, 5
SKETCH_DENSE, SKETCH_SPARSE = 0, 1
PANEL_CHOLQR, PANEL_HQR = 0, 1
PRECISION_FP64, PRECISION_MIXED, PRECISION_MIXED_SKETCH32 = 0, 1, 2
_PRECISIONS = {"fp64": PRECISION_FP64, "mixed": PRECISION_MIXED, "mixed_sketch32": PRECISION_MIXED_SKETCH32}
SCHEDULE_OVERLAP, SCHEDULE_SERIAL = 0, 1
BATCH_PERSISTENT, BATCH_LOCKSTEP = 0, 1

_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_d = ctypes.c_double
_lock = threading.Lock()
_lib = None


class Opts(ctypes.Structure):
    _fields_ = [("sketch_kind", ctypes.c_int), ("sketch_nnz", _i64), ("panel_kind", ctypes.c_int),
                ("precision", _i64), ("schedule", _i64), ("panel_tc", _i64), ("reserved", _i64 * 2)]


NPHASES = 8
PHASES = ["sketch", "lupp", "sketch_qr", "permute", "panel", "trailing", "sketch_update", "other"]


class Profile(ctypes.Structure):
    _fields_ = [("ms", _d * NPHASES), ("flops", _d * NPHASES), ("calls", _i64)]


class Request(ctypes.Structure):
    _fields_ = [("id", _u64), ("m", _i64), ("n", _i64), ("b", _i64), ("d", _i64), ("seed", _u64),
                ("A_host", _vp), ("A_out_host", _vp), ("jpvt_out_host", _vp), ("tau_out_host", _vp)]


class Completion(ctypes.Structure):
    _fields_ = [("id", _u64), ("status", ctypes.c_int32), ("lane", ctypes.c_int32), ("rank", _i64),
                ("trunc_rank", _i64), ("t_submit", _d), ("t_admit", _d), ("t_start", _d), ("t_done", _d)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", _i64), ("completed", _i64), ("batches", _i64), ("max_batch", _i64),
                ("large_runs", _i64), ("peak_request_bytes", _i64), ("request_arena_bytes", _i64),
                ("in_use_bytes", _i64)]


SERVER_DRYRUN = 1
SERVER_MIXED = 2


class BqrrpError(RuntimeError):
    def __init__(self, fn, code, msg):
        super().__init__(f"{fn} returned {code}: {msg}")
        self.code = code


_SIGS = {
    "bqrrp_factor": ([_i64, _i64, _vp, _i64, _i64, _i64, _u64, _vp, _vp, ctypes.POINTER(_i64), ctypes.POINTER(Opts),
                      _vp, _sz, _vp], ctypes.c_int),
    "bqrrp_workspace_query": ([_i64, _i64, _i64, _i64, ctypes.POINTER(Opts)], _sz),
    "bqrrp_factor_host": ([_i64, _i64, _vp, _i64, _i64, _i64, _u64, _vp, _vp, ctypes.POINTER(_i64),
                           ctypes.POINTER(Opts), _vp, _sz, _vp], ctypes.c_int),
    "bqrrp_workspace_query_host": ([_i64, _i64, _i64, _i64, ctypes.POINTER(Opts)], _sz),
    "bqrrp_sketch_operator": ([_i64, _i64, _u64, ctypes.c_int, _i64, _vp, _i64, _vp], ctypes.c_int),
    "bqrrp_sketch_apply": ([_i64, _i64, _i64, _vp, _i64, _u64, ctypes.c_int, _i64, _vp, _i64, _vp, _sz, _vp],
                           ctypes.c_int),
    "bqrrp_sketch_apply_workspace": ([_i64, _i64, ctypes.c_int, _i64], _sz),
    "bqrrp_sketch_apply_sparse_noalloc": ([_i64, _i64, _i64, _vp, _i64, _u64, _i64, _vp, _i64, _vp], ctypes.c_int),
    "bqrrp_qrcp_wide": ([_i64, _i64, _vp, _i64, _vp, _vp, _vp, _sz, _vp], ctypes.c_int),
    "bqrrp_qrcp_wide_workspace": ([_i64, _i64], _sz),
    "bqrrp_selftest_lu_wait_timeout": ([_i64, _i64, _vp, _i64, _vp, _vp, _sz, _vp], ctypes.c_int),
    "bqrrp_col_perm": ([_i64, _i64, _vp, _i64, _vp, _i64, _vp, _sz, _vp], ctypes.c_int),
    "bqrrp_col_perm_workspace": ([_i64, _i64, _i64], _sz),
    "bqrrp_cholqr_panel": ([_i64, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _vp, ctypes.POINTER(_i64), _vp, _sz,
                            _vp], ctypes.c_int),
    "bqrrp_cholqr_panel_workspace": ([_i64, _i64], _sz),
    "bqrrp_geqrf": ([_i64, _i64, _vp, _i64, _vp, _i64, _vp, _sz, _vp], ctypes.c_int),
    "bqrrp_geqrf_workspace": ([_i64, _i64, _i64], _sz),
    "bqrrp_geqrf_mixed": ([_i64, _i64, _vp, _i64, _vp, _vp, _sz, _vp], ctypes.c_int),
    "bqrrp_geqrf_mixed_workspace": ([_i64, _i64], _sz),
    "bqrrp_dgemm": ([ctypes.c_char, ctypes.c_char, _i64, _i64, _i64, _d, _vp, _i64, _vp, _i64, _d, _vp, _i64, _vp,
                     _sz, _vp], ctypes.c_int),
    "bqrrp_dgemm_workspace": ([_i64, _i64, _i64], _sz),
    "bqrrp_probe_fp64_peak": ([ctypes.c_int, _vp], _d),
    "bqrrp_dgemm_ozaki": ([ctypes.c_char, ctypes.c_char, _i64, _i64, _i64, _d, _vp, _i64, _vp, _i64, _d, _vp, _i64,
                           _vp, _sz, _vp], ctypes.c_int),
    "bqrrp_dgemm_ozaki_workspace": ([_i64, _i64, _i64], _sz),
    "bqrrp_sketch_apply_tc": ([_i64, _i64, _i64, _vp, _i64, _u64, _vp, _i64, _vp, _sz, _vp], ctypes.c_int),
    "bqrrp_sketch_apply_tc_workspace": ([_i64, _i64, _i64], _sz),
    "bqrrp_batch_plan_create": ([ctypes.POINTER(_vp), _i64, _vp, _vp, _vp, _vp, _vp, _d], ctypes.c_int),
    "bqrrp_batch_plan_create_tiles": ([ctypes.POINTER(_vp), _i64, _vp, _vp, _vp, _vp, _vp, _vp, _d], ctypes.c_int),
    "bqrrp_batch_workspace_bytes": ([_vp], _sz),
    "bqrrp_batch_factor": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp, ctypes.c_int], ctypes.c_int),
    "bqrrp_batch_plan_destroy": ([_vp], None),
    "bqrrp_batch_launches": ([_vp], ctypes.c_int),
    "bqrrp_batch_plan_set_form": ([_vp, ctypes.c_int], ctypes.c_int),
    "bqrrp_batch_flops": ([_vp, ctypes.c_int], _d),
    "bqrrp_batch_autotune_workspace_bytes": ([_i64, _vp, _vp], _sz),
    "bqrrp_batch_autotune_tiles": ([_i64, _vp, _vp, _vp, _vp, _d, _vp, _sz, _vp, _vp, _vp, _vp, ctypes.POINTER(_d)],
                                   ctypes.c_int),
    "bqrrp_batch_autotune": ([_i64, _vp, _vp, _vp, _vp, _d, _vp, _sz, _vp, _vp, _vp, ctypes.POINTER(_d)],
                             ctypes.c_int),
    "bqrrp_server_create": ([ctypes.POINTER(_vp), _sz, _sz, _d, _i64, ctypes.c_int, _d], ctypes.c_int),
    "bqrrp_server_submit": ([_vp, ctypes.POINTER(Request)], ctypes.c_int),
    "bqrrp_server_poll": ([_vp, ctypes.POINTER(Completion), ctypes.c_int, _d], ctypes.c_int),
    "bqrrp_server_drain": ([_vp], ctypes.c_int),
    "bqrrp_server_clock": ([_vp], _d),
    "bqrrp_server_last_error": ([_vp], ctypes.c_char_p),
    "bqrrp_server_get_stats": ([_vp, ctypes.POINTER(ServerStats)], ctypes.c_int),
    "bqrrp_server_destroy": ([_vp], None),
    "bqrrp_profile_enable": ([ctypes.c_int], None),
    "bqrrp_profile_reset": ([], None),
    "bqrrp_profile_read": ([ctypes.POINTER(Profile)], ctypes.c_int),
    "bqrrp_launch_counter": ([], _i64),
    "bqrrp_last_error": ([], ctypes.c_char_p),
    "bqrrp_version": ([], ctypes.c_char_p),
}


def header_symbols():
    """Names of the functions declared in include/bqrrp.h."""
    with open(HEADER) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(bqrrp_\w+)\s*\(", text, flags=re.M)))


def lib():
    """Load libbqrrp.so (raises if it is missing: there is no CPU fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2507_00976_b300.build`")
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in _SIGS.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def last_error() -> str:
    return lib().bqrrp_last_error().decode()


def _check(fn, rc):
    if rc != 0:
        raise BqrrpError(fn, rc, last_error())
    return rc


# ----------------------------------------------------------------- torch helpers
def _torch():
    import torch
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def colmajor_empty(m, n, dtype=None, device="cuda"):
    torch = _torch()
    dtype = dtype or torch.float64
    return torch.empty((n, m), dtype=dtype, device=device).t()


def to_colmajor(x, device="cuda"):
    """Column-major float64 copy of a numpy array or tensor on ``device``."""
    torch = _torch()
    t = torch.as_tensor(x, dtype=torch.float64)
    out = colmajor_empty(t.shape[0], t.shape[1], device=device)
    out.copy_(t)
    return out


def _ld(t):
    if t.dim() != 2 or (t.stride(0) != 1 and t.shape[0] > 1):
        raise ValueError("expected a column-major 2-D tensor (stride(0) == 1)")
    return max(int(t.stride(1)), max(int(t.shape[0]), 1))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr() if t is not None else 0)


def make_opts(sketch_kind=SKETCH_DENSE, nnz=8, panel_kind=PANEL_CHOLQR, precision=PRECISION_FP64,
              schedule=SCHEDULE_OVERLAP, panel_tc=0):
    o = Opts()
    o.sketch_kind = sketch_kind
    o.sketch_nnz = nnz
    o.panel_kind = panel_kind
    o.precision = precision
    o.schedule = schedule
    o.panel_tc = panel_tc
    return o


def _workspace(nbytes, device):
    torch = _torch()
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


# ----------------------------------------------------------------- entry points
def bqrrp_workspace_query(m, n, b, d, opts=None):
    return int(lib().bqrrp_workspace_query(m, n, b, d, ctypes.byref(opts) if opts else None))


def bqrrp_factor(A, b, d, seed, jpvt, tau, opts=None, workspace=None, stream=None):
    """A (m x n column-major float64, in/out), jpvt (int64, n), tau (float64, n).
    Returns the rank.  Allocates the workspace with torch when none is given."""
    m, n = A.shape
    if workspace is None:
        workspace = _workspace(bqrrp_workspace_query(m, n, b, d, opts), A.device)
    rank = _i64(0)
    rc = lib().bqrrp_factor(m, n, _ptr(A), _ld(A), b, d, seed, _ptr(jpvt), _ptr(tau), ctypes.byref(rank),
                            ctypes.byref(opts) if opts else None, _ptr(workspace), workspace.numel(), _stream(stream))
    _check("bqrrp_factor", rc)
    return rank.value


def bqrrp_factor_status(A, b, d, seed, jpvt, tau, opts=None, workspace=None, workspace_bytes=None, stream=None):
    """Like bqrrp_factor but returns (status code, rank) instead of raising."""
    m, n = A.shape
    rank = _i64(0)
    nbytes = workspace.numel() if workspace is not None else 0
    if workspace_bytes is not None:
        nbytes = workspace_bytes
    rc = lib().bqrrp_factor(m, n, _ptr(A), _ld(A) if n > 0 else max(m, 1), b, d, seed, _ptr(jpvt), _ptr(tau),
                            ctypes.byref(rank), ctypes.byref(opts) if opts else None, _ptr(workspace), nbytes,
                            _stream(stream))
    return rc, rank.value


def bqrrp_workspace_query_host(m, n, b, d, opts=None):
    return int(lib().bqrrp_workspace_query_host(m, n, b, d, ctypes.byref(opts) if opts else None))


def bqrrp_factor_host(A_host, b, d, seed, jpvt_host, tau_host, workspace, opts=None, stream=None):
    """Host-buffer form: A_host (column-major host tensor, in/out), jpvt_host,
    tau_host host tensors; workspace a device uint8 tensor."""
    m, n = A_host.shape
    rank = _i64(0)
    rc = lib().bqrrp_factor_host(m, n, _ptr(A_host), _ld(A_host), b, d, seed, _ptr(jpvt_host), _ptr(tau_host),
                                 ctypes.byref(rank), ctypes.byref(opts) if opts else None, _ptr(workspace),
                                 workspace.numel(), _stream(stream))
    _check("bqrrp_factor_host", rc)
    return rank.value


def bqrrp_sketch_operator(d, m, seed, kind=SKETCH_DENSE, nnz=8, S=None, stream=None):
    if S is None:
        S = colmajor_empty(d, m)
    rc = lib().bqrrp_sketch_operator(d, m, seed, kind, nnz, _ptr(S), _ld(S), _stream(stream))
    _check("bqrrp_sketch_operator", rc)
    return S


def bqrrp_sketch_apply(A, d, seed, kind=SKETCH_DENSE, nnz=8, Msk=None, stream=None):
    m, n = A.shape
    if Msk is None:
        Msk = colmajor_empty(d, n, device=A.device)
    ws = _workspace(lib().bqrrp_sketch_apply_workspace(d, m, kind, nnz), A.device)
    rc = lib().bqrrp_sketch_apply(d, m, n, _ptr(A), _ld(A), seed, kind, nnz, _ptr(Msk), _ld(Msk), _ptr(ws), ws.numel(),
                                  _stream(stream))
    _check("bqrrp_sketch_apply", rc)
    return Msk


def bqrrp_sketch_apply_sparse_noalloc(A, d, seed, nnz=8, Msk=None, stream=None):
    """Sparse-sign Msk = S*A with the library's fixed scratch (no workspace,
    no allocation inside the call; Msk is allocated here when not given)."""
    m, n = A.shape
    if Msk is None:
        Msk = colmajor_empty(d, n, device=A.device)
    rc = lib().bqrrp_sketch_apply_sparse_noalloc(d, m, n, _ptr(A), _ld(A), seed, nnz, _ptr(Msk), _ld(Msk),
                                                 _stream(stream))
    _check("bqrrp_sketch_apply_sparse_noalloc", rc)
    return Msk


def bqrrp_qrcp_wide(Msk, stream=None):
    """Alg. 2 in place on the d x N sketch; returns (Jsk, ipiv) int64 tensors."""
    torch = _torch()
    d, N = Msk.shape
    Jsk = torch.empty(max(N, 1), dtype=torch.int64, device=Msk.device)
    ipiv = torch.empty(max(min(N, d), 1), dtype=torch.int64, device=Msk.device)
    ws = _workspace(lib().bqrrp_qrcp_wide_workspace(d, N), Msk.device)
    rc = lib().bqrrp_qrcp_wide(d, N, _ptr(Msk), _ld(Msk), _ptr(Jsk), _ptr(ipiv), _ptr(ws), ws.numel(),
                               _stream(stream))
    _check("bqrrp_qrcp_wide", rc)
    return Jsk[:N], ipiv[: min(N, d)]


def bqrrp_selftest_lu_wait_timeout(Msk, stream=None):
    """Failure-detection self-test of the LU pivot exchange (see include/bqrrp.h).
    Returns (status, ipiv of the normal second run)."""
    torch = _torch()
    d, N = Msk.shape
    ipiv = torch.empty(max(min(N, d), 1), dtype=torch.int64, device=Msk.device)
    ws = _workspace(lib().bqrrp_qrcp_wide_workspace(d, N), Msk.device)
    rc = lib().bqrrp_selftest_lu_wait_timeout(d, N, _ptr(Msk), _ld(Msk), _ptr(ipiv), _ptr(ws), ws.numel(),
                                              _stream(stream))
    return rc, ipiv[: min(N, d)]


def bqrrp_col_perm(M, J, max_moved=None, stream=None):
    m, N = M.shape
    mm = N if max_moved is None else max_moved
    ws = _workspace(lib().bqrrp_col_perm_workspace(m, N, mm), M.device)
    rc = lib().bqrrp_col_perm(m, N, _ptr(M), _ld(M), _ptr(J), mm, _ptr(ws), ws.numel(), _stream(stream))
    _check("bqrrp_col_perm", rc)
    return M


def bqrrp_cholqr_panel(M, Rsk, k, stream=None):
    """Alg. 3 in place on the rows x w panel M; returns (T, tau, k kept)."""
    torch = _torch()
    rows, w = M.shape
    T = colmajor_empty(max(k, 1), max(k, 1), device=M.device)
    tau = torch.zeros(max(k, 1), dtype=torch.float64, device=M.device)
    kout = _i64(0)
    ws = _workspace(lib().bqrrp_cholqr_panel_workspace(rows, w), M.device)
    rc = lib().bqrrp_cholqr_panel(rows, w, k, _ptr(M), _ld(M), _ptr(Rsk), _ld(Rsk), _ptr(T), _ld(T), _ptr(tau),
                                  ctypes.byref(kout), _ptr(ws), ws.numel(), _stream(stream))
    _check("bqrrp_cholqr_panel", rc)
    kk = kout.value
    return T[:kk, :kk], tau[:kk], kk


def bqrrp_geqrf(A, nb=0, tau=None, workspace=None, stream=None):
    torch = _torch()
    m, n = A.shape
    if tau is None:
        tau = torch.zeros(max(min(m, n), 1), dtype=torch.float64, device=A.device)
    if workspace is None:
        workspace = _workspace(lib().bqrrp_geqrf_workspace(m, n, nb), A.device)
    rc = lib().bqrrp_geqrf(m, n, _ptr(A), _ld(A), _ptr(tau), nb, _ptr(workspace), workspace.numel(), _stream(stream))
    _check("bqrrp_geqrf", rc)
    return tau


def bqrrp_geqrf_workspace(m, n, nb=0):
    return int(lib().bqrrp_geqrf_workspace(m, n, nb))


def bqrrp_geqrf_mixed_workspace(m, n):
    return int(lib().bqrrp_geqrf_mixed_workspace(m, n))


def bqrrp_geqrf_mixed(A, tau=None, workspace=None, stream=None):
    """Own unpivoted QR with tensor-core (exact-slice) trailing updates."""
    torch = _torch()
    m, n = A.shape
    if tau is None:
        tau = torch.zeros(max(min(m, n), 1), dtype=torch.float64, device=A.device)
    if workspace is None:
        workspace = _workspace(lib().bqrrp_geqrf_mixed_workspace(m, n), A.device)
    rc = lib().bqrrp_geqrf_mixed(m, n, _ptr(A), _ld(A), _ptr(tau), _ptr(workspace), workspace.numel(),
                                 _stream(stream))
    _check("bqrrp_geqrf_mixed", rc)
    return tau


def bqrrp_dgemm(transa, transb, alpha, A, B, beta, C, workspace=None, stream=None):
    M, N = C.shape
    K = A.shape[0] if transa.upper() == "T" else A.shape[1]
    if workspace is None:
        workspace = _workspace(lib().bqrrp_dgemm_workspace(M, N, K), C.device)
    rc = lib().bqrrp_dgemm(transa.encode(), transb.encode(), M, N, K, alpha, _ptr(A), _ld(A), _ptr(B), _ld(B), beta,
                           _ptr(C), _ld(C), _ptr(workspace), workspace.numel(), _stream(stream))
    _check("bqrrp_dgemm", rc)
    return C


def bqrrp_dgemm_ozaki(transa, transb, alpha, A, B, beta, C, stream=None):
    """C = alpha op(A) op(B) + beta C formed from exact bf16 slices on the tensor cores."""
    M, N = C.shape
    K = A.shape[0] if transa.upper() == "T" else A.shape[1]
    ws = _workspace(lib().bqrrp_dgemm_ozaki_workspace(M, N, K), C.device)
    rc = lib().bqrrp_dgemm_ozaki(transa.encode(), transb.encode(), M, N, K, alpha, _ptr(A), _ld(A), _ptr(B), _ld(B),
                                 beta, _ptr(C), _ld(C), _ptr(ws), ws.numel(), _stream(stream))
    _check("bqrrp_dgemm_ozaki", rc)
    return C


def bqrrp_sketch_apply_tc(A, d, seed, Msk=None, stream=None):
    """Dense +-1 sketch S*A on the bf16 tensor cores (exact slices)."""
    m, n = A.shape
    if Msk is None:
        Msk = colmajor_empty(d, n, device=A.device)
    ws = _workspace(lib().bqrrp_sketch_apply_tc_workspace(d, m, n), A.device)
    rc = lib().bqrrp_sketch_apply_tc(d, m, n, _ptr(A), _ld(A), seed, _ptr(Msk), _ld(Msk), _ptr(ws), ws.numel(),
                                     _stream(stream))
    _check("bqrrp_sketch_apply_tc", rc)
    return Msk


def bqrrp_dgemm_workspace(M, N, K):
    return int(lib().bqrrp_dgemm_workspace(M, N, K))


def bqrrp_probe_fp64_peak(iters=2000, stream=None):
    return float(lib().bqrrp_probe_fp64_peak(iters, _stream(stream)))


def bqrrp_profile_enable(on=True):
    lib().bqrrp_profile_enable(1 if on else 0)


def bqrrp_profile_reset():
    lib().bqrrp_profile_reset()


def bqrrp_profile_read():
    """dict phase -> (ms, flops) plus 'calls'."""
    p = Profile()
    lib().bqrrp_profile_read(ctypes.byref(p))
    out = {name: (p.ms[i], p.flops[i]) for i, name in enumerate(PHASES)}
    out["calls"] = p.calls
    return out


def bqrrp_launch_counter():
    return int(lib().bqrrp_launch_counter())


# ----------------------------------------------------------------- convenience
def factor(A, b, d, seed, sketch="dense", nnz=8, panel="cholqr", precision="fp64", schedule="overlap",
           panel_tc=False, stream=None):
    """Factor a copy of A (any 2-D float64 tensor/array); returns
    (F column-major with R and reflectors, jpvt, tau, rank) as device tensors.
    precision: "fp64", "mixed" or "mixed_sketch32"; panel_tc (mixed only):
    the CholQR panel's Gram and tall-solve updates as slice products."""
    torch = _torch()
    F = to_colmajor(A)
    m, n = F.shape
    jpvt = torch.empty(max(n, 1), dtype=torch.int64, device=F.device)
    tau = torch.empty(max(n, 1), dtype=torch.float64, device=F.device)
    opts = make_opts(SKETCH_DENSE if sketch == "dense" else SKETCH_SPARSE, nnz,
                     PANEL_CHOLQR if panel == "cholqr" else PANEL_HQR,
                     _PRECISIONS[precision],
                     SCHEDULE_OVERLAP if schedule == "overlap" else SCHEDULE_SERIAL, 1 if panel_tc else 0)
    rank = bqrrp_factor(F, b, d, seed, jpvt, tau, opts=opts, stream=stream)
    return F, jpvt[:n], tau[:n], rank


# ----------------------------------------------------------------- batched BQRRP
def _host_i64(x):
    import numpy as np
    return np.ascontiguousarray(np.asarray(x, dtype=np.int64))


def _host_u64(x):
    import numpy as np
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint64))


def _np_ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


class BatchPlan:
    """Owner of a ``bqrrp_batch_plan`` handle (host arrays m, n, b, d, seed;
    the packed layout of ``workloads.batch_offsets``).  tiles: optional host
    array of trailing tile widths (32 or 64) per matrix."""

    def __init__(self, m, n, b, d, seeds, trunc_tol=1e-8, tiles=None):
        self.m, self.n, self.b, self.d = _host_i64(m), _host_i64(n), _host_i64(b), _host_i64(d)
        self.seeds = _host_u64(seeds)
        self.batch = len(self.m)
        self.trunc_tol = float(trunc_tol)
        h = _vp()
        if tiles is None:
            rc = lib().bqrrp_batch_plan_create(ctypes.byref(h), self.batch, _np_ptr(self.m), _np_ptr(self.n),
                                               _np_ptr(self.b), _np_ptr(self.d), _np_ptr(self.seeds), self.trunc_tol)
            _check("bqrrp_batch_plan_create", rc)
        else:
            self.tiles = _host_i64(tiles)
            rc = lib().bqrrp_batch_plan_create_tiles(ctypes.byref(h), self.batch, _np_ptr(self.m), _np_ptr(self.n),
                                                     _np_ptr(self.b), _np_ptr(self.d), _np_ptr(self.tiles),
                                                     _np_ptr(self.seeds), self.trunc_tol)
            _check("bqrrp_batch_plan_create_tiles", rc)
        self.handle = h
        self.workspace = None

    def workspace_bytes(self):
        return int(lib().bqrrp_batch_workspace_bytes(self.handle))

    def launches(self):
        return int(lib().bqrrp_batch_launches(self.handle))

    def set_form(self, form):
        """BATCH_PERSISTENT (default) or BATCH_LOCKSTEP launch form."""
        _check("bqrrp_batch_plan_set_form", lib().bqrrp_batch_plan_set_form(self.handle, int(form)))

    def flops(self, phase=-1):
        return float(lib().bqrrp_batch_flops(self.handle, int(phase)))

    def factor(self, A, jpvt, tau, rank, trunc_rank=None, info=None, workspace=None, use_graph=False, stream=None):
        """A: packed float64 (in/out); jpvt int64, tau float64 (sum n); rank,
        trunc_rank int64 and info int32 (one per matrix).  Device tensors."""
        if workspace is None:
            if self.workspace is None:
                self.workspace = _workspace(self.workspace_bytes(), A.device)
            workspace = self.workspace
        rc = lib().bqrrp_batch_factor(self.handle, _ptr(A), _ptr(jpvt), _ptr(tau), _ptr(rank), _ptr(trunc_rank),
                                      _ptr(info), _ptr(workspace), workspace.numel(), _stream(stream),
                                      1 if use_graph else 0)
        _check("bqrrp_batch_factor", rc)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().bqrrp_batch_plan_destroy(self.handle)
            self.handle = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bqrrp_batch_autotune(m, n, seeds, A, trunc_tol=1e-8, stream=None):
    """Pick b and d per matrix by timing on the device (A packed, read only).
    Returns (b, d, best_ms) with b, d numpy int64 arrays."""
    import numpy as np
    m, n, sd = _host_i64(m), _host_i64(n), _host_u64(seeds)
    batch = len(m)
    nbytes = int(lib().bqrrp_batch_autotune_workspace_bytes(batch, _np_ptr(m), _np_ptr(n)))
    ws = _workspace(nbytes, A.device)
    b = np.zeros(batch, dtype=np.int64)
    d = np.zeros(batch, dtype=np.int64)
    best = _d(0.0)
    rc = lib().bqrrp_batch_autotune(batch, _np_ptr(m), _np_ptr(n), _np_ptr(sd), _ptr(A), float(trunc_tol), _ptr(ws),
                                    ws.numel(), _stream(stream), _np_ptr(b), _np_ptr(d), ctypes.byref(best))
    _check("bqrrp_batch_autotune", rc)
    del ws
    return b, d, best.value


def bqrrp_batch_autotune_tiles(m, n, seeds, A, trunc_tol=1e-8, stream=None):
    """Pick b, d and the trailing tile width per matrix by timing on the device
    (A packed, read only).  Returns (b, d, tiles, best_ms), numpy int64 arrays."""
    import numpy as np
    m, n, sd = _host_i64(m), _host_i64(n), _host_u64(seeds)
    batch = len(m)
    nbytes = int(lib().bqrrp_batch_autotune_workspace_bytes(batch, _np_ptr(m), _np_ptr(n)))
    ws = _workspace(nbytes, A.device)
    b = np.zeros(batch, dtype=np.int64)
    d = np.zeros(batch, dtype=np.int64)
    t = np.zeros(batch, dtype=np.int64)
    best = _d(0.0)
    rc = lib().bqrrp_batch_autotune_tiles(batch, _np_ptr(m), _np_ptr(n), _np_ptr(sd), _ptr(A), float(trunc_tol),
                                          _ptr(ws), ws.numel(), _stream(stream), _np_ptr(b), _np_ptr(d), _np_ptr(t),
                                          ctypes.byref(best))
    _check("bqrrp_batch_autotune_tiles", rc)
    del ws
    return b, d, t, best.value


def factor_batched(A_packed, m, n, b, d, seeds, trunc_tol=1e-8, use_graph=False, stream=None,
                   form=BATCH_PERSISTENT, tiles=None):
    """Factor a copy of a packed batch.  Returns (F packed, jpvt, tau, rank,
    trunc_rank, info) as device tensors."""
    torch = _torch()
    import numpy as np
    F = torch.as_tensor(A_packed, dtype=torch.float64).to("cuda").clone()
    tot_j = int(np.sum(np.asarray(n, dtype=np.int64)))
    nb = len(m)
    jpvt = torch.empty(max(tot_j, 1), dtype=torch.int64, device=F.device)
    tau = torch.empty(max(tot_j, 1), dtype=torch.float64, device=F.device)
    rank = torch.empty(max(nb, 1), dtype=torch.int64, device=F.device)
    trunc = torch.empty(max(nb, 1), dtype=torch.int64, device=F.device)
    info = torch.empty(max(nb, 1), dtype=torch.int32, device=F.device)
    plan = BatchPlan(m, n, b, d, seeds, trunc_tol, tiles=tiles)
    try:
        plan.set_form(form)
        plan.factor(F, jpvt, tau, rank, trunc, info, use_graph=use_graph, stream=stream)
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
    finally:
        plan.close()
    return F, jpvt, tau, rank[:nb], trunc[:nb], info[:nb]


# ----------------------------------------------------------------- request loop
def _host_ptr(x):
    """Address of a host buffer (numpy array or CPU torch tensor), or None."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(x.ctypes.data)


class Server:
    """Owner of a ``bqrrp_server``.  Host buffers handed to ``submit`` are kept
    alive here until their completion has been polled."""

    def __init__(self, hbm_budget_bytes, workspace_bytes, trunc_tol=1e-8, small_max_elems=1 << 20, dry=False,
                 dry_gflops=1000.0, mixed=False):
        h = _vp()
        flags = (SERVER_DRYRUN if dry else 0) | (SERVER_MIXED if mixed else 0)
        rc = lib().bqrrp_server_create(ctypes.byref(h), int(hbm_budget_bytes), int(workspace_bytes),
                                       float(trunc_tol), int(small_max_elems), flags, float(dry_gflops))
        _check("bqrrp_server_create", rc)
        self.handle = h
        self._keep = {}

    def submit(self, rid, m, n, b, d, seed, A_host=None, A_out=None, jpvt_out=None, tau_out=None):
        r = Request()
        r.id, r.m, r.n, r.b, r.d, r.seed = int(rid), int(m), int(n), int(b), int(d), int(seed)
        r.A_host, r.A_out_host = _host_ptr(A_host), _host_ptr(A_out)
        r.jpvt_out_host, r.tau_out_host = _host_ptr(jpvt_out), _host_ptr(tau_out)
        self._keep[int(rid)] = (A_host, A_out, jpvt_out, tau_out)
        rc = lib().bqrrp_server_submit(self.handle, ctypes.byref(r))
        if rc != 0:
            self._keep.pop(int(rid), None)
        _check("bqrrp_server_submit", rc)

    def poll(self, max_out=256, wait_s=0.0):
        buf = (Completion * max_out)()
        k = lib().bqrrp_server_poll(self.handle, buf, max_out, float(wait_s))
        out = []
        for i in range(k):
            c = buf[i]
            self._keep.pop(int(c.id), None)
            out.append({f: getattr(c, f) for f, _ in Completion._fields_})
        return out

    def drain(self):
        _check("bqrrp_server_drain", lib().bqrrp_server_drain(self.handle))

    def clock(self):
        return float(lib().bqrrp_server_clock(self.handle))

    def last_error(self):
        return lib().bqrrp_server_last_error(self.handle).decode()

    def stats(self):
        st = ServerStats()
        _check("bqrrp_server_get_stats", lib().bqrrp_server_get_stats(self.handle, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().bqrrp_server_destroy(self.handle)
            self.handle = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
