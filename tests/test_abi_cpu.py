"""Host-side checks of the C ABI (no GPU needed): the library builds and
loads, exports every function include/bqrrp.h declares, sizes workspaces and
rejects invalid arguments before touching the device."""
import ctypes

import pytest

from paper_2507_00976_b300 import binding as B


def test_library_exports_every_declared_symbol():
    L = B.lib()
    declared = B.header_symbols()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(L, name), name
        assert name in B._SIGS, f"binding has no signature for {name}"


def test_workspace_queries_are_consistent():
    small = B.bqrrp_workspace_query(2000, 1000, 128, 160)
    big = B.bqrrp_workspace_query(32768, 32768, 1024, 1280)
    assert 0 < small < big
    # dominant terms: 2 d n + 2 b n + m b + max(m, d) min(n, 2d) doubles, the
    # split-K partials (2048 n doubles), the bf16 slice planes of the dense
    # sketch (7 planes of min(n, 8192) columns of A, one plane of S), plus
    # fixed scratch
    m, n, b, d = 32768, 32768, 1024, 1280
    est = 8 * (2 * d * n + m * b + 2 * b * n + max(m, d) * min(n, 2 * d) + 2048 * n)
    est += 2 * 7 * m * min(n, 8192) + 2 * d * m
    assert est <= big <= est + 256 * 2**20
    assert B.bqrrp_workspace_query(100, 200, 10, 12) == 0          # m < n
    assert B.bqrrp_workspace_query(100, 50, 0, 12) == 0            # b < 1
    assert B.bqrrp_workspace_query(100, 50, 10, 9) == 0            # d < b
    sparse = B.make_opts(B.SKETCH_SPARSE, 8)
    # the sparse sketch's index lists (24 bytes per operator entry) take less
    # room than the dense sketch's slice planes (14 bytes per element of A)
    # (planes padded: k to 32, columns of A to 32, rows of S to 64)
    dense_planes = 2 * 7 * 2016 * 1024 + 2 * 192 * 2016
    sparse_lists = 24 * 2000 * 8
    sp = B.bqrrp_workspace_query(2000, 1000, 128, 160, sparse)
    assert abs(sp - (small - dense_planes + sparse_lists)) <= 2**20
    host = B.bqrrp_workspace_query_host(2000, 1000, 128, 160)
    assert host >= small + 2000 * 1000 * 8


def _factor_rc(m, n, b, d, lda=None, opts=None, ws_bytes=0):
    rank = ctypes.c_int64(7)
    rc = B.lib().bqrrp_factor(m, n, None, lda if lda is not None else max(m, 1), b, d, 1, None, None,
                              ctypes.byref(rank), ctypes.byref(opts) if opts else None, None, ws_bytes, None)
    return rc, rank.value


def test_argument_errors_follow_info_convention():
    assert _factor_rc(10, 20, 4, 5)[0] == -1
    assert _factor_rc(10, 8, 4, 5, lda=5)[0] == -4
    assert _factor_rc(10, 8, 0, 5)[0] == -5
    assert _factor_rc(10, 8, 4, 3)[0] == -6
    bad = B.make_opts(7, 8)
    assert _factor_rc(10, 8, 4, 5, opts=bad)[0] == -11
    assert _factor_rc(10, 8, 4, 5, opts=B.make_opts(schedule=2))[0] == -11
    bad = B.make_opts()
    bad.reserved[1] = 1
    assert _factor_rc(10, 8, 4, 5, opts=bad)[0] == -11
    # the tensor-core panel only with a mixed precision, and only 0 or 1
    assert _factor_rc(10, 8, 4, 5, opts=B.make_opts(panel_tc=1))[0] == -11
    assert _factor_rc(10, 8, 4, 5, opts=B.make_opts(precision=B.PRECISION_MIXED, panel_tc=2))[0] == -11
    assert _factor_rc(10, 8, 4, 5, opts=B.make_opts(precision=B.PRECISION_MIXED, panel_tc=1))[0] == -3
    assert _factor_rc(10, 8, 4, 5, opts=B.make_opts(schedule=B.SCHEDULE_SERIAL))[0] == -3   # valid opts, A NULL
    assert _factor_rc(10, 8, 4, 5)[0] == -3                         # A is NULL
    rc, rank = _factor_rc(10, 0, 4, 5)
    assert rc == 0 and rank == 0                                     # empty: nothing to do
    assert "d < b" in (_factor_rc(10, 8, 4, 3) and B.last_error())
    L = B.lib()
    assert L.bqrrp_sketch_operator(-1, 4, 0, 0, 8, None, 1, None) == -1
    assert L.bqrrp_sketch_operator(4, 4, 0, 3, 8, None, 4, None) == -4
    assert L.bqrrp_sketch_operator(4, 4, 0, 1, 9, None, 4, None) == -5
    assert L.bqrrp_dgemm(b"X", b"N", 1, 1, 1, 1.0, None, 1, None, 1, 0.0, None, 1, None, 0, None) == -1
    assert L.bqrrp_geqrf(4, 4, None, 2, None, 0, None, 0, None) == -4


def test_batched_plan_rejects_bad_shapes_before_touching_a_device():
    """bqrrp_batch_plan_create validates every matrix on the host first."""
    import numpy as np
    one = np.array([1], dtype=np.int64)
    cases = [((5, 8, 4, 5), -3), ((50, 8, 200, 250), -5), ((50, 8, 16, 8), -6),
             ((9000, 5000, 16, 20), B.EUNSUPPORTED)]
    for (m, n, b, d), code in cases:
        with pytest.raises(B.BqrrpError) as e:
            B.BatchPlan(np.array([m]), np.array([n]), np.array([b]), np.array([d]), one)
        assert e.value.code == code
