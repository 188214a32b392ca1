"""End-to-end GPU parity of bqrrp_factor (C ABI) against the CPU oracle.

Bar (from the method's specification): pivot vectors identical where every
LU pivot step of the oracle is gapped (relative top-2 margin > 1e-6, far above
the 1e-13-level differences two FP64 summation orders produce); ranks equal;
||AP - QR||_F / ||A||_F <= 1e-12; ||Q^T Q - I||_F <= 1e-12; the rank-s
truncation error ||R(s:, s:)||_F at every block boundary s within 1.1x of the
oracle's; R itself within 1e-10 * ||A||_F of the oracle's (R is unique up to
row signs, and both sides use the same sign rule); tau_j within
100 sqrt(m) u ||A||_F / |R_jj| (a reflector is only as well determined as the
trailing block it annihilates).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2507_00976_b300 as bq
from checks import metrics, trailing_norms, upper_r
from gpu_util import np_
from paper_2507_00976_b300 import binding as B
from paper_2507_00976_b300 import workloads as W

pytestmark = pytest.mark.gpu


def run_gpu(A, b, d, seed, sketch="dense", panel="cholqr"):
    F, jpvt, tau, rank = bq.factor(A, b, d, seed, sketch=sketch, panel=panel)
    torch.cuda.synchronize()
    return np_(F), np_(jpvt), np_(tau), rank


def compare(A, b, d, seed, sketch="dense", panel="cholqr", expect_rank=None):
    kind = 0 if sketch == "dense" else 1
    fo = oracle.bqrrp(A, b, d, seed, sketch_kind=kind, panel=panel)
    F, jpvt, tau, rank = run_gpu(A, b, d, seed, sketch, panel)
    assert rank == fo.rank
    if expect_rank is not None:
        assert rank == expect_rank
    gapped = all(t["margin"] > 1e-6 for t in fo.trace)
    if gapped:
        # beyond the numerical rank the sketch is rounding noise, so only the
        # first `rank` pivots are determined by the input
        assert np.array_equal(jpvt[:rank], fo.jpvt[:rank])
        assert set(jpvt[rank:]) == set(fo.jpvt[rank:])
    res, orth, ok = metrics(A, F, jpvt, tau, rank)
    assert ok and res <= 1e-12 and orth <= 1e-12, (res, orth)
    n = A.shape[1]
    bounds = list(range(0, n, b))
    tg = trailing_norms(F, rank, bounds)
    to = trailing_norms(fo.A, fo.rank, bounds)
    nrm = np.linalg.norm(A)
    assert np.all(tg <= 1.1 * to + 1e-13 * nrm)
    if gapped and rank == n:
        R = upper_r(F, rank)[:n]
        Ro = upper_r(fo.A, fo.rank)[:n]
        assert np.linalg.norm(R - Ro) <= 1e-10 * nrm
        # tau_j is fixed only up to the conditioning of the trailing block it
        # comes from: relative error ~ u ||A||_F / |R_jj| (times a sqrt(m) factor)
        m = A.shape[0]
        rjj = np.abs(np.diag(Ro)[:rank])
        bound = 100 * np.sqrt(m) * 2.0 ** -53 * nrm / np.maximum(rjj, 1e-300)
        assert np.all(np.abs(tau[:rank] - fo.tau[:rank]) <= np.minimum(bound, 1.0) + 1e-14)
    return F, jpvt, tau, rank, fo


def test_c1_parity():
    """2000 x 1000, sigma_k = 10^(-10(k-1)/999), b = 128, d = 160, Philox seed 1."""
    A = W.c1_matrix()
    compare(A, 128, 160, 1, expect_rank=1000)


@pytest.mark.parametrize("m,n,b,d", [(777, 500, 64, 80), (300, 300, 300, 375), (1000, 100, 128, 160),
                                     (513, 257, 32, 40), (4100, 130, 64, 80), (65, 65, 8, 10),
                                     # degenerate blocks: b = 1 (d = 1 and d > b), 1 x 1, one column, d = b
                                     (40, 17, 1, 1), (40, 17, 1, 3), (1, 1, 1, 1), (50, 1, 4, 5), (30, 30, 7, 7)])
def test_shapes_with_ragged_tails(m, n, b, d):
    A = W.gaussian(m, n, m * 3 + n)
    compare(A, b, d, 5, expect_rank=n)


def test_exact_low_rank():
    A = W.low_rank(1000, 600, 150, 4)
    compare(A, 64, 80, 2, expect_rank=150)


def test_low_rank_at_block_boundary():
    A = W.low_rank(700, 400, 128, 8)
    compare(A, 64, 80, 2, expect_rank=128)


def test_sparse_sketch_at_the_largest_configured_block():
    """b = 2048, d = ceil(1.25 b) = 2560 with the sparse sketch (the largest
    block of the configuration's sweep): the sketch rows exceed one CTA's row
    tile.  Held to the properties that hold at any size."""
    import torch
    from checks import metrics
    m, n = 3000, 2600
    A = W.gaussian(m, n, 21)
    F, jpvt, tau, rank = bq.factor(A, 2048, 2560, 4, sketch="sparse")
    torch.cuda.synchronize()
    assert rank == n
    res, orth, perm_ok = metrics(A, F.cpu().numpy(), jpvt.cpu().numpy(), tau.cpu().numpy(), rank)
    assert perm_ok and res <= 1e-12 and orth <= 1e-12, (res, orth)


def test_sparse_sign_sketch():
    A = W.c1_matrix()
    compare(A, 128, 160, 1, sketch="sparse")


def test_householder_panel_variant():
    A = W.gaussian(900, 700, 12)
    compare(A, 96, 120, 3, panel="hqr", expect_rank=700)


def test_kahan_matrix_valid_factorization():
    A = W.kahan(512)
    F, jpvt, tau, rank = run_gpu(A, 64, 80, 3)
    res, orth, ok = metrics(A, F, jpvt, tau, rank)
    assert ok and res <= 1e-12 and orth <= 1e-12


def test_zero_matrix():
    F, jpvt, tau, rank = run_gpu(np.zeros((300, 200)), 32, 40, 1)
    assert rank == 0 and np.all(tau == 0) and sorted(jpvt) == list(range(1, 201))


def test_deterministic_and_host_entry_point_identical():
    A = W.gaussian(1500, 900, 21)
    F1, j1, t1, r1 = run_gpu(A, 100, 125, 9)
    F2, j2, t2, r2 = run_gpu(A, 100, 125, 9)
    assert np.array_equal(F1, F2) and np.array_equal(j1, j2) and np.array_equal(t1, t2) and r1 == r2
    m, n = A.shape
    Ah = torch.empty((n, m), dtype=torch.float64).pin_memory().t()
    Ah.copy_(torch.as_tensor(A))
    jh = torch.empty(n, dtype=torch.int64).pin_memory()
    th = torch.empty(n, dtype=torch.float64).pin_memory()
    ws = torch.empty(B.bqrrp_workspace_query_host(m, n, 100, 125), dtype=torch.uint8, device="cuda")
    r3 = B.bqrrp_factor_host(Ah, 100, 125, 9, jh, th, ws)
    assert r3 == r1
    assert np.array_equal(Ah.numpy(), F1) and np.array_equal(jh.numpy(), j1) and np.array_equal(th.numpy(), t1)


@pytest.mark.parametrize("case", [
    ("gaussian", 1500, 900, 100, 125),      # ragged last block
    ("low_rank", 1100, 700, 96, 120),       # stops inside the third block
    ("low_rank", 1024, 1024, 128, 160),     # rank 256: stops at a block boundary
    ("sparse", 900, 800, 64, 80),           # sparse-sign sketch
    ("gaussian", 3000, 500, 64, 80),        # tall
    ("gaussian", 2000, 1500, 600, 700),     # d > 640: R^sk by the blocked Householder QR
])
def test_overlap_schedule_identical_to_serial(case):
    """The overlap schedule (sketch update and the next block's Alg. 2 on a
    side stream during the trailing update) gives the serial schedule's
    results bit for bit, with the phase profiler off and on."""
    kind, m, n, b, d = case
    if kind == "low_rank":
        A = W.low_rank(m, n, 250 if n == 700 else 256, 8)
    else:
        A = W.gaussian(m, n, 9)
    sketch = "sparse" if kind == "sparse" else "dense"
    ref = [np_(x) if torch.is_tensor(x) else x for x in bq.factor(A, b, d, 5, sketch=sketch, schedule="serial")]
    for prof in (False, True):
        B.bqrrp_profile_enable(prof)
        try:
            got = [np_(x) if torch.is_tensor(x) else x for x in bq.factor(A, b, d, 5, sketch=sketch)]
        finally:
            B.bqrrp_profile_enable(False)
        torch.cuda.synchronize()
        assert got[3] == ref[3]
        for x, y in zip(got[:3], ref[:3]):
            assert np.array_equal(x, y)
    if kind == "low_rank":
        assert ref[3] < n


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("rank_deficient", [False, True])
def test_host_entry_point_padded_ld(pinned, rank_deficient):
    """Host buffers with ld > m, pinned (A copied in by column halves, each
    sketched once it has arrived, and column blocks copied back while later
    blocks are factored) and pageable (one copy each way), full rank and with
    an early stop; the results equal the device entry point's bit for bit and
    the padding rows are left alone."""
    m, n, b, d = 1300, 1100, 96, 120
    A = W.low_rank(m, n, 250, 4) if rank_deficient else W.gaussian(m, n, 5)
    F1, j1, t1, r1 = run_gpu(A, b, d, 17)
    ld = m + 13
    buf = torch.full((n, ld), -7.0, dtype=torch.float64)
    if pinned:
        buf = buf.pin_memory()
    Ah = buf.t()[:m]
    Ah.copy_(torch.as_tensor(A))
    jh = torch.empty(n, dtype=torch.int64)
    th = torch.empty(n, dtype=torch.float64)
    if pinned:
        jh, th = jh.pin_memory(), th.pin_memory()
    ws = torch.empty(B.bqrrp_workspace_query_host(m, n, b, d), dtype=torch.uint8, device="cuda")
    r2 = B.bqrrp_factor_host(Ah, b, d, 17, jh, th, ws)
    assert r2 == r1 and (r1 < n) == rank_deficient
    assert np.array_equal(Ah.numpy(), F1) and np.array_equal(jh.numpy(), j1) and np.array_equal(th.numpy(), t1)
    assert torch.all(buf[:, m:] == -7.0)


@pytest.mark.parametrize("precision,sketch", [("fp64", "sparse"), ("mixed", "dense")])
def test_host_entry_point_other_forms(precision, sketch):
    """Pinned host buffers with the sparse sketch and with the mixed form (A
    copied in whole before the sketch): the device entry point's results bit
    for bit."""
    m, n, b, d = 1200, 1100, 96, 120
    A = W.gaussian(m, n, 6)
    F1, j1, t1, r1 = [np_(x) if torch.is_tensor(x) else x
                      for x in bq.factor(A, b, d, 7, sketch=sketch, precision=precision)]
    Ah = torch.empty((n, m), dtype=torch.float64).pin_memory().t()
    Ah.copy_(torch.as_tensor(A))
    jh = torch.empty(n, dtype=torch.int64).pin_memory()
    th = torch.empty(n, dtype=torch.float64).pin_memory()
    opts = B.make_opts(B.SKETCH_DENSE if sketch == "dense" else B.SKETCH_SPARSE, 8, B.PANEL_CHOLQR,
                       B.PRECISION_FP64 if precision == "fp64" else B.PRECISION_MIXED)
    ws = torch.empty(B.bqrrp_workspace_query_host(m, n, b, d, opts), dtype=torch.uint8, device="cuda")
    assert B.bqrrp_factor_host(Ah, b, d, 7, jh, th, ws, opts=opts) == r1
    assert np.array_equal(Ah.numpy(), F1) and np.array_equal(jh.numpy(), j1) and np.array_equal(th.numpy(), t1)


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("col", [5, 1000])     # in the first or the second half of the columns
def test_host_entry_point_nan_leaves_host_buffer_unchanged(pinned, col):
    m, n = 1400, 1200
    A = W.gaussian(m, n, 3)
    A[11, col] = np.nan
    buf = torch.empty((n, m), dtype=torch.float64)
    if pinned:
        buf = buf.pin_memory()
    Ah = buf.t()
    Ah.copy_(torch.as_tensor(A))
    before = Ah.clone()
    jh = torch.empty(n, dtype=torch.int64)
    th = torch.empty(n, dtype=torch.float64)
    ws = torch.empty(B.bqrrp_workspace_query_host(m, n, 64, 80), dtype=torch.uint8, device="cuda")
    with pytest.raises(B.BqrrpError) as e:
        B.bqrrp_factor_host(Ah, 64, 80, 1, jh, th, ws)
    assert e.value.code == B.ENUMERIC
    assert torch.equal(torch.isnan(Ah), torch.isnan(before))
    assert torch.equal(torch.nan_to_num(Ah), torch.nan_to_num(before))
    # the same workspace then factors a finite matrix correctly
    A[11, col] = 0.5
    Ah.copy_(torch.as_tensor(A))
    F1, j1, t1, r1 = run_gpu(A, 64, 80, 1)
    assert B.bqrrp_factor_host(Ah, 64, 80, 1, jh, th, ws) == r1
    assert np.array_equal(Ah.numpy(), F1) and np.array_equal(jh.numpy(), j1)


def test_error_codes():
    A = bq.to_colmajor(W.gaussian(40, 30, 1))
    jp = torch.empty(30, dtype=torch.int64, device="cuda")
    tau = torch.empty(30, dtype=torch.float64, device="cuda")
    need = B.bqrrp_workspace_query(40, 30, 8, 10)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    rc, _ = B.bqrrp_factor_status(A, 8, 10, 1, jp, tau, workspace=ws, workspace_bytes=need - 4096)
    assert rc == B.ENOMEM
    A2 = A.clone()
    A2[5, 5] = float("nan")
    before = A2.clone()
    rc, rank = B.bqrrp_factor_status(A2, 8, 10, 1, jp, tau, workspace=ws)
    assert rc == B.ENUMERIC and rank == -1
    assert torch.equal(torch.isnan(A2), torch.isnan(before))
    wide = bq.to_colmajor(W.gaussian(20, 30, 1))
    rc, _ = B.bqrrp_factor_status(wide, 8, 10, 1, jp, tau, workspace=ws)
    assert rc == -1
