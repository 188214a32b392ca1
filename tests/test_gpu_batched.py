"""GPU parity of the batched BQRRP entry points against the per-matrix oracle.

Every matrix of a batch is held to the single-matrix bar:
- rank equal to the oracle's;
- pivots identical where the oracle's LU margins are gapped (> 1e-6);
- ||AP - QR||_F / ||A||_F <= 1e-12 and ||Q^T Q - I||_F <= 1e-12;
- block-boundary truncation errors within 1.1x of the oracle's;
- the truncation rank equal to the oracle's, unless the oracle's own tail
  norm lies within 1e-9 (relative) of the threshold there, where two summation
  orders may legitimately decide differently.

The batch adds no arithmetic, so a matrix's result must not depend on its
batch: that is checked bit for bit, as is graph replay against eager launches.
"""
import numpy as np
import pytest
import torch

import oracle
from checks import metrics, trailing_norms
from gpu_util import np_
from paper_2507_00976_b300 import binding as B
from paper_2507_00976_b300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-8


def pack(mats):
    return np.concatenate([np.asarray(A, dtype=np.float64).ravel(order="F") for A in mats]) \
        if mats else np.zeros(1)


def unpack(F, jpvt, tau, m, n):
    offA, offJ, _, _ = W.batch_offsets(m, n)
    out = []
    for i in range(len(m)):
        mi, ni = int(m[i]), int(n[i])
        Fi = F[offA[i]:offA[i] + mi * ni].reshape((mi, ni), order="F")
        out.append((Fi, jpvt[offJ[i]:offJ[i] + ni], tau[offJ[i]:offJ[i] + ni]))
    return out


def run_batch(mats, b, d, seeds, use_graph=False, tol=TOL, form=B.BATCH_PERSISTENT, tiles=None):
    m = np.array([A.shape[0] for A in mats], dtype=np.int64)
    n = np.array([A.shape[1] for A in mats], dtype=np.int64)
    F, jpvt, tau, rank, trunc, info = B.factor_batched(pack(mats), m, n, b, d, seeds, tol, use_graph=use_graph,
                                                       form=form, tiles=tiles)
    return m, n, np_(F), np_(jpvt), np_(tau), np_(rank), np_(trunc), np_(info)


def trunc_margin_ok(Fo, rank, anorm, tol, got):
    """The oracle's cut is decided by a single comparison; accept another cut
    only if the tail norm at the boundary is within 1e-9 of the threshold."""
    want = oracle.trunc_rank(Fo, rank, anorm, tol)
    if got == want:
        return True
    R = np.triu(Fo)[:rank]
    i = min(got, want)
    tail = np.linalg.norm(R[i:, i:])
    return abs(tail - tol * anorm) <= 1e-9 * tol * anorm


def check_against_oracle(mats, b, d, seeds, res):
    m, n, F, jpvt, tau, rank, trunc, info = res
    parts = unpack(F, jpvt, tau, m, n)
    for i, A in enumerate(mats):
        fo = oracle.bqrrp(A, int(b[i]), int(d[i]), int(seeds[i]))
        Fi, Ji, Ti = parts[i]
        assert info[i] == 0
        assert rank[i] == fo.rank, (i, rank[i], fo.rank)
        r = int(rank[i])
        if all(t["margin"] > 1e-6 for t in fo.trace):
            assert np.array_equal(Ji[:r], fo.jpvt[:r]), i
        rs, orth, ok = metrics(A, Fi, Ji, Ti, r)
        assert ok and rs <= 1e-12 and orth <= 1e-12, (i, rs, orth)
        bounds = list(range(0, A.shape[1], int(b[i])))
        assert np.all(trailing_norms(Fi, r, bounds) <= 1.1 * trailing_norms(fo.A, fo.rank, bounds)
                      + 1e-13 * np.linalg.norm(A)), i
        assert trunc_margin_ok(fo.A, fo.rank, np.linalg.norm(A), TOL, int(trunc[i])), (i, trunc[i])


def test_batched_matches_oracle_mixed_shapes_and_blocks():
    m, n = W.batched_shapes(40, 21, m_hi=320)
    mats = [W.batched_matrix(int(a), int(c), 500 + i) for i, (a, c) in enumerate(zip(m, n))]
    b = np.array([[16, 32, 64, 128][i % 4] for i in range(len(mats))], dtype=np.int64)
    d = np.array([int(np.ceil((1.25 if i % 3 else 1.5) * bb)) for i, bb in enumerate(b)], dtype=np.int64)
    seeds = np.arange(len(mats), dtype=np.uint64) * 7 + 3
    check_against_oracle(mats, b, d, seeds, run_batch(mats, b, d, seeds))


def test_batched_full_size_shapes():
    """The largest shapes of the workload (m up to 1024) against the oracle."""
    shapes = [(1024, 1000), (1000, 517), (777, 777), (1024, 33), (513, 200)]
    mats = [W.batched_matrix(a, c, 900 + i) for i, (a, c) in enumerate(shapes)]
    b = np.array([64, 32, 128, 16, 32], dtype=np.int64)
    d = np.ceil(1.25 * b).astype(np.int64)
    seeds = np.array([11, 12, 13, 14, 15], dtype=np.uint64)
    check_against_oracle(mats, b, d, seeds, run_batch(mats, b, d, seeds))


def test_batched_edge_cases():
    mats = [
        W.low_rank(300, 200, 37, 5),                 # rank found inside a block
        W.low_rank(200, 130, 64, 6),                 # rank at a block boundary (b = 32)
        np.zeros((70, 40)),                          # zero matrix: rank 0
        W.gaussian(65, 1, 3),                        # single column
        W.gaussian(100, 100, 4),                     # square
        W.gaussian(90, 40, 5),                       # b > n: one block
        W.gaussian(33, 33, 6),                       # n < d
    ]
    b = np.array([32, 32, 16, 16, 32, 64, 32], dtype=np.int64)
    d = np.array([40, 40, 20, 20, 40, 80, 40], dtype=np.int64)
    seeds = np.arange(7, dtype=np.uint64) + 40
    res = run_batch(mats, b, d, seeds)
    m, n, F, jpvt, tau, rank, trunc, info = res
    assert list(rank[:3]) == [37, 64, 0]
    check_against_oracle(mats, b, d, seeds, res)


def test_batched_nonfinite_matrix_is_left_untouched():
    mats = [W.gaussian(80, 50, 1), W.gaussian(60, 40, 2), W.gaussian(70, 30, 3)]
    mats[1][5, 7] = np.nan
    b = np.array([16, 16, 16], dtype=np.int64)
    d = np.array([20, 20, 20], dtype=np.int64)
    seeds = np.array([1, 2, 3], dtype=np.uint64)
    m, n, F, jpvt, tau, rank, trunc, info = run_batch(mats, b, d, seeds)
    parts = unpack(F, jpvt, tau, m, n)
    assert list(info) == [0, B.ENUMERIC, 0] and rank[1] == 0
    assert np.array_equal(parts[1][0], mats[1], equal_nan=True)
    assert np.array_equal(parts[1][1], np.arange(1, 41)) and np.all(parts[1][2] == 0.0)
    check_against_oracle([mats[0], mats[2]], b[[0, 2]], d[[0, 2]], seeds[[0, 2]],
                         (m[[0, 2]], n[[0, 2]],
                          np.concatenate([parts[0][0].ravel(order="F"), parts[2][0].ravel(order="F")]),
                          np.concatenate([parts[0][1], parts[2][1]]), np.concatenate([parts[0][2], parts[2][2]]),
                          rank[[0, 2]], trunc[[0, 2]], info[[0, 2]]))


def test_batched_result_independent_of_batch_and_graph():
    m, n = W.batched_shapes(24, 8, m_hi=400)
    mats = [W.batched_matrix(int(a), int(c), 70 + i) for i, (a, c) in enumerate(zip(m, n))]
    b = np.array([[32, 16, 64][i % 3] for i in range(24)], dtype=np.int64)
    d = np.ceil(1.25 * b).astype(np.int64)
    seeds = np.arange(24, dtype=np.uint64) + 1000
    eager = run_batch(mats, b, d, seeds, use_graph=False)
    graph = run_batch(mats, b, d, seeds, use_graph=True)
    for x, y in zip(eager, graph):
        assert np.array_equal(x, y)
    # each matrix alone (a batch of one) gives the same bits as in the mix
    parts = unpack(eager[2], eager[3], eager[4], eager[0], eager[1])
    for i in [0, 5, 11, 23]:
        alone = run_batch([mats[i]], b[[i]], d[[i]], seeds[[i]])
        assert np.array_equal(alone[2], parts[i][0].ravel(order="F"))
        assert np.array_equal(alone[3], parts[i][1]) and np.array_equal(alone[4], parts[i][2])
        assert alone[5][0] == eager[5][i] and alone[6][0] == eager[6][i]


def test_batched_graph_replay_is_repeatable():
    m, n = W.batched_shapes(16, 2, m_hi=256)
    mats = [W.batched_matrix(int(a), int(c), 10 + i) for i, (a, c) in enumerate(zip(m, n))]
    b = np.full(16, 32, dtype=np.int64)
    d = np.full(16, 40, dtype=np.int64)
    seeds = np.arange(16, dtype=np.uint64)
    A0 = torch.as_tensor(pack(mats), device="cuda")
    plan = B.BatchPlan(m, n, b, d, seeds, TOL)
    tot_j = int(n.sum())
    outs = []
    A = A0.clone()
    jpvt = torch.empty(tot_j, dtype=torch.int64, device="cuda")
    tau = torch.empty(tot_j, dtype=torch.float64, device="cuda")
    rank = torch.empty(16, dtype=torch.int64, device="cuda")
    trunc = torch.empty(16, dtype=torch.int64, device="cuda")
    for _ in range(3):
        A.copy_(A0)
        plan.factor(A, jpvt, tau, rank, trunc, use_graph=True)
        torch.cuda.synchronize()
        outs.append((np_(A), np_(jpvt), np_(tau), np_(rank), np_(trunc)))
    plan.close()
    for o in outs[1:]:
        for x, y in zip(outs[0], o):
            assert np.array_equal(x, y)


def test_batched_autotune_choices_are_valid_and_meet_the_bar():
    m, n = W.batched_shapes(60, 5, m_hi=600)
    mats = [W.batched_matrix(int(a), int(c), 300 + i) for i, (a, c) in enumerate(zip(m, n))]
    seeds = np.arange(60, dtype=np.uint64) + 9
    A = torch.as_tensor(pack(mats), device="cuda")
    A_before = A.clone()
    b, d, best = B.bqrrp_batch_autotune(m, n, seeds, A, TOL)
    assert torch.equal(A, A_before)                       # the caller's matrices are not touched
    assert best > 0
    assert np.all(d >= b) and np.all(d <= 256) and np.all(b >= 1) and np.all(b <= n)
    # one candidate block size per size class of n, capped at n
    cls = np.minimum(np.floor(np.log2(np.maximum(n, 1) / 32.0)).clip(0), 5).astype(int)
    for c in set(cls.tolist()):
        sel = cls == c
        assert any(np.array_equal(b[sel], np.minimum(cand, n[sel])) for cand in (16, 32, 64, 128)), c
    assert np.allclose(np.ceil(1.25 * b), d) or np.allclose(np.minimum(np.ceil(1.5 * b), 256), d)
    pick = [0, 17, 42, 59]
    sub = [mats[i] for i in pick]
    check_against_oracle(sub, b[pick], d[pick], seeds[pick], run_batch(sub, b[pick], d[pick], seeds[pick]))


def test_dependency_driven_and_lockstep_forms_agree_bitwise():
    """The default form runs every phase from one device task queue; the
    lock-step form (bqrrp_batch_plan_set_form(BQRRP_BATCH_LOCKSTEP)) launches
    one kernel per phase and iteration.  Both run the same per-phase
    arithmetic."""
    m, n = W.batched_shapes(30, 17, m_hi=500)
    mats = [W.batched_matrix(int(a), int(c), 800 + i) for i, (a, c) in enumerate(zip(m, n))]
    b = np.array([[16, 32, 64][i % 3] for i in range(30)], dtype=np.int64)
    d = np.ceil(1.25 * b).astype(np.int64)
    seeds = np.arange(30, dtype=np.uint64) + 77
    mega = run_batch(mats, b, d, seeds, use_graph=True)
    lock = run_batch(mats, b, d, seeds, use_graph=True, form=B.BATCH_LOCKSTEP)
    for x, y in zip(mega, lock):
        assert np.array_equal(x, y)
    check_against_oracle(mats[:6], b[:6], d[:6], seeds[:6],
                         (mega[0][:6], mega[1][:6], mega[2][:W.batch_offsets(mega[0][:6], mega[1][:6])[2]],
                          mega[3][:W.batch_offsets(mega[0][:6], mega[1][:6])[3]],
                          mega[4][:W.batch_offsets(mega[0][:6], mega[1][:6])[3]], mega[5][:6], mega[6][:6], mega[7][:6]))


def test_batched_narrow_tiles_meet_the_bar():
    """32-column trailing tiles (every other matrix), mixed shapes and block
    sizes, against the oracle; both launch forms give the same bits, and a
    matrix alone gives the same bits as in the mix."""
    m, n = W.batched_shapes(30, 41, m_hi=600)
    mats = [W.batched_matrix(int(a), int(c), 1300 + i) for i, (a, c) in enumerate(zip(m, n))]
    b = np.array([[16, 32, 64, 128, 8][i % 5] for i in range(30)], dtype=np.int64)
    b = np.minimum(b, np.maximum(n, 1))
    d = np.ceil(1.25 * b).astype(np.int64)
    tiles = np.array([32 if i % 2 == 0 else 64 for i in range(30)], dtype=np.int64)
    seeds = np.arange(30, dtype=np.uint64) + 500
    mega = run_batch(mats, b, d, seeds, use_graph=True, tiles=tiles)
    lock = run_batch(mats, b, d, seeds, form=B.BATCH_LOCKSTEP, tiles=tiles)
    for x, y in zip(mega, lock):
        assert np.array_equal(x, y)
    check_against_oracle(mats, b, d, seeds, mega)
    parts = unpack(mega[2], mega[3], mega[4], mega[0], mega[1])
    for i in [0, 7, 28]:
        alone = run_batch([mats[i]], b[[i]], d[[i]], seeds[[i]], tiles=tiles[[i]])
        assert np.array_equal(alone[2], parts[i][0].ravel(order="F"))


def test_batched_narrow_tiles_full_size_and_edges():
    shapes = [(1024, 1000), (1024, 33), (700, 64), (300, 31)]
    mats = [W.batched_matrix(a, c, 1400 + i) for i, (a, c) in enumerate(shapes)]
    mats += [W.low_rank(300, 200, 37, 5), np.zeros((70, 40)), W.gaussian(65, 1, 3)]
    b = np.array([16, 16, 32, 128, 32, 16, 16], dtype=np.int64)
    b = np.minimum(b, [A.shape[1] for A in mats])
    d = np.ceil(1.25 * b).astype(np.int64)
    seeds = np.arange(len(mats), dtype=np.uint64) + 40
    tiles = np.full(len(mats), 32, dtype=np.int64)
    check_against_oracle(mats, b, d, seeds, run_batch(mats, b, d, seeds, tiles=tiles))


def test_batched_tile_width_is_validated():
    with pytest.raises(B.BqrrpError):
        B.BatchPlan([64], [32], [16], [20], [1], TOL, tiles=[48])


def test_batched_autotune_tiles_choices_are_valid():
    m, n = W.batched_shapes(60, 6, m_hi=600)
    mats = [W.batched_matrix(int(a), int(c), 600 + i) for i, (a, c) in enumerate(zip(m, n))]
    seeds = np.arange(60, dtype=np.uint64) + 19
    A = torch.as_tensor(pack(mats), device="cuda")
    A_before = A.clone()
    b, d, tiles, best = B.bqrrp_batch_autotune_tiles(m, n, seeds, A, TOL)
    assert torch.equal(A, A_before)
    assert best > 0
    assert np.all(np.isin(tiles, [32, 64]))
    assert np.all(d >= b) and np.all(b >= 1) and np.all(b <= n)
    # one tile width per size class of n
    cls = np.minimum(np.floor(np.log2(np.maximum(n, 1) / 32.0)).clip(0), 5).astype(int)
    for c in set(cls.tolist()):
        assert len(set(tiles[cls == c].tolist())) == 1, c
    pick = [1, 30, 58]
    sub = [mats[i] for i in pick]
    check_against_oracle(sub, b[pick], d[pick], seeds[pick],
                         run_batch(sub, b[pick], d[pick], seeds[pick], tiles=tiles[pick]))
