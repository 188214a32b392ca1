"""Pins for the CPU oracle: each test checks an oracle routine against
something other than itself -- published known-answer vectors, LAPACK
(through scipy), exact rational arithmetic, brute force on tiny inputs,
closed forms derived from the paper's relations, or invariants the paper
states.  All run on the CPU (``-m "not gpu"``).
"""
from fractions import Fraction
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from checks import form_q, form_q_slow, metrics, trailing_norms, upper_r
from paper_2507_00976_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- Philox
def test_philox_known_answer_vectors():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(x, 16) for x in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = oracle.philox4x32_10(r[0:4], r[4:6])
        assert [int(x) for x in out] == r[6:10]


# ----------------------------------------------------------------- sketch
def test_dense_sketch_is_pm1_prefix_stable_and_balanced():
    S_small = oracle.sketch_operator(100, 700, 11)
    S_big = oracle.sketch_operator(300, 700, 11)
    assert set(np.unique(S_big)) == {-1.0, 1.0}
    assert np.array_equal(S_small, S_big[:100])           # rows prefix-stable in d
    assert not np.array_equal(S_big[:128], S_big[128:256])  # row blocks independent
    assert abs(S_big.mean()) < 0.01
    assert not np.array_equal(S_big, oracle.sketch_operator(300, 700, 12))
    # seed uses both 32-bit halves of the key
    assert not np.array_equal(oracle.sketch_operator(40, 50, 5), oracle.sketch_operator(40, 50, 5 + (1 << 32)))


def test_dense_sketch_bit_layout_matches_generator():
    d, m, seed = 200, 9, (3 << 32) | 17
    S = oracle.sketch_operator(d, m, seed)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for j in range(m):
        for blk in range(2):
            out = oracle.philox4x32_10([j, blk, 0, 0], key)
            for q in range(128):
                r = blk * 128 + q
                if r >= d:
                    break
                bit = (int(out[q // 32]) >> (q % 32)) & 1
                assert S[r, j] == (-1.0 if bit else 1.0)


@pytest.mark.parametrize("d,nnz", [(8, 8), (40, 8), (300, 8), (17, 3)])
def test_sparse_sketch_structure(d, nnz):
    m = 6000
    S = oracle.sketch_operator(d, m, 99, kind=1, nnz=nnz)
    nz = S != 0
    assert np.all(nz.sum(axis=0) == nnz)
    assert set(np.unique(S[nz])) <= {-1.0, 1.0}
    counts = nz.sum(axis=1)
    expect = m * nnz / d
    assert counts.min() > 0.6 * expect and counts.max() < 1.5 * expect
    with pytest.raises(ValueError):
        oracle.sketch_operator(4, 10, 1, kind=1, nnz=5)


def test_sketch_apply_exact_on_integer_data():
    rng = np.random.default_rng(0)
    A = rng.integers(-50, 50, size=(333, 21)).astype(np.float64)
    S = oracle.sketch_operator(37, 333, 4)
    out = oracle.sketch_apply(S, A)
    assert np.array_equal(out, S @ A)      # all partial sums are exact integers


# ----------------------------------------------------------------- GEQRF
@pytest.mark.parametrize("shape", [(50, 30), (40, 40), (30, 50), (1, 5), (7, 1)])
def test_geqrf_matches_lapack_dgeqrf(shape):
    A = W.gaussian(*shape, seed=3)
    if shape[1] > 3:
        A[:, 2] = 0.0      # a zero column below the diagonal gives tau = 0 there
        A[:2, 2] = 1.0
    F, tau = oracle.geqrf(A)
    (qr, tau_l), _ = sla.qr(A, mode="raw")
    scale = max(1.0, np.abs(A).max())
    np.testing.assert_allclose(F, qr, atol=1e-13 * scale, rtol=0)
    np.testing.assert_allclose(tau, tau_l, atol=1e-14, rtol=0)


# ----------------------------------------------------------------- QRCP (BG)
def _greedy_max_norm_order(A):
    """Brute force: repeatedly take the first column of largest residual norm
    after projecting out the columns already chosen (no Householder)."""
    m, n = A.shape
    chosen = []
    for _ in range(min(m, n)):
        if chosen:
            Qc, _ = np.linalg.qr(A[:, chosen])
            Rm = A - Qc @ (Qc.T @ A)
        else:
            Rm = A.copy()
        norms = np.linalg.norm(Rm, axis=0)
        norms[chosen] = -1.0
        chosen.append(int(np.argmax(norms)))
    return chosen


@pytest.mark.parametrize("seed", range(5))
def test_qrcp_bg_brute_force_tiny(seed):
    A = W.gaussian(8, 6, seed)
    F, jpvt, tau = oracle.qrcp_bg(A)
    assert list(jpvt[:6] - 1) == _greedy_max_norm_order(A)
    res, orth, ok = metrics(A, F, jpvt, np.r_[tau, np.zeros(6 - len(tau))], 6)
    assert res < 1e-14 and orth < 1e-14 and ok


def test_qrcp_bg_matches_lapack_dgeqp3():
    A = W.gaussian(60, 40, 8)
    F, jpvt, tau = oracle.qrcp_bg(A)
    R_l, P = sla.qr(A, pivoting=True, mode="r")
    assert list(jpvt - 1) == list(P)
    np.testing.assert_allclose(np.triu(F)[:40], R_l[:40], atol=1e-12 * np.abs(A).max())


@pytest.mark.parametrize("b", [1, 7, 8, 40])
@pytest.mark.parametrize("panel", ["cholqr", "hqr"])
def test_identity_sketch_with_bg_reduces_bqrrp_to_dgeqp3(b, panel):
    """Special case derived from the sketch update of Alg. 1: with S = I_m
    (d = m) and qrcp_wide by Businger-Golub, R^sk11 = D R11 with D = +-1, so
    the update zeroes the first w sketch rows and leaves the trailing R of the
    pivoted QR.  The whole loop (block pivots, composition of J, panel,
    trailing update, sketch update) then makes Businger-Golub's choices: the
    pivots equal LAPACK dgeqp3's and R equals its R up to row signs."""
    A = W.gaussian(60, 40, 8)
    fo = oracle.bqrrp(A, b, 60, 0, sketch_kind=2, panel=panel)
    R_l, P = sla.qr(A, pivoting=True, mode="r")
    assert fo.rank == 40
    assert list(fo.jpvt - 1) == list(P)
    np.testing.assert_allclose(np.abs(np.triu(fo.A)[:40]), np.abs(R_l[:40]), atol=1e-12 * np.abs(A).max())
    res, orth, ok = metrics(A, fo.A, fo.jpvt, fo.tau, fo.rank)
    assert res < 1e-13 and orth < 1e-13 and ok


def test_identity_sketch_hook_requires_d_equal_m():
    assert oracle.bqrrp_status(W.gaussian(30, 20, 1), 4, 29, sketch_kind=2) == -6


# ----------------------------------------------------------------- LUPP
@pytest.mark.parametrize("shape", [(200, 30), (30, 30), (20, 40)])
def test_lupp_matches_lapack_dgetrf(shape):
    X = W.gaussian(*shape, seed=21)
    LU, ipiv, margin = oracle.lupp(X)
    lu_l, piv_l = sla.lu_factor(X)
    assert list(ipiv) == list(piv_l[: len(ipiv)])
    np.testing.assert_allclose(LU, lu_l, atol=1e-12, rtol=0)
    assert 0 < margin <= 1


def test_lupp_zero_pivot_continues_like_getrf():
    X = W.gaussian(12, 6, seed=2)
    X[:, 2] = X[:, 0] * 2.0 + X[:, 1] * 0.5           # rank drop: exact zero pivot column later
    X[:, 2] = X[:, 0] + X[:, 1]
    X = np.round(X * 4) / 4                             # dyadic data keeps the cancellation exact
    X[:, 2] = X[:, 0] + X[:, 1]
    LU, ipiv, _ = oracle.lupp(X)
    lu_l, piv_l = sla.lu_factor(X, check_finite=True)
    assert list(ipiv) == list(piv_l[:6])


def _exact_lupp(rows):
    """Partial-pivoting LU in exact rationals; first-max tie rule."""
    X = [[Fraction(v) for v in r] for r in rows]
    N, d = len(X), len(X[0])
    ipiv = []
    for j in range(min(N, d)):
        best, p = -1, j
        for t in range(j, N):
            if abs(X[t][j]) > best:
                best, p = abs(X[t][j]), t
        ipiv.append(p)
        X[j], X[p] = X[p], X[j]
        if X[j][j] != 0:
            for t in range(j + 1, N):
                l = X[t][j] / X[j][j]
                X[t][j] = l
                for c in range(j + 1, d):
                    X[t][c] -= l * X[j][c]
    return ipiv


@pytest.mark.parametrize("rows", [
    [[1, 2, 3], [-1, 0, 2], [1, 5, -4], [0, 1, 1]],     # three-way tie in column 0
    [[0, 1, 1], [0, 2, 2], [0, 4, -1], [0, 4, 3]],      # zero first column, tie later
    [[2, -2, 1], [4, 1, 0], [-4, 3, 2], [1, 1, 1]],
])
def test_lupp_first_max_rule_exact(rows):
    X = np.array(rows, dtype=np.float64)
    _, ipiv, _ = oracle.lupp(X)
    assert list(ipiv) == _exact_lupp(rows)


def test_piv_transform_matches_lapack_permutation():
    X = W.gaussian(50, 12, seed=5)
    _, ipiv, _ = oracle.lupp(X)
    J = oracle.piv_transform(50, ipiv)
    P, L, U = sla.lu(X)                  # X = P L U  ->  (P^T X)[t] = X[perm[t]]
    perm = np.argmax(P, axis=0)
    assert list(J) == list(perm)
    assert sorted(J) == list(range(50))


def _col_perm_sequential(M, Jqr1):
    """Alg. 4 (Sec. 2.5): swap, then find-and-update the pivot vector
    (1-based).  Reading: the find runs over the entries not yet placed
    (indices > i); over the whole vector it can hit an already-placed entry
    holding the same value and mis-track a column."""
    M = M.copy()
    J = list(Jqr1)
    n = M.shape[1]
    for i in range(n):
        j = J[i] - 1
        M[:, [i, j]] = M[:, [j, i]]
        for idx in range(i + 1, n):
            if J[idx] == i + 1:
                J[idx] = j + 1
                break
    return M


def test_parallel_gather_equals_sequential_alg4():
    rng = np.random.default_rng(1)
    M = rng.standard_normal((7, 15))
    Jsk = rng.permutation(15)
    gathered = M[:, Jsk]                                  # Alg. 5 semantics used by the oracle
    assert np.array_equal(gathered, _col_perm_sequential(M, Jsk + 1))


# ----------------------------------------------------------------- ORHR_COL
def _larft(Y, tau):
    """Forward column-wise compact-WY T from reflectors (LAPACK larft
    recurrence): T(0:j, j) = -tau_j T(0:j,0:j) Y(:,0:j)^T Y(:,j)."""
    k = len(tau)
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = tau[j]
        if j:
            T[:j, j] = -tau[j] * T[:j, :j] @ (Y[:, :j].T @ Y[:, j])
    return T


@pytest.mark.parametrize("rows,k", [(50, 12), (12, 12), (200, 1), (64, 40)])
def test_orhr_col_reconstruction_identities(rows, k):
    Q, _ = np.linalg.qr(W.gaussian(rows, k, seed=rows + k))
    Y, T, D = oracle.orhr_col(Q)
    assert np.allclose(np.triu(Y, 1)[:k], 0) and np.allclose(np.diag(Y[:k]), 1)
    assert np.allclose(np.tril(T, -1), 0)
    tau = np.diag(T)
    assert np.all(tau >= 1 - 1e-14) and np.all(tau <= 2 + 1e-14)
    H = np.eye(rows) - Y @ T @ Y.T
    np.testing.assert_allclose(H[:, :k], Q * D[None, :], atol=1e-13)
    # product of the individual reflectors equals the compact form
    P = np.eye(rows)
    for j in range(k):
        v = Y[:, j]
        P = P @ (np.eye(rows) - tau[j] * np.outer(v, v))
    np.testing.assert_allclose(P, H, atol=1e-13)
    np.testing.assert_allclose(T, _larft(Y, tau), atol=1e-12)


def test_orhr_col_identity_columns():
    Q = np.eye(9)[:, :4]
    Y, T, D = oracle.orhr_col(Q)
    H = np.eye(9) - Y @ T @ Y.T
    np.testing.assert_allclose(H[:, :4], Q * D[None, :], atol=1e-15)


# ----------------------------------------------------------------- BQRRP
@pytest.mark.parametrize("panel", ["cholqr", "hqr"])
@pytest.mark.parametrize("shape,b,d", [((300, 200), 32, 40), ((257, 131), 16, 20), ((90, 90), 90, 113),
                                       ((64, 40), 7, 9)])
def test_bqrrp_is_a_valid_qrcp(panel, shape, b, d):
    A = W.gaussian(*shape, seed=sum(shape))
    f = oracle.bqrrp(A, b, d, 5, panel=panel)
    assert f.rank == shape[1]
    res, orth, ok = metrics(A, f.A, f.jpvt, f.tau, f.rank)
    assert ok and res < 1e-14 and orth < 1e-13
    assert all(t["k"] == t["w"] for t in f.trace)


def test_bqrrp_r_equals_qr_of_permuted_input():
    A = W.spectrum(200, 150, W.geometric_sigma(150, -8), 9)
    f = oracle.bqrrp(A, 24, 30, 3)
    R = upper_r(f.A, f.rank)[:150]
    R_l = sla.qr(A[:, f.jpvt - 1], mode="r")[0][:150]
    sg = np.sign(np.diag(R) * np.diag(R_l))
    np.testing.assert_allclose(R, sg[:, None] * R_l, atol=1e-13 * np.linalg.norm(A))


def test_bqrrp_cholqr_and_householder_panels_agree():
    A = W.gaussian(260, 180, 2)
    f1 = oracle.bqrrp(A, 32, 40, 8, panel="cholqr")
    f2 = oracle.bqrrp(A, 32, 40, 8, panel="hqr")
    assert np.array_equal(f1.jpvt, f2.jpvt)
    np.testing.assert_allclose(np.abs(np.triu(f1.A)), np.abs(np.triu(f2.A)), atol=1e-12)


def test_gamma_invariance_of_first_block_pivots():
    """Sec. 2.1: with Alg. 2 the first b pivots are the same for gamma = 1
    and gamma > 1 (prefix-stable sketch rows)."""
    for seed in range(3):
        A = W.gaussian(400, 250, seed)
        b = 40
        p1 = oracle.bqrrp(A, b, b, 17 + seed, max_iters=1).jpvt[:b]
        p2 = oracle.bqrrp(A, b, 50, 17 + seed, max_iters=1).jpvt[:b]
        p3 = oracle.bqrrp(A, b, 120, 17 + seed, max_iters=1).jpvt[:b]
        assert np.array_equal(p1, p2) and np.array_equal(p1, p3)


def test_sketch_update_closed_form():
    """After one iteration the updated sketch equals (Qsk^T S Q)(:, b:) M22',
    derived from S M P = Qsk Rsk and M P = Q R (Alg. 1 sample update)."""
    m, n, b, d, seed = 120, 64, 32, 40, 6
    A = W.gaussian(m, n, 4)
    f = oracle.bqrrp(A, b, d, seed, max_iters=1, want_sketch=True)
    assert f.rank == b
    S = oracle.sketch_operator(d, m, seed)
    Msk_perm = S @ A[:, f.jpvt - 1]
    Qsk, Rsk = sla.qr(Msk_perm, mode="economic")
    Q = form_q(f.A, f.tau, b)
    M22 = f.A[b:, b:]
    closed = (Qsk.T @ S @ Q)[:, b:] @ M22
    np.testing.assert_allclose(f.sketch[:, b:], closed, atol=1e-11 * np.abs(closed).max())


@pytest.mark.parametrize("r,b,d", [(37, 16, 20), (32, 16, 20), (1, 8, 10), (100, 25, 30)])
def test_bqrrp_returns_exact_rank(r, b, d):
    A = W.low_rank(300, 200, r, seed=r)
    f = oracle.bqrrp(A, b, d, 1)
    assert f.rank == r
    res, orth, ok = metrics(A, f.A, f.jpvt, f.tau, f.rank)
    assert ok and res < 1e-12 and orth < 1e-13


def test_bqrrp_zero_matrix():
    f = oracle.bqrrp(np.zeros((30, 20)), 8, 10, 1)
    assert f.rank == 0 and np.all(f.tau == 0) and sorted(f.jpvt) == list(range(1, 21))


def test_bqrrp_rank_revealing_bounds():
    n = 160
    sig = W.geometric_sigma(n, -9)
    A = W.spectrum(220, n, sig, 12)
    f = oracle.bqrrp(A, 20, 25, 2)
    tn = trailing_norms(f.A, f.rank)
    tail = np.sqrt(np.cumsum((sig ** 2)[::-1])[::-1])
    assert np.all(tn >= tail * (1 - 1e-8))                           # Eckart-Young
    ratio = np.abs(np.diag(f.A)[:n]) / sig
    assert ratio.min() >= (n * (n + 1) / 2) ** -0.5 * 0.5             # Sec. 6 bounds (loose)
    assert ratio.max() <= 2.0 ** (n - 1)


def test_bqrrp_kahan_smoke():
    """Sec. 6 matrix; the paper's ratio curves are figures only (parity
    unpinned), so this checks a valid factorization."""
    A = W.kahan(256)
    f = oracle.bqrrp(A, 32, 40, 3)
    assert np.all(np.isfinite(f.A))
    res, orth, ok = metrics(A, f.A, f.jpvt, f.tau, f.rank)
    assert ok and res < 1e-13 and orth < 1e-13


def test_bqrrp_sparse_sketch_valid():
    A = W.gaussian(300, 200, 4)
    f = oracle.bqrrp(A, 32, 40, 5, sketch_kind=1, nnz=8)
    res, orth, ok = metrics(A, f.A, f.jpvt, f.tau, f.rank)
    assert f.rank == 200 and ok and res < 1e-14 and orth < 1e-13


def test_bqrrp_argument_checks():
    A = W.gaussian(10, 8, 1)
    assert oracle.bqrrp_status(A, 4, 5) == 0
    assert oracle.bqrrp_status(W.gaussian(5, 8, 1), 4, 5) == -1
    assert oracle.bqrrp_status(A, 0, 5) == -5
    assert oracle.bqrrp_status(A, 4, 3) == -6
    assert oracle.bqrrp_status(A, 4, 5, lda=5) == -4
    assert oracle.bqrrp_status(A, 4, 5, sketch_kind=1, nnz=9) == -9
    B = A.copy()
    B[3, 3] = np.nan
    assert oracle.bqrrp_status(B, 4, 5) == 3
    assert oracle.bqrrp_status(np.zeros((4, 0)), 4, 5) == 0


def test_c1_oracle_meets_targets():
    A = W.c1_matrix()
    f = oracle.bqrrp(A, 128, 160, 1)
    assert f.rank == 1000
    res, orth, ok = metrics(A, f.A, f.jpvt, f.tau, f.rank)
    assert ok and res < 1e-14 and orth < 1e-12
    assert [t["w"] for t in f.trace] == [128] * 7 + [104]
