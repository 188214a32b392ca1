"""GPU parity of each BQRRP step against the CPU oracle, through the C ABI.

Integer and index results (sketch operator, pivots, permutations) must be
bit-exact.  Floating-point results are compared normwise with tolerances
derived from the arithmetic: a sum of K products carries at most about
K*u*sum|a_i b_i| of rounding difference between two summation orders
(u = 2^-53); factorizations are compared through quantities they determine
uniquely (R up to row signs, reconstructed products).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2507_00976_b300 as bq
from gpu_util import np_
from paper_2507_00976_b300 import binding as B
from paper_2507_00976_b300 import workloads as W

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


def dev(x):
    return bq.to_colmajor(x)


# ------------------------------------------------------------- sketch (a0, a1)
@pytest.mark.parametrize("d,m,seed", [(160, 2000, 1), (300, 777, (5 << 32) | 3), (1, 1, 0), (129, 64, 9)])
def test_sketch_operator_dense_bitexact(d, m, seed):
    S = bq.bqrrp_sketch_operator(d, m, seed)
    torch.cuda.synchronize()
    assert np.array_equal(np_(S), oracle.sketch_operator(d, m, seed))


@pytest.mark.parametrize("d,m,nnz", [(8, 500, 8), (40, 1000, 8), (17, 300, 3), (640, 333, 8)])
def test_sketch_operator_sparse_bitexact(d, m, nnz):
    S = bq.bqrrp_sketch_operator(d, m, 77, kind=1, nnz=nnz)
    torch.cuda.synchronize()
    assert np.array_equal(np_(S), oracle.sketch_operator(d, m, 77, kind=1, nnz=nnz))


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("d,m,n", [(160, 2000, 1000), (37, 333, 21), (64, 4097, 65),
                                   (2560, 3000, 50),     # d = ceil(1.25 * 2048): the sparse kernel's rows in two tiles
                                   (4100, 700, 9)])      # three row tiles, a ragged last one
def test_sketch_apply_exact_on_integer_data(kind, d, m, n):
    rng = np.random.default_rng(d + m)
    A = rng.integers(-40, 40, size=(m, n)).astype(np.float64)
    Msk = bq.bqrrp_sketch_apply(dev(A), d, 5, kind=kind, nnz=8)
    ref = oracle.sketch_apply(oracle.sketch_operator(d, m, 5, kind=kind, nnz=8), A)
    assert np.array_equal(np_(Msk), ref)          # every partial sum is an exact integer


@pytest.mark.parametrize("kind", [0, 1])
def test_sketch_apply_gaussian(kind):
    d, m, n = 160, 2000, 1000
    A = W.gaussian(m, n, 3)
    Msk = np_(bq.bqrrp_sketch_apply(dev(A), d, 11, kind=kind, nnz=8))
    ref = oracle.sketch_apply(oracle.sketch_operator(d, m, 11, kind=kind, nnz=8), A)
    bound = 2 * m * U * np.abs(A).sum(axis=0)[None, :]
    assert np.all(np.abs(Msk - ref) <= bound)


# ------------------------------------------------------------- DGEMM
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (64, 64, 64), (65, 63, 17), (130, 257, 300), (7, 100, 5000),
                                   (512, 96, 20000), (33, 40, 0)])
def test_dgemm_matches_fp64_reference(ta, tb, M, N, K):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.standard_normal((K, M) if ta == "T" else (M, K))
    B = rng.standard_normal((N, K) if tb == "T" else (K, N))
    C0 = rng.standard_normal((M, N))
    Cd = dev(C0)
    bq.bqrrp_dgemm(ta, tb, -0.5, dev(A), dev(B), 2.0, Cd)
    opA = A.T if ta == "T" else A
    opB = B.T if tb == "T" else B
    ref = -0.5 * (opA @ opB) + 2.0 * C0
    bound = 2 * (K + 2) * U * (0.5 * np.abs(opA) @ np.abs(opB) + 2 * np.abs(C0)) + 1e-300
    assert np.all(np.abs(np_(Cd) - ref) <= bound)


def test_dgemm_beta_zero_ignores_nan_in_c():
    A = np.ones((70, 5))
    B = np.ones((5, 90))
    C = dev(np.full((70, 90), np.nan))
    bq.bqrrp_dgemm("N", "N", 1.0, dev(A), dev(B), 0.0, C)
    assert np.all(np_(C) == 5.0)


# ------------------------------------------------------------- GEQRF (own unpivoted QR)
@pytest.mark.parametrize("m,n", [(300, 200), (1000, 1000), (2049, 130), (64, 64), (70, 200), (5000, 65)])
def test_geqrf_matches_oracle(m, n):
    A = W.gaussian(m, n, m + n)
    Ad = dev(A)
    tau = np_(bq.bqrrp_geqrf(Ad))
    F = np_(Ad)
    Fo, tau_o = oracle.geqrf(A)
    k = min(m, n)
    nrm = np.linalg.norm(A)
    assert np.linalg.norm(np.triu(F)[:k] - np.triu(Fo)[:k]) <= 1e-13 * np.sqrt(m * n) * nrm
    assert np.max(np.abs(tau[:k] - tau_o)) <= 1e-12
    assert np.linalg.norm(np.tril(F, -1) - np.tril(Fo, -1)) <= 1e-12 * np.sqrt(m * n)


# ------------------------------------------------------------- Alg. 2 (qrcp_wide)
@pytest.mark.parametrize("d,N", [(160, 1000), (40, 300), (64, 30), (100, 100), (320, 16384), (7, 9), (130, 131)])
def test_qrcp_wide_pivots_bitexact_and_rsk(d, N):
    Msk0 = W.gaussian(d, N, d * 1000 + N)
    Md = dev(Msk0)
    Jsk, ipiv = bq.bqrrp_qrcp_wide(Md)
    _, ipiv_o, margin = oracle.lupp(Msk0.T.copy())
    J_o = oracle.piv_transform(N, ipiv_o)
    assert margin > 1e-9
    assert np.array_equal(np_(ipiv), ipiv_o)
    assert np.array_equal(np_(Jsk), J_o)
    Ro, _ = oracle.geqrf(Msk0[:, J_o])
    Ro = np.triu(Ro)
    R = np_(Md)
    assert np.all(np.tril(R, -1) == 0)
    # R^sk is unique up to row signs (the GPU forms it from the LU factors as
    # R(U^T) L^T; the signs cancel in everything derived from it)
    k = min(d, N)
    sg = np.ones(d)
    sg[:k] = np.sign(np.diag(R)[:k] * np.diag(Ro)[:k])
    assert np.linalg.norm(sg[:, None] * R - Ro) <= 1e-12 * np.sqrt(d * N) * np.linalg.norm(Msk0)


@pytest.mark.parametrize("d,N", [(40, 300), (64, 130)])
def test_qrcp_wide_exact_ties_take_the_first_maximum(d, N):
    # duplicated and negated sketch columns make rows of X = Msk^T tie exactly
    # in |value|; within one 64-step panel equal rows cancel exactly, so the
    # oracle's first-maximum choices are unique and must be reproduced
    Msk0 = W.gaussian(d, N, 77 + d)
    Msk0[:, N // 2:N // 2 + 40] = Msk0[:, 0:40]
    Msk0[:, N - 5] = -Msk0[:, 3]
    Jsk, ipiv = bq.bqrrp_qrcp_wide(dev(Msk0))
    _, ipiv_o, _ = oracle.lupp(Msk0.T.copy())
    assert np.array_equal(np_(ipiv), ipiv_o)
    assert np.array_equal(np_(Jsk), oracle.piv_transform(N, ipiv_o))


def test_lu_exchange_wait_times_out_and_context_stays_usable():
    # one CTA withholds its first candidate, so every bounded wait of that LU
    # launch runs out (a flag nothing sets); the status must say so, and the
    # same LU must then complete in the same context with the oracle's pivots
    Msk0 = W.gaussian(64, 4096, 5)
    rc, ipiv = B.bqrrp_selftest_lu_wait_timeout(dev(Msk0))
    assert rc == 0, B.last_error()
    _, ipiv_o, margin = oracle.lupp(Msk0.T.copy())
    assert margin > 1e-9
    assert np.array_equal(np_(ipiv), ipiv_o)
    _, ipiv2 = bq.bqrrp_qrcp_wide(dev(Msk0))
    assert np.array_equal(np_(ipiv2), ipiv_o)


def test_qrcp_wide_nonfinite_sketch_gives_identity_pivots():
    Msk0 = W.gaussian(20, 50, 1)
    Msk0[3, 7] = np.inf
    Jsk, _ = bq.bqrrp_qrcp_wide(dev(Msk0))
    assert np.array_equal(np_(Jsk), np.arange(50))


# ------------------------------------------------------------- Alg. 5 (col_perm)
@pytest.mark.parametrize("m,N,moves", [(1000, 300, "perm"), (4097, 64, "perm"), (3, 500, "swaps"),
                                       (128, 40, "none"), (1, 7, "perm"), (8192 + 1000, 96, "perm")])
def test_col_perm_bitexact(m, N, moves):
    rng = np.random.default_rng(m + N)
    M = rng.standard_normal((m, N))
    if moves == "perm":
        J = rng.permutation(N)
    elif moves == "swaps":
        J = np.arange(N)
        for _ in range(20):
            a, b = rng.integers(0, N, 2)
            J[[a, b]] = J[[b, a]]
    else:
        J = np.arange(N)
    Md = dev(M)
    bq.bqrrp_col_perm(Md, torch.as_tensor(J, dtype=torch.int64, device="cuda"))
    assert np.array_equal(np_(Md), M[:, J])


# ------------------------------------------------------------- Alg. 3 (CholQR panel)
@pytest.mark.parametrize("rows,w,d", [(300, 32, 40), (1000, 100, 125), (2065, 128, 160), (4096, 64, 80),
                                      (100, 100, 125), (6000, 200, 250)])
def test_cholqr_panel_matches_oracle(rows, w, d):
    Mp = W.spectrum(rows, w, W.geometric_sigma(w, -6), rows + w)
    S = oracle.sketch_operator(d, rows, 3)
    Rsk, _ = oracle.geqrf(S @ Mp)
    Rsk = np.triu(Rsk)[:w, :w].copy()
    Fo, To, tau_o, ko = oracle.cholqr_panel(Mp, Rsk, w)
    assert ko == w
    Md = dev(Mp)
    T, tau, k = bq.bqrrp_cholqr_panel(Md, dev(Rsk), w)
    assert k == w
    F = np_(Md)
    nrm = np.linalg.norm(Mp)
    assert np.linalg.norm(np.triu(F)[:w] - np.triu(Fo)[:w]) <= 1e-12 * nrm
    assert np.linalg.norm(np.tril(F, -1) - np.tril(Fo, -1)) <= 1e-10 * np.sqrt(rows * w)
    assert np.max(np.abs(np_(tau) - tau_o)) <= 1e-10
    assert np.linalg.norm(np_(T) - To) <= 1e-10 * np.linalg.norm(To)
    assert np.all(np_(tau) >= 1 - 1e-12) and np.all(np_(tau) <= 2 + 1e-12)
