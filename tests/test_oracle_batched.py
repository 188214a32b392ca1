"""Pins of the oracle's batched-workload pieces: the truncation rule (the
Sec. 6 residual measure ||R(i:, i:)||_F used as a cut-off), the Frobenius
norm, and the workload generator's distributions.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_2507_00976_b300 import workloads as W


def _brute_trunc(R, rank, anorm, tol):
    """Definition written out with numpy block norms, one i at a time."""
    Ru = np.triu(R)
    for i in range(rank + 1):
        if np.linalg.norm(Ru[i:rank, i:]) <= tol * anorm:
            return i
    return rank


@pytest.mark.parametrize("m,n,rank", [(9, 7, 7), (12, 12, 12), (10, 6, 4), (5, 5, 0), (30, 20, 20)])
def test_trunc_rank_matches_block_norm_definition(m, n, rank):
    rng = np.random.default_rng(m * n + rank)
    # geometric row scales so that the cut lands in the middle for some tol
    R = rng.standard_normal((m, n)) * (10.0 ** -np.arange(m))[:, None]
    anorm = np.linalg.norm(np.triu(R))
    for tol in [0.0, 1e-12, 1e-6, 1e-3, 0.1, 0.5, 0.999, 2.0]:
        assert oracle.trunc_rank(R, rank, anorm, tol) == _brute_trunc(R, rank, anorm, tol), tol


def test_trunc_rank_exact_low_rank_recovers_rank():
    A = W.low_rank(300, 200, 37, 5)
    f = oracle.bqrrp(A, 32, 40, 7)
    assert f.rank == 37
    assert oracle.trunc_rank(f.A, f.rank, np.linalg.norm(A), 1e-10) == 37


@pytest.mark.parametrize("tol", [1e-2, 1e-4, 1e-6, 1e-8])
def test_trunc_rank_respects_eckart_young(tol):
    """||R(i:, i:)||_F >= (sum_{j>=i} sigma_j^2)^(1/2) for any A P = Q R, so the
    cut can never come before the SVD's optimal cut at the same tolerance."""
    m, n = 260, 180
    sig = W.batched_sigma(n)
    A = W.spectrum(m, n, sig, 11)
    f = oracle.bqrrp(A, 32, 40, 2)
    anorm = np.linalg.norm(sig)
    tails = np.sqrt(np.cumsum((sig ** 2)[::-1])[::-1])
    svd_cut = int(np.argmax(tails <= tol * anorm)) if np.any(tails <= tol * anorm) else n
    cut = oracle.trunc_rank(f.A, f.rank, anorm, tol)
    assert cut >= svd_cut
    # BQRRP is rank revealing on this spectrum: every trailing block of R is
    # within a small factor of the optimal tail (measured 5.3), so the cut
    # lands where the optimal tail has fallen by at most that factor
    R = np.triu(f.A)[:n]
    ratio = max(np.linalg.norm(R[i:, i:]) / tails[i] for i in range(n))
    assert ratio < 20
    assert cut <= n


def test_fro_norm_plain_sum():
    A = W.gaussian(37, 23, 3)
    assert abs(oracle.fro_norm(A) - np.sqrt((A * A).sum())) <= 1e-14 * oracle.fro_norm(A)
    assert oracle.fro_norm(np.zeros((4, 3))) == 0.0


def test_batched_shapes_distribution():
    m, n = W.batched_shapes(20000, 3)
    assert m.min() >= 64 and m.max() <= 1024 and np.all(n >= 32) and np.all(n <= m)
    # log m uniform on [log 64, log 1024]: quartiles at 128, 256, 512
    q = np.quantile(m, [0.25, 0.5, 0.75])
    assert np.allclose(q, [128, 256, 512], rtol=0.05)
    # given m, (log n - log 32)/(log m - log 32) is uniform on [0, 1]
    u = (np.log(n + 0.5) - np.log(32)) / (np.log(m) - np.log(32))
    assert abs(np.mean(u) - 0.5) < 0.02


def test_batched_matrix_has_the_stated_spectrum():
    A = W.batched_matrix(120, 50, 4)
    s = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(s, 10.0 ** (-8.0 * np.arange(50) / 49), rtol=1e-6, atol=1e-15)


def test_batch_offsets_pack_back_to_back():
    m = np.array([5, 7, 3])
    n = np.array([2, 7, 1])
    offA, offJ, tA, tJ = W.batch_offsets(m, n)
    assert list(offA) == [0, 10, 59] and tA == 62
    assert list(offJ) == [0, 2, 9] and tJ == 10


def test_bqrrp_batched_is_the_per_matrix_oracle():
    m, n = W.batched_shapes(5, 9, m_hi=200)
    mats = [W.batched_matrix(int(a), int(b), 100 + i) for i, (a, b) in enumerate(zip(m, n))]
    bs = [16, 32, 16, 64, 32]
    ds = [20, 40, 24, 80, 40]
    res = oracle.bqrrp_batched(mats, bs, ds, list(range(5)), 1e-8)
    for i in range(5):
        f = oracle.bqrrp(mats[i], bs[i], ds[i], i)
        assert np.array_equal(res.F[i], f.A) and np.array_equal(res.jpvt[i], f.jpvt)
        assert res.rank[i] == f.rank == n[i]
        assert res.trunc_rank[i] == oracle.trunc_rank(f.A, f.rank, np.linalg.norm(mats[i]), 1e-8)
