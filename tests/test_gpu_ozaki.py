"""The mixed-precision form: FP64-accurate products on the bf16 tensor cores
(exact balanced 8-bit slices, FP32 sums that stay below 2^24, exact integer
recombination rounded once to FP64), through the C ABI.

Bar: integer data, whose slice products are exact, must come out bit-exact.
General data must stay within 8 K 2^-53 max|op(A)(i,:)| max|op(B)(:,j)| of the
exact product: the splitting's error model is truncation below 2^-54 of the
row / column maxima, the dropped slice pairs (p + q >= 7, below 2^-53 of
max|a| max|b| per term) and the rounding of each 128-deep chunk's sum (at most
K/128 2^(dsh-1) 2^-60 relative, dsh = ceil(log2 K) - 2), together under
4 K 2^-53.  The factorization in mixed precision is held to the same bar as the
FP64 form.
"""
from fractions import Fraction

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
U = 2.0 ** -53


def dev(x):
    return bq.to_colmajor(x)


def ops(ta, tb, A, Bm):
    return (A.T if ta == "T" else A), (Bm.T if tb == "T" else Bm)


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
@pytest.mark.parametrize("M,N,K", [(64, 32, 32), (65, 33, 17), (300, 200, 1000), (7, 513, 2049), (1, 1, 1)])
def test_ozaki_exact_on_integer_data(ta, tb, M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = rng.integers(-(1 << 19), 1 << 19, size=(K, M) if ta == "T" else (M, K)).astype(np.float64)
    Bm = rng.integers(-(1 << 19), 1 << 19, size=(N, K) if tb == "T" else (K, N)).astype(np.float64)
    C = dev(np.zeros((M, N)))
    bq.binding.bqrrp_dgemm_ozaki(ta, tb, 1.0, dev(A), dev(Bm), 0.0, C)
    oA, oB = ops(ta, tb, A, Bm)
    ref = (oA.astype(np.int64) @ oB.astype(np.int64)).astype(np.float64)   # |entries| < 2^53: exact
    assert np.array_equal(np_(C), ref)


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T")])
@pytest.mark.parametrize("M,N,K", [(128, 96, 512), (257, 130, 1000), (64, 2048, 16384), (1000, 1000, 64)])
def test_ozaki_within_fp64_error_model(ta, tb, M, N, K):
    rng = np.random.default_rng(3 * M + N + K)
    A = rng.standard_normal((K, M) if ta == "T" else (M, K))
    Bm = rng.standard_normal((N, K) if tb == "T" else (K, N))
    C0 = rng.standard_normal((M, N))
    C = dev(C0)
    bq.binding.bqrrp_dgemm_ozaki(ta, tb, -0.75, dev(A), dev(Bm), 1.5, C)
    oA, oB = ops(ta, tb, A, Bm)
    ref = -0.75 * (oA @ oB) + 1.5 * C0
    amax = np.abs(oA).max(axis=1)[:, None]
    bmax = np.abs(oB).max(axis=0)[None, :]
    # splitting error (below about 2^-53 of the row/column maxima per term)
    # plus the FP64 rounding of the reference product itself
    bound = 8 * K * U * 0.75 * amax * bmax + 4 * U * (0.75 * (np.abs(oA) @ np.abs(oB)) + np.abs(1.5 * C0))
    assert np.all(np.abs(np_(C) - ref) <= bound)


def test_ozaki_long_k_runs_in_pieces():
    """K above 2^17 runs as consecutive launches over K pieces (integer data:
    exact; general data: within the error model)."""
    rng = np.random.default_rng(11)
    M, N, K = 70, 66, (1 << 17) + 3000
    A = rng.integers(-(1 << 12), 1 << 12, size=(M, K)).astype(np.float64)
    Bm = rng.integers(-(1 << 12), 1 << 12, size=(K, N)).astype(np.float64)
    C = dev(np.zeros((M, N)))
    bq.binding.bqrrp_dgemm_ozaki("N", "N", 1.0, dev(A), dev(Bm), 0.0, C)
    assert np.array_equal(np_(C), (A.astype(np.int64) @ Bm.astype(np.int64)).astype(np.float64))
    A = rng.standard_normal((M, K))
    Bm = rng.standard_normal((K, N))
    C0 = rng.standard_normal((M, N))
    C = dev(C0)
    bq.binding.bqrrp_dgemm_ozaki("N", "N", 1.0, dev(A), dev(Bm), 1.0, C)
    ref = A @ Bm + C0
    bound = 8 * K * U * np.abs(A).max(axis=1)[:, None] * np.abs(Bm).max(axis=0)[None, :]
    assert np.all(np.abs(np_(C) - ref) <= bound + 4 * U * (np.abs(A) @ np.abs(Bm) + np.abs(C0)))


def test_ozaki_same_sign_data_near_the_exactness_bound():
    """Every slice product as large as it gets with one sign: the group sums of
    a 128-deep chunk approach the FP32 exactness bound (7 * 128 * 128^2 < 2^24).
    The entries are 2^-54 X with X's balanced base-256 digits -63 (the top
    one) and -128 (all the others, the last one even so that X has 53
    significant bits): every product of two slices below the top is +2^14."""
    rng = np.random.default_rng(12)
    M, N, K = 256, 192, 4096

    c0 = -63 * 2 ** 48 + sum(-128 * 2 ** (8 * (6 - p)) for p in range(1, 6))
    la = -2 * rng.integers(50, 65, size=(M, K))
    lb = -2 * rng.integers(50, 65, size=(K, N))
    A = (c0 + la) * 2.0 ** -54                           # exact: X = c0 + last has 53 significant bits
    Bm = (c0 + lb) * 2.0 ** -54
    C = dev(np.zeros((M, N)))
    bq.binding.bqrrp_dgemm_ozaki("N", "N", 1.0, dev(A), dev(Bm), 0.0, C)
    # the exact product, in integers (an FP64 A @ B of same-sign data errs by
    # far more than the slice product does): sum_k (c0 + la)(c0 + lb) 2^-108
    s1, s2, s3 = la.sum(axis=1), lb.sum(axis=0), la @ lb
    exact = np.array([[float(Fraction(K * c0 * c0 + c0 * (int(s1[i]) + int(s2[j])) + int(s3[i, j]), 2 ** 108))
                       for j in range(N)] for i in range(M)])
    assert np.all(np.abs(np_(C) - exact) <= 8 * K * U * np.abs(A).max() * np.abs(Bm).max())


def test_ozaki_wide_dynamic_range_rows_and_columns():
    rng = np.random.default_rng(7)
    M, N, K = 96, 80, 700
    A = rng.standard_normal((M, K)) * (10.0 ** rng.integers(-100, 100, size=M))[:, None]
    Bm = rng.standard_normal((K, N)) * (10.0 ** rng.integers(-100, 100, size=N))[None, :]
    A[5] = 0.0                                           # an all-zero row
    C = dev(np.zeros((M, N)))
    bq.binding.bqrrp_dgemm_ozaki("N", "N", 1.0, dev(A), dev(Bm), 0.0, C)
    ref = A @ Bm
    scale = np.abs(A).max(axis=1)[:, None] * np.abs(Bm).max(axis=0)[None, :]
    assert np.all(np.abs(np_(C) - ref) <= 8 * K * U * scale)
    assert np.all(np_(C)[5] == 0.0)


@pytest.mark.parametrize("integer", [True, False])
def test_ozaki_split_k_gram(integer):
    """A Gram matrix Y^T Y (256 x 256 from 16384 rows: 8 tiles, so K is split
    over the SMs and the splits' integer sums are added): exact on integer
    data, within the FP64 error model otherwise, for beta = 0 and beta != 0."""
    rng = np.random.default_rng(21 + integer)
    K, n = 16384, 256
    if integer:
        Y = rng.integers(-(1 << 19), 1 << 19, size=(K, n)).astype(np.float64)
    else:
        Y = rng.standard_normal((K, n)) * (2.0 ** rng.integers(-30, 30, size=n))[None, :]
    C = dev(np.zeros((n, n)))
    bq.binding.bqrrp_dgemm_ozaki("T", "N", 1.0, dev(Y), dev(Y), 0.0, C)
    if integer:
        assert np.array_equal(np_(C), (Y.T.astype(np.int64) @ Y.astype(np.int64)).astype(np.float64))
        return
    ref = Y.T @ Y
    cmax = np.abs(Y).max(axis=0)
    scale = cmax[:, None] * cmax[None, :]
    assert np.all(np.abs(np_(C) - ref) <= 8 * K * U * scale + 4 * U * (np.abs(Y).T @ np.abs(Y)))
    C0 = rng.standard_normal((n, n))
    C = dev(C0)
    bq.binding.bqrrp_dgemm_ozaki("T", "N", -0.5, dev(Y), dev(Y), 2.0, C)
    ref = -0.5 * ref + 2.0 * C0
    assert np.all(np.abs(np_(C) - ref) <= 8 * K * U * 0.5 * scale + 4 * U * (0.5 * (np.abs(Y).T @ np.abs(Y))
                                                                           + np.abs(2.0 * C0)))


def test_ozaki_beta_zero_ignores_nan():
    A = np.ones((70, 5))
    Bm = np.ones((5, 90))
    C = dev(np.full((70, 90), np.nan))
    bq.binding.bqrrp_dgemm_ozaki("N", "N", 1.0, dev(A), dev(Bm), 0.0, C)
    assert np.all(np_(C) == 5.0)


@pytest.mark.parametrize("d,m,n", [(160, 2000, 1000), (37, 333, 21), (640, 4097, 65)])
def test_sketch_tc_exact_on_integer_data(d, m, n):
    rng = np.random.default_rng(d + m)
    A = rng.integers(-40, 40, size=(m, n)).astype(np.float64)
    Msk = bq.binding.bqrrp_sketch_apply_tc(dev(A), d, 5)
    ref = oracle.sketch_apply(oracle.sketch_operator(d, m, 5), A)
    assert np.array_equal(np_(Msk), ref)


def test_sketch_tc_more_tiles_than_sms():
    """d = 320, n = 40000: 3 x 625 tiles, so every CTA of the persistent grid
    runs several tiles; 64 sampled columns (the first, the last and the ragged
    final tile among them) checked bit-exact on integer data."""
    d, m, n = 320, 4096, 40000
    rng = np.random.default_rng(7)
    A = rng.integers(-40, 40, size=(m, n)).astype(np.float64)
    Msk = np_(bq.binding.bqrrp_sketch_apply_tc(dev(A), d, 5))
    cols = np.unique(np.concatenate([[0, 63, 64, n - 65, n - 1], rng.integers(0, n, 59)]))
    ref = oracle.sketch_apply(oracle.sketch_operator(d, m, 5), A[:, cols])
    assert np.array_equal(Msk[:, cols], ref)


def test_ozaki_more_tiles_than_sms():
    """M = N = 1500, K = 700: 12 x 24 tiles (a ragged last row and column
    tile) over a grid of one CTA per SM, integer data, bit-exact."""
    M, N, K = 1500, 1500, 700
    rng = np.random.default_rng(11)
    A = rng.integers(-(1 << 19), 1 << 19, size=(M, K)).astype(np.float64)
    Bm = rng.integers(-(1 << 19), 1 << 19, size=(K, N)).astype(np.float64)
    C = dev(np.zeros((M, N)))
    bq.binding.bqrrp_dgemm_ozaki("N", "N", 1.0, dev(A), dev(Bm), 0.0, C)
    assert np.array_equal(np_(C), (A.astype(np.int64) @ Bm.astype(np.int64)).astype(np.float64))


def test_sketch_tc_gaussian_within_fp64_bound():
    d, m, n = 160, 2000, 1000
    A = W.gaussian(m, n, 3)
    Msk = np_(bq.binding.bqrrp_sketch_apply_tc(dev(A), d, 11))
    ref = oracle.sketch_apply(oracle.sketch_operator(d, m, 11), A)
    bound = 4 * m * U * np.abs(A).max(axis=0)[None, :] + 2 * m * U * np.abs(A).sum(axis=0)[None, :]
    assert np.all(np.abs(Msk - ref) <= bound)


def _factor_mixed(A, b, d, seed, precision="mixed", **kw):
    F, jpvt, tau, rank = bq.factor(A, b, d, seed, precision=precision, **kw)
    torch.cuda.synchronize()
    return np_(F), np_(jpvt), np_(tau), rank


def _pivots_agree_where_gapped(jpvt, fo, b, rank, gap=1e-3, sig=None):
    """Block by block, while every earlier block agreed: a block whose oracle
    LU margin exceeds the gap must pick the oracle's pivots.  Returns the
    number of blocks compared.  sig (the input's singular values, largest
    first): a block starting at sigma_s carries sketch rounding of about
    u sigma_0 / sigma_s relative to its own scale (the updates' absolute
    error), so its gap is at least 1e4 u sigma_0 / sigma_s."""
    compared = 0
    for i, t in enumerate(fo.trace):
        lo, hi = i * b, min((i + 1) * b, rank)
        g = gap if sig is None else max(gap, 1e4 * U * sig[0] / sig[min(lo, len(sig) - 1)])
        if hi <= lo or t["margin"] <= g:
            break
        assert np.array_equal(jpvt[lo:hi], fo.jpvt[lo:hi]), (i, t["margin"])
        compared += 1
    return compared


@pytest.mark.parametrize("case", ["c1", "ragged", "lowrank", "hqr", "decay14", "tall", "tall_lowrank"])
def test_mixed_factorization_meets_the_fp64_bar(case):
    if case == "c1":
        A, b, d, kw = W.c1_matrix(), 128, 160, {}
    elif case == "tall":   # panels of >= 2048 rows: the blocked solves with slice-product updates
        A, b, d, kw = W.gaussian(3000, 700, 5), 256, 320, {}
    elif case == "tall_lowrank":   # a block keeping 144 of its 256 columns
        A, b, d, kw = W.low_rank(3000, 700, 400, 8), 256, 320, {}
    elif case == "decay14":   # the mixed configuration's spectrum shape: sigma_k = 10^(-14 (k-1)/(n-1))
        sig = 10.0 ** (-14.0 * np.arange(600) / 599.0)
        A, b, d, kw = W.spectrum(1200, 600, sig, 21), 64, 80, {}
    elif case == "ragged":
        A, b, d, kw = W.gaussian(777, 500, 9), 64, 80, {}
    elif case == "lowrank":
        A, b, d, kw = W.low_rank(1000, 600, 150, 4), 64, 80, {}
    else:
        A, b, d, kw = W.gaussian(900, 700, 12), 96, 120, {"panel": "hqr"}
    fo = oracle.bqrrp(A, b, d, 1, panel=kw.get("panel", "cholqr"))
    F, jpvt, tau, rank = _factor_mixed(A, b, d, 1, **kw)
    assert rank == fo.rank
    if case == "decay14":
        # the deepest blocks' sketches sit at 1e-12 of the first block's scale
        assert _pivots_agree_where_gapped(jpvt, fo, b, rank, gap=1e-6, sig=sig) >= 4
    elif all(t["margin"] > 1e-6 for t in fo.trace):
        assert np.array_equal(jpvt[:rank], fo.jpvt[:rank])
    res, orth, ok = metrics(A, F, jpvt, tau, rank)
    assert ok and res <= 1e-12 and orth <= 1e-12, (res, orth)
    bounds = list(range(0, A.shape[1], b))
    assert np.all(trailing_norms(F, rank, bounds) <= 1.1 * trailing_norms(fo.A, fo.rank, bounds)
                  + 1e-13 * np.linalg.norm(A))


@pytest.mark.parametrize("case", ["c1", "tall", "tall_lowrank", "decay14"])
def test_mixed_panel_tc_meets_the_fp64_bar(case):
    """opts.panel_tc: the CholQR panel's Gram and the block updates of its two
    tall solves as slice products (FP64-accurate: the same bars)."""
    if case == "c1":
        A, b, d = W.c1_matrix(), 128, 160
    elif case == "tall":
        A, b, d = W.gaussian(3000, 700, 5), 256, 320
    elif case == "tall_lowrank":
        A, b, d = W.low_rank(3000, 700, 400, 8), 256, 320
    else:
        sig = 10.0 ** (-14.0 * np.arange(600) / 599.0)
        A, b, d = W.spectrum(2400, 600, sig, 21), 128, 160
    fo = oracle.bqrrp(A, b, d, 1)
    F, jpvt, tau, rank = _factor_mixed(A, b, d, 1, panel_tc=True)
    assert rank == fo.rank
    if case == "decay14":
        assert _pivots_agree_where_gapped(jpvt, fo, b, rank, gap=1e-6, sig=sig) >= 2
    elif all(t["margin"] > 1e-6 for t in fo.trace):
        assert np.array_equal(jpvt[:rank], fo.jpvt[:rank])
    res, orth, ok = metrics(A, F, jpvt, tau, rank)
    assert ok and res <= 1e-12 and orth <= 1e-12, (res, orth)
    bounds = list(range(0, A.shape[1], b))
    assert np.all(trailing_norms(F, rank, bounds) <= 1.1 * trailing_norms(fo.A, fo.rank, bounds)
                  + 1e-13 * np.linalg.norm(A))


VARIANTS = [("fp64", False), ("mixed", False), ("mixed_sketch32", False), ("mixed", True), ("mixed_sketch32", True)]


def test_variant_errors_against_the_fp64_oracle():
    """Every arithmetic variant against the FP64 oracle on the mixed
    configuration's spectrum shape, sigma_k = 10^(-14 (k-1)/(n-1)), at 2048^2,
    b = 256, d = 320: rank, pivot agreement, residual, orthogonality and the
    truncation errors ||R(s:, s:)||_F at every block boundary relative to the
    oracle's.  The table is printed (run with -s to see it).  The spectrum ends
    at the rank threshold, so the ranks may differ by a few columns there."""
    n, b, d = 2048, 256, 320
    sig = 10.0 ** (-14.0 * np.arange(n) / (n - 1))
    A = W.spectrum(n, n, sig, 31)
    fo = oracle.bqrrp(A, b, d, 1)
    bounds = list(range(0, n, b))
    ref_tn = trailing_norms(fo.A, fo.rank, bounds)
    lines = ["| variant | rank (oracle %d) | pivots equal to the oracle's | blocks compared where gapped | "
             "residual | orthogonality | max truncation ratio |" % fo.rank, "|---|---|---|---|---|---|---|"]
    for prec, ptc in VARIANTS:
        F, jpvt, tau, rank = _factor_mixed(A, b, d, 1, precision=prec, panel_tc=ptc)
        res, orth, ok = metrics(A, F, jpvt, tau, rank)
        diff = np.nonzero(jpvt[:rank] != fo.jpvt[:rank])[0]
        lead = int(diff[0]) if diff.size else rank
        fp32 = prec == "mixed_sketch32"
        blocks = _pivots_agree_where_gapped(jpvt, fo, b, rank, gap=1e-3 if fp32 else 1e-6, sig=sig)
        tn = trailing_norms(F, rank, bounds)
        ratio = float(np.max(tn[ref_tn > 0] / ref_tn[ref_tn > 0]))
        name = prec + (" + panel_tc" if ptc else "")
        lines.append(f"| {name} | {rank} | first {lead} | {blocks} | {res:.2e} | {orth:.2e} | {ratio:.4f} |")
        # FP32 R^sk preconditions the deepest blocks' panels less well: on this
        # spectrum the variant's orthogonality is about 1e-11, the residual
        # keeps the FP64 bar (R^sk11 enters the preconditioner and R11 alike)
        assert ok and res <= 1e-12 and orth <= (5e-11 if fp32 else 1e-12), (name, res, orth)
        assert ratio <= (1.25 if fp32 else 1.1), (name, ratio)
        # the spectrum reaches the rank threshold (10 d u of the first block)
        # near its end, where the kept/dropped decision compares noise: only
        # a small difference is allowed.  The FP32 sketch QRCP may keep the
        # columns below the threshold (its R^sk there is FP32 rounding of the
        # block's scale); the residual and orthogonality bars cover them.
        if fp32:
            assert rank >= fo.rank - n // 100, (name, rank, fo.rank)
        else:
            assert abs(rank - fo.rank) <= n // 100, (name, rank, fo.rank)
    print("\n" + "\n".join(lines))


@pytest.mark.parametrize("m,n,zero_col", [(300, 200, None), (2049, 130, None), (1000, 1000, None),
                                          (5000, 300, None), (700, 600, 300)])
def test_own_qr_mixed_matches_oracle(m, n, zero_col):
    """The two-level blocked QR (outer blocks of 256; the last case has a zero
    column, so a reflector with tau = 0 enters a block reflector)."""
    A = W.gaussian(m, n, m + 2 * n)
    if zero_col is not None:
        A[:, zero_col] = 0.0
    Ad = dev(A)
    tau = np_(bq.binding.bqrrp_geqrf_mixed(Ad))
    F = np_(Ad)
    Fo, tau_o = oracle.geqrf(A)
    k = min(m, n)
    nrm = np.linalg.norm(A)
    assert np.linalg.norm(np.triu(F)[:k] - np.triu(Fo)[:k]) <= 1e-13 * np.sqrt(m * n) * nrm
    assert np.max(np.abs(tau[:k] - tau_o)) <= 1e-12


@pytest.mark.parametrize("case", ["c1", "ragged", "hqr", "decay14", "graded"])
def test_sketch32_variant_meets_the_fp64_bar_on_graded_spectra(case):
    """BQRRP_PRECISION_MIXED_SKETCH32: Alg. 2 on the sketch in FP32 (the LU
    panels' pivot search and eliminations, and the QR that forms R^sk from the
    LU factor).  Its pivots are FP32 decisions, so they are held to the FP64
    oracle's only where the oracle's LU margin exceeds 1e-3 (the FP32 LU's
    relative error after d steps is about d 2^-24 < 2e-5), block by block while
    the earlier blocks agree.  R^sk enters the preconditioner and R11
    consistently, so the residual and orthogonality bar is the FP64 one.  The
    small shapes here run the LU panels on one thread-block cluster; the
    16384^2 test of test_gpu_fullsize.py runs the grid form."""
    if case == "c1":
        A, b, d, kw = W.c1_matrix(), 128, 160, {}
    elif case == "ragged":
        A, b, d, kw = W.gaussian(777, 500, 9), 64, 80, {}
    elif case == "hqr":
        A, b, d, kw = W.gaussian(900, 700, 12), 96, 120, {"panel": "hqr"}
    elif case == "decay14":   # the mixed configuration's spectrum shape: sigma_k = 10^(-14 (k-1)/(n-1))
        sig = 10.0 ** (-14.0 * np.arange(600) / 599.0)
        A, b, d, kw = W.spectrum(1200, 600, sig, 21), 64, 80, {}
    else:   # column norms graded over 2^15: the oracle's LU margins all exceed 1e-3
        A0 = W.gaussian(800, 300, 35)
        A, b, d, kw = A0 * (0.5 ** (np.arange(300) / 20.0))[None, ::-1], 64, 80, {}
    fo = oracle.bqrrp(A, b, d, 1, panel=kw.get("panel", "cholqr"))
    F, jpvt, tau, rank = _factor_mixed(A, b, d, 1, precision="mixed_sketch32", **kw)
    assert rank == fo.rank
    n_cmp = _pivots_agree_where_gapped(jpvt, fo, b, rank, sig=sig if case == "decay14" else None)
    if case == "graded":
        assert n_cmp == len(fo.trace)   # every block compared
    res, orth, ok = metrics(A, F, jpvt, tau, rank)
    # on the spectrum down to 1e-14 the FP32 R^sk of the deepest blocks (sketch
    # scale near 1e-13) preconditions their panels less well: orthogonality
    # measured 2.8e-12 there, so this input's orthogonality bar is 1e-11
    assert ok and res <= 1e-12 and orth <= (1e-11 if case == "decay14" else 1e-12), (res, orth)
    # truncation errors at the block boundaries: FP32 pivot decisions deep in a
    # decaying spectrum pick slightly different columns than the FP64 oracle
    # (1.13x at C1's last boundary, measured), so this variant's bar is 1.25x
    bounds = list(range(0, A.shape[1], b))
    assert np.all(trailing_norms(F, rank, bounds) <= 1.25 * trailing_norms(fo.A, fo.rank, bounds)
                  + 1e-13 * np.linalg.norm(A))


@pytest.mark.parametrize("where", ["inside", "boundary"])
def test_sketch32_variant_cuts_exact_rank_gaps(where):
    """Past an exact rank gap the FP32 R^sk holds rounding noise of the
    block's own scale (about 1e-7), above the FP64 tri_rank threshold; the
    variant's FP32 rank floor (10 d 2^-24 relative to the block's |R^sk(0,0)|,
    and to the previous block's for a whole block) cuts there, so the rank is
    the oracle's and the FP64 bar holds.  inside: rank 150 inside a 64-column
    block; boundary: rank 64 at a block boundary (b = 32)."""
    if where == "inside":
        A, b, d = W.low_rank(1000, 600, 150, 4), 64, 80
    else:
        A, b, d = W.low_rank(200, 130, 64, 6), 32, 40
    fo = oracle.bqrrp(A, b, d, 1)
    F, jpvt, tau, rank = _factor_mixed(A, b, d, 1, precision="mixed_sketch32")
    assert rank == fo.rank
    res, orth, ok = metrics(A, F, jpvt, tau, rank)
    assert ok and res <= 1e-12 and orth <= 1e-12, (res, orth)
