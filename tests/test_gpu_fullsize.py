"""The bench's configuration at full size: m = n = 16384, b = 256, d = 320,
iid N(0,1), dense Philox +-1 sketch, CholQR panel, in the launch configuration
bench.py times (bqrrp_factor on device buffers), for the FP64 and the mixed
form.  The oracle cannot factor 16384^2 in a test's time, so it is held to:
  - properties that hold at any size: full rank, R upper triangular,
    ||AP - QR||_F / ||A||_F <= 1e-12 and ||Q^T Q - I||_F <= 1e-12, with Q formed
    on the test side by a library routine (torch householder_product);
  - a sampled oracle output: the first block's b pivots, recomputed on the host
    from the oracle's own sketch operator (a library matmul for S A) and the
    oracle's LU with partial pivoting, compared where every LU step is gapped.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2507_00976_b300 as bq
from paper_2507_00976_b300 import workloads as W

pytestmark = pytest.mark.gpu

M = N = 16384
BLK, D, SEED = 256, 320, 3


@pytest.fixture(scope="module")
def problem():
    A = W.gaussian(M, N, 11)
    S = oracle.sketch_operator(D, M, SEED)              # the oracle's Philox +-1 operator
    Msk = S @ A                                          # library product, host side
    _, ipiv, margin = oracle.lupp(Msk.T.copy())
    J0 = oracle.piv_transform(N, ipiv)[:BLK]             # the first block's pivots (0-based)
    return A, J0, margin


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_factorization(problem, precision):
    A, J0, margin = problem
    Ad = bq.to_colmajor(A)
    F, jpvt, tau, rank = bq.factor(Ad, BLK, D, SEED, precision=precision)
    torch.cuda.synchronize()
    assert rank == N
    j = jpvt.to(torch.int64) - 1
    assert torch.equal(torch.sort(j).values, torch.arange(N, device=j.device))
    assert margin > 1e-9            # every LU step of this input is gapped (2.4e-4)
    assert np.array_equal(j[:BLK].cpu().numpy(), J0)
    R = torch.triu(F)
    Q = torch.linalg.householder_product(F, tau[:N])
    del F
    nA = torch.linalg.norm(Ad)
    res = torch.linalg.norm(Ad[:, j] - Q @ R) / nA
    del R
    QtQ = Q.T @ Q
    QtQ.diagonal().sub_(1.0)
    orth = torch.linalg.norm(QtQ)
    assert res.item() <= 1e-12 and orth.item() <= 1e-12, (precision, res.item(), orth.item())
