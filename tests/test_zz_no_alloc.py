"""bqrrp_sketch_apply_sparse_noalloc: the allocation-free form of the
sparse-sign sketch, for callers that cannot allocate device memory or pass a
workspace.  Its output must match the workspace-based entry point
bqrrp_sketch_apply (sparse kind) on consecutive calls -- the second call has a
different shape and seed, so leftovers in the shared fixed scratch would show.
Collected last on purpose (file name) so that a stop-at-first-failure run has
already run everything else."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2507_00976_b300 as bq
from gpu_util import np_
from paper_2507_00976_b300 import binding as B
from paper_2507_00976_b300 import workloads as W

U = 2.0 ** -53


def test_noalloc_rejects_oversize_shapes_before_touching_the_device():
    L = B.lib()
    rc = L.bqrrp_sketch_apply_sparse_noalloc(5000, 100, 10, None, 100, 1, 8, None, 5000, None)
    assert rc == B.EUNSUPPORTED and "4096" in B.last_error()
    rc = L.bqrrp_sketch_apply_sparse_noalloc(4097, 100, 10, None, 100, 1, 8, None, 4097, None)
    assert rc == B.EUNSUPPORTED and "4096" in B.last_error()
    rc = L.bqrrp_sketch_apply_sparse_noalloc(64, 65537, 10, None, 65537, 1, 8, None, 64, None)
    assert rc == B.EUNSUPPORTED and "524288" in B.last_error()
    rc = L.bqrrp_sketch_apply_sparse_noalloc(64, 70000, 10, None, 70000, 1, 8, None, 64, None)
    assert rc == B.EUNSUPPORTED and "524288" in B.last_error()
    assert L.bqrrp_sketch_apply_sparse_noalloc(64, 100, 10, None, 100, 1, 65, None, 64, None) == -7


@pytest.mark.gpu
def test_noalloc_matches_workspace_entry_point_on_consecutive_calls():
    cases = [(640, 16384, 300, 11, W.gaussian(16384, 300, 1)),
             (160, 2000, 257, 3, np.random.default_rng(2).integers(-30, 30, size=(2000, 257)).astype(np.float64)),
             # the stated maxima: d = 4096 sketch rows (two row tiles of the kernel) and
             # m * nnz = 2^19 operator entries
             (4096, 65536, 40, 5, np.random.default_rng(3).integers(-30, 30, size=(65536, 40)).astype(np.float64)),
             # small d: every CSR row holds about m * nnz / d = 2^16 entries
             (8, 65536, 24, 7, W.gaussian(65536, 24, 4))]
    for d, m, n, seed, A in cases:
        Ad = bq.to_colmajor(A)
        ref = np_(bq.bqrrp_sketch_apply(Ad, d, seed, kind=B.SKETCH_SPARSE, nnz=8))
        got = np_(B.bqrrp_sketch_apply_sparse_noalloc(Ad, d, seed, nnz=8))
        bound = 2 * m * U * np.abs(A).sum(axis=0)[None, :]
        assert np.all(np.abs(got - ref) <= bound)
        if np.all(A == np.round(A)):
            # integer data: every partial sum is exact, so the two entry points agree
            # bit for bit, and both equal the oracle (checked where its dense d x m
            # operator is small)
            assert np.array_equal(got, ref)
            if d * m <= 1 << 24:
                assert np.array_equal(got, oracle.sketch_apply(oracle.sketch_operator(d, m, seed, kind=1, nnz=8), A))
