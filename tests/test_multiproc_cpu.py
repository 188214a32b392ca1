"""The N > 1 bench path on CPU: world size 2 over gloo.  One factorization
does not shard, so N GPUs run N replicas; what crosses ranks is only the
max-over-ranks timing and the whole-job throughput.  The ranks here run the
CPU oracle on their own (distinct) seeded matrices, as replicas do."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    import bench
    import oracle
    from checks import metrics
    from paper_2507_00976_b300 import workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seed = bench.rank_seed(2, rank)
    A = W.gaussian(120, 80, seed)
    f = oracle.bqrrp(A, 16, 20, 1)
    res, orth, ok = metrics(A, f.A, f.jpvt, f.tau, f.rank)
    local_ms = 100.0 * (rank + 1)               # a known, rank-dependent time
    mx = bench.max_over_ranks(local_ms, dist, "cpu")
    value = bench.job_gflops(bench.canonical_flops(120, 80), 3, world, mx)
    dist.barrier()
    dist.destroy_process_group()
    out[rank] = (mx, value, float(res), float(orth), bool(ok), seed, float(np.abs(A).sum()))


def test_replicas_aggregate_over_gloo_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()   # no fork of this (possibly multi-threaded) process
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    r0, r1 = out[0], out[1]
    assert r0[0] == r1[0] == 200.0                        # max over ranks
    expect = (2 * 120 * 80 ** 2 - 2 * 80 ** 3 / 3) * 3 * world / 0.2 / 1e9
    assert abs(r0[1] - expect) < 1e-9 * expect and r0[1] == r1[1]
    assert r0[5] != r1[5] and r0[6] != r1[6]              # independent problems per rank
    for r in (r0, r1):
        assert r[4] and r[2] < 1e-13 and r[3] < 1e-13
