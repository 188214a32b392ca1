"""The request loop on the GPU: every request's result equals the direct call
that computes it alone (a batch of one for the small lane, bqrrp_factor for
the large lane) bit for bit, meets the oracle's bar, and the device pool never
holds more request state than its budget."""
import numpy as np
import pytest
import torch

import oracle
import paper_2507_00976_b300 as bq
from checks import metrics
from gpu_util import np_
from paper_2507_00976_b300 import binding as B
from paper_2507_00976_b300 import workloads as W

pytestmark = pytest.mark.gpu
MiB = 1 << 20
TOL = 1e-8


def make_requests():
    rng = np.random.default_rng(5)
    shapes = [(256, 256, 32, 40), (300, 200, 64, 80), (256, 256, 64, 80), (700, 500, 64, 80),
              (1024, 300, 32, 40), (513, 257, 32, 40)]
    reqs = []
    for i in range(14):
        m, n, b, d = shapes[i % len(shapes)]
        decay = 10.0 ** rng.uniform(-14, -4)
        sig = decay ** (np.arange(n) / max(n - 1, 1))
        A = np.asfortranarray(W.spectrum(m, n, sig, 40 + i))
        reqs.append(dict(id=i, m=m, n=n, b=b, d=d, seed=100 + i, A=A))
    return reqs


@pytest.mark.parametrize("mixed", [False, True])
def test_server_matches_direct_calls_and_oracle(mixed):
    """mixed: the large lane factors with BQRRP_PRECISION_MIXED (BQRRP_SERVER_MIXED)."""
    reqs = make_requests()
    S = B.Server(2048 * MiB, 256 * MiB, trunc_tol=TOL, small_max_elems=1 << 17, mixed=mixed)
    outs = {}
    order = np.random.default_rng(1).permutation(len(reqs))
    for k in order:
        r = reqs[k]
        Ao = np.zeros((r["m"], r["n"]), order="F")
        jo = np.zeros(r["n"], dtype=np.int64)
        to = np.zeros(r["n"])
        outs[r["id"]] = (Ao, jo, to)
        S.submit(r["id"], r["m"], r["n"], r["b"], r["d"], r["seed"], r["A"], Ao, jo, to)
    S.drain()
    done = {c["id"]: c for c in S.poll(64)}
    st = S.stats()
    err = S.last_error()
    S.close()
    assert err == ""
    assert len(done) == len(reqs) and st["peak_request_bytes"] <= st["request_arena_bytes"]
    for r in reqs:
        c = done[r["id"]]
        Ao, jo, to = outs[r["id"]]
        assert c["status"] == 0
        small = r["m"] * r["n"] <= (1 << 17)
        assert c["lane"] == (0 if small else 1)
        if small:
            F, J, T, rk, tr, inf = B.factor_batched(r["A"].ravel(order="F"), np.array([r["m"]]), np.array([r["n"]]),
                                                    np.array([r["b"]]), np.array([r["d"]]),
                                                    np.array([r["seed"]], dtype=np.uint64), TOL)
            assert np.array_equal(Ao.ravel(order="F"), np_(F))
            assert np.array_equal(jo, np_(J)) and np.array_equal(to, np_(T))
            assert c["rank"] == int(np_(rk)[0]) and c["trunc_rank"] == int(np_(tr)[0])
        else:
            F, J, T, rk = bq.factor(r["A"], r["b"], r["d"], r["seed"], precision="mixed" if mixed else "fp64")
            torch.cuda.synchronize()
            assert np.array_equal(Ao, np_(F)) and np.array_equal(jo, np_(J)) and np.array_equal(to, np_(T))
            assert c["rank"] == rk
            want = oracle.trunc_rank(Ao, rk, np.linalg.norm(r["A"]), TOL)
            if c["trunc_rank"] != want:
                R = np.triu(Ao)[:rk]
                i = min(want, c["trunc_rank"])
                assert abs(np.linalg.norm(R[i:, i:]) - TOL * np.linalg.norm(r["A"])) <= 1e-9 * TOL * np.linalg.norm(r["A"])
    for r in reqs[:5]:   # both lanes
        Ao, jo, to = outs[r["id"]]
        res, orth, ok = metrics(r["A"], Ao, jo, to, done[r["id"]]["rank"])
        assert ok and res <= 1e-12 and orth <= 1e-12


def test_server_small_budget_admits_in_turn():
    reqs = make_requests()[:8]
    one = max(r["m"] * r["n"] * 8 for r in reqs) + 64 * 1024
    S = B.Server(2 * one + 256 * MiB, 256 * MiB, trunc_tol=TOL, small_max_elems=1 << 17)
    for r in reqs:
        S.submit(r["id"], r["m"], r["n"], r["b"], r["d"], r["seed"], r["A"])
    S.drain()
    done = S.poll(64)
    st = S.stats()
    S.close()
    assert len(done) == 8 and all(c["status"] == 0 for c in done)
    assert st["peak_request_bytes"] <= st["request_arena_bytes"] <= 2 * one + 256
