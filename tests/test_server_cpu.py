"""Host-side tests of the request loop (bqrrp_server_*) in dry-run mode: the
GPU work is replaced by a modelled service time, so admission by the HBM
budget, lane routing, continuous batching and the completion records are
checked without a GPU."""
import time

import pytest

from paper_2507_00976_b300 import binding as B

MiB = 1 << 20


def state_bytes(m, n):
    up = lambda x: (x + 255) // 256 * 256
    return up(m * n * 8) + 2 * up(n * 8)


def collect(S, count, timeout=30.0):
    out, t0 = [], time.time()
    while len(out) < count and time.time() - t0 < timeout:
        out += S.poll(256, 0.05)
    return out


def test_every_request_completes_with_ordered_timestamps():
    S = B.Server(512 * MiB, 16 * MiB, dry=True, dry_gflops=200.0)
    shapes = [(256, 256), (1024, 512), (2048, 1024), (256, 256), (4096, 2048)]
    for i, (m, n) in enumerate(shapes * 4):
        S.submit(i, m, n, 32, 40, i)
    S.drain()
    done = collect(S, 20)
    assert sorted(c["id"] for c in done) == list(range(20))
    for c in done:
        assert c["status"] == 0
        assert c["t_submit"] <= c["t_admit"] <= c["t_start"] <= c["t_done"]
    st = S.stats()
    assert st["submitted"] == st["completed"] == 20 and st["in_use_bytes"] == 0
    S.close()


def test_lane_routing_by_size():
    S = B.Server(512 * MiB, 16 * MiB, small_max_elems=1 << 20, dry=True)
    S.submit(1, 1024, 1024, 32, 40, 0)        # 2^20 elements: small lane
    S.submit(2, 1025, 1024, 32, 40, 0)        # one more row: large lane
    S.drain()
    lanes = {c["id"]: c["lane"] for c in collect(S, 2)}
    assert lanes == {1: 0, 2: 1}
    S.close()


def test_admission_never_exceeds_the_budget():
    one = state_bytes(1024, 512)
    arena = 3 * one + 1000                     # room for three such requests at a time
    S = B.Server(arena + 16 * MiB, 16 * MiB, small_max_elems=0, dry=True, dry_gflops=50.0)
    assert S.stats()["request_arena_bytes"] >= 3 * one
    for i in range(12):
        S.submit(i, 1024, 512, 64, 80, i)
    S.drain()
    st = S.stats()
    assert st["completed"] == 12
    assert st["peak_request_bytes"] <= st["request_arena_bytes"]
    assert st["peak_request_bytes"] <= 3 * state_bytes(1024, 512) + 3 * 256
    # large lane: two workers, each admitting one request at a time, first come
    # first served -- admissions follow submission order and at most two large
    # requests run at once
    done = collect(S, 12)
    by_admit = [c["id"] for c in sorted(done, key=lambda c: c["t_admit"])]
    assert by_admit == sorted(by_admit)
    events = sorted([(c["t_start"], 1) for c in done] + [(c["t_done"], -1) for c in done])
    running, most = 0, 0
    for _, step in events:
        running += step
        most = max(most, running)
    assert most <= 2
    S.close()


def test_continuous_batching_groups_small_requests():
    S = B.Server(1 << 30, 16 * MiB, dry=True, dry_gflops=20.0)
    # a long large request first; the small ones arriving meanwhile are batched together
    S.submit(0, 4096, 2048, 256, 320, 0)
    time.sleep(0.01)
    for i in range(1, 41):
        S.submit(i, 256, 256, 64, 80, i)
    S.drain()
    done = collect(S, 41)
    st = S.stats()
    assert st["completed"] == 41 and st["large_runs"] == 1
    assert st["batches"] < 10 and st["max_batch"] >= 10
    small = [c for c in done if c["lane"] == 0]
    assert len(small) == 40
    S.close()


def test_bad_and_oversize_requests_are_refused():
    S = B.Server(64 * MiB, 16 * MiB, dry=True)
    with pytest.raises(B.BqrrpError) as e:
        S.submit(1, 100, 200, 16, 20, 0)       # m < n
    assert e.value.code == -2
    with pytest.raises(B.BqrrpError) as e:
        S.submit(2, 200, 100, 200, 250, 0)     # small lane needs b <= 128
    assert e.value.code == -2
    with pytest.raises(B.BqrrpError) as e:
        S.submit(3, 8192, 4096, 512, 640, 0)   # 268 MB of state, a 48 MB arena
    assert e.value.code == B.ENOMEM
    S.submit(4, 300, 200, 32, 40, 0)
    S.drain()
    assert [c["id"] for c in collect(S, 1)] == [4]
    S.close()


def test_server_arguments_checked():
    with pytest.raises(B.BqrrpError):
        B.Server(1 * MiB, 1 * MiB, dry=True)   # budget must exceed the workspace arena
