"""The tensor-core slice GEMM's schedule (csrc/tc_schedule.cuh), simulated on
the CPU before any GPU run: the header's role loops, compiled with g++, drive
simulated mbarriers (hardware parity-wait rule) in random interleavings.  The
simulator (tests/sim/tc_schedule_sim.cpp) fails on a deadlock, on a wait that
could confuse two barrier phases, on an MMA reading the wrong A plane or B
half, on a slot refilled before its uses are released, on an MMA into busy
accumulators, and on an accumulator read that does not see exactly its
chunk's k blocks."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "sim", "tc_schedule_sim.cpp")


@pytest.fixture(scope="module")
def sim(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("tcsim") / "tc_schedule_sim")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-o", exe, SRC])
    return exe


CASES = [
    # SA, KB, CL, mt, nct, grid
    (7, 1, 2, 3, 2, 2),        # one k block per tile: both halves end at once
    (7, 2, 2, 2, 3, 4),
    (7, 3, 2, 5, 2, 3),        # odd k blocks: the early half keeps its role
    (7, 4, 2, 4, 4, 5),        # even k blocks: the roles alternate between tiles
    (7, 9, 2, 70, 2, 7),       # more row tiles than one raster group
    (7, 512, 2, 2, 1, 2),      # long K (W = Y^T C): many chunks per tile
    (1, 5, 2048, 3, 3, 2),     # the sketch: one A plane, one chunk per tile
    (1, 40, 16, 2, 2, 3),      # the sketch with several chunks per tile
    (1, 1, 2048, 1, 1, 1),
]


@pytest.mark.parametrize("case", CASES)
def test_schedule_simulation(sim, case):
    for seed in (1, 2, 3):
        out = subprocess.run([sim] + [str(x) for x in case] + [str(seed)], capture_output=True, text=True,
                             timeout=300)
        assert out.returncode == 0 and out.stdout.strip() == "ok", (case, seed, out.stderr[-2000:])
