"""The bench's reference arm (the CPU oracle on host cores) keeps the JSON
contract of the single-matrix line: the same metric, unit and config as the
GPU arm, plus the reference arm's own keys."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "GFLOP/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1 and d["value"] > 0
    assert d["config"]["workload"].startswith("FP64 BQRRP m=32768 n=32768 b=256 d=320")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_config_names_the_schedule_and_host_lapack_context_runs():
    import argparse
    import sys as _sys
    _sys.path.insert(0, ROOT)
    import bench
    a = argparse.Namespace(m=16384, n=16384, b=256, d=320, family="gaussian", sketch="dense", panel="cholqr",
                           precision="fp64", seed=2, schedule="overlap", workload="single")
    assert bench.config(a, 1)["schedule"] == "overlap"
    a.panel = "hqr"
    assert bench.config(a, 1)["schedule"] == "serial"           # the Householder panel runs serially
    a.panel, a.precision = "cholqr", "mixed"
    assert bench.config(a, 1)["schedule"] == "serial"           # so does the mixed form
    ctx = bench.host_lapack_context(a, s=256)
    assert ctx["geqp3_gflops"] > 0 and ctx["geqrf_gflops"] > 0 and ctx["size"] == "256x256"


def test_cpu_plan_measures_c1_on_one_and_all_cores_and_labels_extrapolations():
    import argparse
    import sys as _sys
    _sys.path.insert(0, ROOT)
    import bench
    a = argparse.Namespace(m=32768, n=32768, b=256, d=320, family="gaussian", sketch="dense", panel="cholqr",
                           precision="fp64", seed=2, schedule="overlap", workload="single")
    cb = bench.cpu_plan(a, budget_s=0.0)        # no budget: C1 twice and the 4096^2 run only
    sizes = [(r["size"], r["threads"]) for r in cb["runs"]]
    _, ncpu = bench.host_cpu()
    assert sizes == [("2000x1000 (C1)", 1), ("2000x1000 (C1)", ncpu), ("4096x4096", ncpu)]
    assert cb["kind"] == "oracle" and cb["cores"] == ncpu and cb["value"] == cb["runs"][-1]["gflops"]
    assert set(cb["extrapolated"]) == {"16384x16384", "32768x32768"}
    for e in cb["extrapolated"].values():
        assert e["how"].startswith("extrapolated") and e["from"] == "4096x4096"
