#!/usr/bin/env python
"""Benchmark: FP64 BQRRP on B300, canonical GFLOP/s (2mn^2 - 2n^3/3 per solve,
the GEQRF count the paper uses, Sec. 1.4) next to the library's own unpivoted
blocked Householder QR on the same input, with p50/p99 solve latency.

Default workload: one m = n = 32768 matrix with iid N(0,1) entries (the
paper's performance matrices, at the configuration's largest size), block
b = 256 (the fastest block size of the configuration's sweep on this part),
sketch d = ceil(1.25 b) = 320 rows of a Philox +-1 operator, CholQR panel,
FP64, overlap schedule.  One step = one complete bqrrp_factor call on a fresh
copy of the input already resident in HBM.  vs_baseline is the metric's own
comparison: BQRRP GFLOP/s over the library's own unpivoted QR GFLOP/s on the
same input (Sec. 7.2 compares BQRRP with unpivoted QR on the GPU).

  python bench.py [--gpus N --steps K --warmup W] [--n 16384 --b 1024 ...]
  python bench.py --impl reference ...   # the CPU oracle, timed on the host

Multi-GPU: the factorization of one matrix does not shard (every block needs
a global pivot choice), so N GPUs run N independent replicas ("replicas
only"); value = total canonical FLOPs of all ranks / max over ranks of the
timed region.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BQRRP GFLOP/s (2mn²−2n³/3) vs own unpivoted QR on 1 B300; p50/p99 solve latency"
SM_COUNT = 148
SM_MAX_MHZ = 2032.0
# FP64: 2 DFMA per clock per SM (the measured DFMA rate is 1.82-1.97 per clock
# per SM; tcgen05 has no f64 kind), 2 FLOP per DFMA.
FP64_PEAK_TFLOPS = SM_COUNT * 2 * 2 * SM_MAX_MHZ * 1e6 / 1e12
# the FP64-accurate tensor-core product runs 28 bf16 slice products per FP64
# product (seven balanced 8-bit slices per operand, the pairs with p + q <= 6)
OZ_PRODUCTS = 28


def bf16_peak():
    """Measured cuBLAS bf16 throughput of this part (sustained: the slice GEMMs run
    inside a seconds-long factorization) and where the number came from."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["bf16_tflops_sustained"]), "measured (MEASURED_PEAKS.json bf16_tflops_sustained)"
    except (OSError, KeyError, ValueError):
        return 1400.0, "fallback (sustained bf16 of an earlier B300 measurement)"


def mixed_roofline(fp64eq_tflops):
    """Tensor roofline of the slice GEMM: bf16 work = 28 x the FP64-equivalent rate."""
    if not fp64eq_tflops:
        return None
    peak, src = bf16_peak()
    ach = OZ_PRODUCTS * fp64eq_tflops
    return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": None, "kernel": ("ozaki_tc_kernel (bf16 slice products: persistent 128x64 tiles, tcgen05.mma kind::f16 "
                                        "M=128 N<=256 stacked planes, TMA-fed 128B-swizzled smem, FP32 group "
                                        "accumulators in all 512 TMEM columns, epilogue of one half overlapping the "
                                        "other half's MMAs)"),
            "fp64_equivalent_tflops": fp64eq_tflops, "peak_source": src,
            "counting": "28 bf16 slice products per FP64 product, all of them formed (no discarded products)"}


# DRAM traffic of one trailing C -= Y.W2 launch (dgemm_kernel<0,0>, rows k.. of the
# block), from an ncu capture of the 8192^2, b = 256 solve (one launch at
# s = 2304: C 5888 x 5888, K = 256): dram__bytes_read.sum + dram__bytes_write.sum
# = 302,608,896 + 220,156,160 bytes against 578.8 MB of operand bytes (C read and
# written once, Y and W2 read once).  The traffic follows the operand bytes, so a
# launch of another size is scaled by them.
TRAILING_CAPTURE = {"rows": 5888, "cols": 5888, "k": 256, "dram_bytes": 302608896 + 220156160}


def gemm_operand_bytes(rows, cols, k):
    """C (rows x cols) read and written once, Y (rows x k) and W2 (k x cols) read once, FP64."""
    return 8.0 * (2 * rows * cols + rows * k + k * cols)


def trailing_traffic(m, n, b):
    """DRAM bytes of the first block's C -= Y.W2 launch of an m x n solve with block b,
    scaled from the capture by operand bytes."""
    cap = TRAILING_CAPTURE
    ratio = cap["dram_bytes"] / gemm_operand_bytes(cap["rows"], cap["cols"], cap["k"])
    rows, cols = m - b, n - b
    return {"bytes": ratio * gemm_operand_bytes(rows, cols, b), "launch": f"C -= Y.W2, C {rows}x{cols}, K={b}",
            "dram_over_operand_bytes": ratio,
            "how": ("scaled by operand bytes from one ncu capture of the 8192^2, b=256 solve "
                    "(C 5888x5888, K=256: 522.8 MB of DRAM traffic against 578.8 MB of operand bytes)")}


def canonical_flops(m, n):
    return 2.0 * m * n * n - 2.0 * n ** 3 / 3.0


def rank_seed(base, rank):
    """Each replica factors its own matrix (independent problems)."""
    return base + 1000 * rank


def max_over_ranks(x, dist=None, device="cpu"):
    """Max of a per-rank float over all ranks (the timed region's length)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gflops(flops_per_step, steps, world, max_total_ms):
    """Whole-job throughput: all ranks' canonical FLOPs over the slowest rank's time."""
    return flops_per_step * steps * world / (max_total_ms * 1e-3) / 1e9


def parse():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=32768)
    p.add_argument("--m", type=int, default=None)
    p.add_argument("--b", type=int, default=256,
                   help="block size (the configuration sweeps 256, 512, 1024, 2048; 256 is the fastest on this part)")
    p.add_argument("--d", type=int, default=None)
    p.add_argument("--family", choices=["gaussian", "spectrum"], default="gaussian")
    p.add_argument("--decay", type=float, default=12.0,
                   help="family spectrum: sigma_k = 10^(-decay (k-1)/(n-1)) (14: the mixed configuration)")
    p.add_argument("--sketch", choices=["dense", "sparse"], default="dense")
    p.add_argument("--panel", choices=["cholqr", "hqr"], default="cholqr")
    p.add_argument("--panel-tc", action="store_true",
                   help="with a mixed --precision: the panel's Gram and tall-solve updates as slice products")
    p.add_argument("--precision", choices=["fp64", "mixed", "mixed_sketch32"], default="fp64",
                   help="mixed: sketch and trailing-update products on the bf16 tensor cores (exact slices)")
    p.add_argument("--seed", type=int, default=2)
    p.add_argument("--schedule", choices=["overlap", "serial"], default="overlap",
                   help="overlap: the sketch update and the next block's Alg. 2 on a side stream during the "
                        "trailing update; serial: one stream")
    p.add_argument("--skip-qr", action="store_true", help="do not time the own unpivoted QR")
    p.add_argument("--skip-e2e", action="store_true", help="do not time the host-buffer entry point")
    p.add_argument("--skip-cpu", action="store_true", help="do not time the CPU oracle sample")
    p.add_argument("--qr-reps", type=int, default=3, help="timed runs of the own unpivoted QR")
    p.add_argument("--cpu-budget", type=float, default=60.0,
                   help="seconds of host time the CPU oracle plan may take (the largest sizes are skipped beyond it)")
    p.add_argument("--skip-mixed", action="store_true",
                   help="with --precision fp64, do not also time the mixed-precision form on the same input")
    p.add_argument("--only", choices=["factor", "gemm", "ozaki", "geqrf"], default="factor",
                   help="gemm: time the library's FP64 GEMM alone (C -= A B, the trailing-update shape); "
                        "geqrf: time the library's own unpivoted QR alone on the m x n input")
    p.add_argument("--gemm", type=int, nargs=3, default=[8192, 8192, 512], metavar=("M", "N", "K"))
    p.add_argument("--workload", choices=["single", "batched", "serving"], default="single",
                   help="batched: 4096 independent matrices (m log-uniform in [64, 1024], n log-uniform in "
                        "[32, m], sigma_k = 10^(-8(k-1)/(n-1))), autotuned b, d and tile width, one CUDA graph per step")
    p.add_argument("--batch", type=int, default=4096)
    p.add_argument("--requests", type=int, default=200,
                   help="serving: requests per load level (a bounded sample of the 20000-request stream)")
    p.add_argument("--loads", type=float, nargs="+", default=[0.5, 0.8, 1.2])
    p.add_argument("--serving-precision", choices=["fp64", "mixed"], default="fp64",
                   help="serving: arithmetic of the large lane (mixed: FP64-accurate products on the tensor cores)")
    p.add_argument("--batch-b", type=int, default=0,
                   help="batched: fixed block size for every matrix instead of the autotuner (d = ceil(1.25 b))")
    p.add_argument("--batch-tile", type=int, default=64, choices=[32, 64],
                   help="batched, with --batch-b: trailing tile width (columns) of every matrix")
    a = p.parse_args()
    a.m = a.m or a.n
    a.d = a.d or int(math.ceil(1.25 * a.b))
    return a


def workload_name(a):
    dec = getattr(a, "decay", 12.0)
    fam = "iid N(0,1)" if a.family == "gaussian" else f"U diag(sigma) V^T, sigma geometric 1..1e-{dec:g}"
    sk = "dense Philox +-1" if a.sketch == "dense" else "sparse-sign (8 nnz/col)"
    prec = {"fp64": "FP64", "mixed": "mixed-precision (bf16 tensor-core slices, FP64 accuracy)",
            "mixed_sketch32": "mixed-precision (bf16 tensor-core slices, FP64 accuracy; FP32 sketch QR)"}[a.precision]
    if getattr(a, "panel_tc", False) and a.precision != "fp64":
        prec += " with the panel's Gram and tall-solve updates as slices"
    return f"{prec} BQRRP m={a.m} n={a.n} b={a.b} d={a.d}, {fam}, {sk} sketch, {a.panel} panel"


def config(a, world):
    return {"workload": workload_name(a), "m": a.m, "n": a.n, "b": a.b, "d": a.d, "family": a.family,
            "decay": getattr(a, "decay", 12.0) if a.family == "spectrum" else None,
            "sketch": a.sketch, "panel": a.panel, "precision": a.precision,
            "panel_tc": bool(getattr(a, "panel_tc", False) and a.precision != "fp64"), "seed": a.seed,
            "schedule": a.schedule if (a.precision == "fp64" and a.panel == "cholqr") else "serial",
            "l2": f"inputs larger than L2 (A is {a.m * a.n * 8 / 1e9:.2f} GB, L2 126 MB)",
            "parallelism": "replicas" if world > 1 else "single"}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="bqrrp_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


# ------------------------------------------------------------------ CPU oracle baseline
def host_cpu():
    """Host CPU model and hardware thread count."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return model, os.cpu_count() or 1


def time_oracle(A, b, d, threads, sketch_kind=0):
    """Seconds of one oracle BQRRP call with this many threads."""
    import oracle
    oracle.set_threads(threads)
    t0 = time.perf_counter()
    oracle.bqrrp(A, b, d, 1, sketch_kind=sketch_kind)
    dt = time.perf_counter() - t0
    oracle.set_threads(1)
    return dt


def cpu_plan(a, budget_s=60.0):
    """The oracle, as it stands, timed on the host (the measurement plan of the
    configuration): C1 (2000 x 1000, b = 128, d = 160) on one thread and on all
    cores; then m = n = 4096 and 8192 with the bench's b and d on all cores
    (8192 only if the 4096 time, scaled by n^3, fits the budget); the bench's
    size is extrapolated from the largest measured one by n^3 scaling and
    labelled as such.  Returns the cpu_baseline object: value = the all-core
    rate at the largest measured size."""
    from paper_2507_00976_b300 import workloads as W
    model, ncpu = host_cpu()
    sk = 0 if a.sketch == "dense" else 1
    runs = []
    C1 = W.c1_matrix()
    fl1 = canonical_flops(2000, 1000)
    for th in (1, ncpu):
        dt = time_oracle(C1, 128, 160, th, sk)
        runs.append({"size": "2000x1000 (C1)", "b": 128, "d": 160, "threads": th, "s": dt, "gflops": fl1 / dt / 1e9})
    t_used = sum(r["s"] for r in runs)
    last = None
    for s in (4096, 8192):
        if last is not None and t_used + last["s"] * (s / last["n"]) ** 3 > budget_s:
            break
        A = W.gaussian(s, s, a.seed) if a.family == "gaussian" else W.spectrum(s, s, W.geometric_sigma(s, -getattr(a, "decay", 12.0)),
                                                                                a.seed)
        dt = time_oracle(A, a.b, a.d, ncpu, sk)
        t_used += dt
        last = {"size": f"{s}x{s}", "n": s, "b": a.b, "d": a.d, "threads": ncpu, "s": dt,
                "gflops": canonical_flops(s, s) / dt / 1e9}
        runs.append(last)
        del A
    extrap = {}
    for s in sorted({16384, 32768, a.n}):
        if s > last["n"]:
            t = last["s"] * (s / last["n"]) ** 3
            extrap[f"{s}x{s}"] = {"s": t, "gflops": canonical_flops(s, s) / t / 1e9,
                                  "from": last["size"], "how": "extrapolated by n^3 scaling, not measured"}
    return {"value": last["gflops"], "unit": "GFLOP/s", "cores": ncpu, "kind": "oracle",
            "sample": (f"oracle BQRRP on {last['size']} ({a.family}), b={a.b}, d={a.d}, {ncpu} threads (OpenMP over "
                       f"independent columns), {last['s']:.1f} s; the bench's {a.n}x{a.n} is extrapolated below"),
            "host_cpu": model, "nproc": ncpu, "runs": runs, "extrapolated": extrap}


def host_lapack_context(a, s=4096):
    """Host LAPACK (scipy) on the same s x s sample: GEQP3 (the paper's CPU
    comparison routine) and GEQRF, on all host cores.  Context, not a target."""
    import numpy as np
    import scipy.linalg as sla

    from paper_2507_00976_b300 import workloads as W
    A = W.gaussian(s, s, a.seed) if a.family == "gaussian" else W.spectrum(s, s, W.geometric_sigma(s, -getattr(a, "decay", 12.0)), a.seed)
    threads = None
    try:
        from threadpoolctl import threadpool_info
        threads = max((p.get("num_threads", 0) for p in threadpool_info()), default=None)
    except Exception:
        threads = os.cpu_count()
    out = {"size": f"{s}x{s}", "threads": threads, "library": "scipy.linalg (host LAPACK)",
           "note": "the paper's CPU comparison routine on this host: context, not a target"}
    for name, fn in (("geqp3", lambda: sla.qr(A, mode="r", pivoting=True)), ("geqrf", lambda: sla.qr(A, mode="r"))):
        t0 = time.perf_counter()
        fn()
        dt = time.perf_counter() - t0
        out[f"{name}_gflops"] = canonical_flops(s, s) / dt / 1e9
        out[f"{name}_s"] = dt
    return out


def run_reference(a, world, rank):
    """--impl reference: the oracle, as it stands, on the host cores."""
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2507_00976_b300 import workloads as W
    s = 2048
    b, d = a.b, a.d
    _, ncpu = host_cpu()
    A = W.gaussian(s, s, a.seed) if a.family == "gaussian" else W.spectrum(s, s, W.geometric_sigma(s, -getattr(a, "decay", 12.0)), a.seed)
    oracle.set_threads(ncpu)
    for _ in range(a.warmup):
        oracle.bqrrp(A, b, d, 1)
    times = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        oracle.bqrrp(A, b, d, 1)
        times.append(time.perf_counter() - t0)
    oracle.set_threads(1)
    tot = sum(times)
    value = canonical_flops(s, s) * len(times) / tot / 1e9
    sample = (f"oracle BQRRP on {s}x{s} (a bounded sample of the workload: same family, b, d), b={b}, d={d}, "
              f"{ncpu} threads (OpenMP over independent columns) per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config(a, world),
            "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": ncpu, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_own_qr(A, A0, precision, reps):
    """Event-timed runs of the library's own unpivoted QR on copies of A0."""
    import torch

    from paper_2507_00976_b300 import binding as B
    m, n = A.shape
    tau = torch.empty(n, dtype=torch.float64, device="cuda")
    if precision.startswith("mixed"):
        ws = torch.empty(B.bqrrp_geqrf_mixed_workspace(m, n), dtype=torch.uint8, device="cuda")
    else:
        ws = torch.empty(B.bqrrp_geqrf_workspace(m, n, 0), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    out = []
    for _ in range(reps):
        A.copy_(A0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if precision.startswith("mixed"):
            B.bqrrp_geqrf_mixed(A, tau=tau, workspace=ws)
        else:
            B.bqrrp_geqrf(A, 0, tau=tau, workspace=ws)
        e1.record(stream)
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


# ------------------------------------------------------------------ GEMM alone
def run_gemm(a):
    import torch

    from paper_2507_00976_b300 import binding as B
    M, N, K = a.gemm
    g = torch.Generator(device="cuda")
    g.manual_seed(a.seed)
    A = torch.randn((K, M), generator=g, dtype=torch.float64, device="cuda").t()
    Bm = torch.randn((N, K), generator=g, dtype=torch.float64, device="cuda").t()
    C = torch.randn((N, M), generator=g, dtype=torch.float64, device="cuda").t()
    ws = torch.empty(B.bqrrp_dgemm_workspace(M, N, K), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    if a.only == "ozaki":
        run = lambda: B.bqrrp_dgemm_ozaki("N", "N", -1.0, A, Bm, 1.0, C)
    else:
        run = lambda: B.bqrrp_dgemm("N", "N", -1.0, A, Bm, 1.0, C, workspace=ws)
    for _ in range(a.warmup):
        run()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    tf = 2.0 * M * N * K / (ms * 1e-3) / 1e12
    name = "FP64 GEMM TFLOP/s (C -= A B)" if a.only == "gemm" else \
        "FP64-accurate GEMM on bf16 tensor cores, FP64-equivalent TFLOP/s (C -= A B)"
    line = {"metric": name, "value": tf, "unit": "TFLOP/s", "ms_per_step": ms, "steps": a.steps, "warmup": a.warmup,
            "config": {"M": M, "N": N, "K": K}, "frac_of_fp64_peak": tf / FP64_PEAK_TFLOPS}
    if a.only == "ozaki":
        # OZ_PRODUCTS bf16 slice products per FP64 product
        line["bf16_tensor_tflops"] = OZ_PRODUCTS * tf
        line["roofline"] = mixed_roofline(tf)
    print(json.dumps(line), flush=True)


def run_geqrf(a):
    import torch

    import paper_2507_00976_b300 as bq
    from paper_2507_00976_b300 import binding as B
    from paper_2507_00976_b300 import workloads as W
    m, n = a.m, a.n
    A0 = W.gaussian_torch(m, n, a.seed)
    A = bq.colmajor_empty(m, n)
    tau = torch.empty(n, dtype=torch.float64, device="cuda")
    ws = torch.empty(B.bqrrp_geqrf_workspace(m, n, 0), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    ms = []
    for i in range(a.warmup + a.steps):
        A.copy_(A0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.bqrrp_geqrf(A, 0, tau=tau, workspace=ws)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= a.warmup:
            ms.append(e0.elapsed_time(e1))
    t = statistics.mean(ms)
    print(json.dumps({"metric": "own unpivoted QR GFLOP/s (2mn^2-2n^3/3)", "value": canonical_flops(m, n) / (t * 1e-3) / 1e9,
                      "unit": "GFLOP/s", "ms_per_step": t, "steps": a.steps, "warmup": a.warmup,
                      "config": {"m": m, "n": n}}), flush=True)


# ------------------------------------------------------------------ GPU arm
# ------------------------------------------------------------------ batched workload
def batched_cpu_sample(m, n, b, d, seeds, budget_s=15.0):
    """The oracle, as it stands, on matrices of the batch taken in order until
    about budget_s of CPU time; returns (GFLOP/s, description, threads)."""
    import numpy as np

    import oracle
    from paper_2507_00976_b300 import workloads as W
    done, fl, t_tot = 0, 0.0, 0.0
    for i in range(len(m)):
        A = W.batched_matrix(int(m[i]), int(n[i]), 7000 + i)
        t0 = time.perf_counter()
        oracle.bqrrp(A, int(b[i]), int(d[i]), int(seeds[i]))
        t_tot += time.perf_counter() - t0
        fl += canonical_flops(int(m[i]), int(n[i]))
        done += 1
        if t_tot >= budget_s:
            break
    return fl / t_tot / 1e9, (f"oracle BQRRP on the first {done} matrices of the batch (same shapes, b, d), "
                              f"1 thread, {t_tot:.1f} s"), 1


def run_batched(a, world, rank, local):
    import numpy as np
    import torch

    from paper_2507_00976_b300 import binding as B
    from paper_2507_00976_b300 import workloads as W

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    seed = rank_seed(a.seed, rank)
    m, n = W.batched_shapes(a.batch, seed)
    seeds = (np.arange(a.batch, dtype=np.uint64) + np.uint64(seed * 100000))
    tol = 1e-8
    A0 = W.batched_torch(m, n, seed)
    flops = float(sum(canonical_flops(int(x), int(y)) for x, y in zip(m, n)))
    tot_j = int(n.sum())
    t_tune = time.perf_counter()
    if a.batch_b > 0:
        b = np.full(a.batch, a.batch_b, dtype=np.int64)
        d = np.full(a.batch, int(math.ceil(1.25 * a.batch_b)), dtype=np.int64)
        tiles = np.full(a.batch, a.batch_tile, dtype=np.int64)
        tuned_ms = None
    else:
        b, d, tiles, tuned_ms = B.bqrrp_batch_autotune_tiles(m, n, seeds, A0, tol)
    t_tune = time.perf_counter() - t_tune
    plan = B.BatchPlan(m, n, b, d, seeds, tol, tiles=tiles)
    A = torch.empty_like(A0)
    jpvt = torch.empty(tot_j, dtype=torch.int64, device="cuda")
    tau = torch.empty(tot_j, dtype=torch.float64, device="cuda")
    rk = torch.empty(a.batch, dtype=torch.int64, device="cuda")
    tr = torch.empty(a.batch, dtype=torch.int64, device="cuda")
    info = torch.empty(a.batch, dtype=torch.int32, device="cuda")
    ws = torch.empty(plan.workspace_bytes(), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def one_step():
        A.copy_(A0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.factor(A, jpvt, tau, rk, tr, info, workspace=ws, use_graph=True)
        e1.record(stream)
        return e0, e1

    for _ in range(max(3, a.warmup)):
        one_step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    l0 = B.bqrrp_launch_counter()
    t0 = time.perf_counter()
    evs = [one_step() for _ in range(a.steps)]
    barrier()
    t_wall = time.perf_counter() - t0
    clocks = sampler.stop()
    launches = (B.bqrrp_launch_counter() - l0) or plan.launches() * a.steps   # graph replays count no launches
    step_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    tot_ms = max_over_ranks(sum(step_ms), dist, "cuda")
    value = job_gflops(flops, a.steps, world, tot_ms)
    ranks, truncs, infos = rk.cpu().numpy(), tr.cpu().numpy(), info.cpu().numpy()

    # one profiled eager step: per-phase device time and algorithmic FLOPs
    A.copy_(A0)
    B.bqrrp_profile_reset()
    B.bqrrp_profile_enable(True)
    plan.factor(A, jpvt, tau, rk, tr, info, workspace=ws, use_graph=False)
    B.bqrrp_profile_enable(False)
    prof = B.bqrrp_profile_read()
    tot_p = sum(prof[p][0] for p in B.PHASES) or 1e-9
    phases = {}
    for name in B.PHASES:
        ms, fl = prof[name]
        phases[name] = {"ms_per_step": ms, "share": ms / tot_p,
                        "tflops": (fl / (ms * 1e-3) / 1e12) if ms > 0 and fl > 0 else None}
    dom = max(B.PHASES, key=lambda p: prof[p][0])
    dms, dfl = prof[dom]
    kern = {"sketch": "bat_sketch_kernel", "lupp": "bat_qrcp_kernel", "permute": "bat_perm_kernel",
            "panel": "bat_panel_kernel", "trailing": "bat_trailing_kernel", "sketch_update": "bat_skupdate_kernel",
            "other": "bat_init_kernel / bat_finish_kernel"}.get(dom, dom)
    ach = dfl / (dms * 1e-3) / 1e12 if dms > 0 and dfl > 0 else None
    roofline = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": (ach / FP64_PEAK_TFLOPS) if ach else None, "traffic": None,
                "kernel": f"{kern} (dominant phase '{dom}', {dms:.1f} ms of {tot_p:.1f} ms in an eager profiled step)",
                "peak_source": "derived: 148 SMs x 2 DFMA/clk/SM x 2 FLOP x 2032 MHz",
                "whole_step_tflops": flops / (statistics.mean(step_ms) * 1e-3) / 1e12}

    # end to end: pinned host A in, factor, A / jpvt / tau / rank / truncation out
    e2e = None
    if not a.skip_e2e:
        Ah0 = torch.empty(A0.numel(), dtype=torch.float64).pin_memory()
        Ah0.copy_(A0)
        Ah = torch.empty_like(Ah0).pin_memory()
        jh = torch.empty(tot_j, dtype=torch.int64).pin_memory()
        th = torch.empty(tot_j, dtype=torch.float64).pin_memory()
        rh = torch.empty(a.batch, dtype=torch.int64).pin_memory()
        trh = torch.empty(a.batch, dtype=torch.int64).pin_memory()
        ems = []
        for _ in range(max(1, min(a.steps, 3))):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            A.copy_(Ah0, non_blocking=True)
            plan.factor(A, jpvt, tau, rk, tr, info, workspace=ws, use_graph=True)
            Ah.copy_(A, non_blocking=True)
            jh.copy_(jpvt, non_blocking=True)
            th.copy_(tau, non_blocking=True)
            rh.copy_(rk, non_blocking=True)
            trh.copy_(tr, non_blocking=True)
            e1.record(stream)
            torch.cuda.synchronize()
            ems.append(e0.elapsed_time(e1))
        tot_e = max_over_ranks(sum(ems), dist, "cuda")
        e2e = {"value": job_gflops(flops, len(ems), world, tot_e), "unit": "GFLOP/s",
               "h2d_bytes_per_step": A0.numel() * 8,
               "d2h_bytes_per_step": A0.numel() * 8 + tot_j * 16 + a.batch * 16, "steps": len(ems),
               "entry_point": "bqrrp_batch_factor with pinned host copies in the timed region"}
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    cpu = None
    if not a.skip_cpu and world == 1:
        gf, sample, cores = batched_cpu_sample(m, n, b, d, seeds)
        cpu = {"value": gf, "unit": "GFLOP/s", "cores": cores, "kind": "oracle", "sample": sample}
    lat = sorted(step_ms)
    p99 = lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]
    classes = {}
    for lo, hi in [(0, 64), (64, 128), (128, 256), (256, 512), (512, 1024), (1024, 1 << 30)]:
        sel = (n >= lo) & (n < hi)
        if sel.any():
            classes[f"n in [{lo},{hi})"] = {"count": int(sel.sum()), "b": sorted(set(b[sel].tolist())),
                                           "d": sorted(set(d[sel].tolist())),
                                           "tile_cols": sorted(set(tiles[sel].tolist()))}
    line = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": a.steps,
        "warmup": max(3, a.warmup), "ms_per_step": tot_ms / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"batched FP64 BQRRP: {a.batch} matrices, m log-uniform in [64, 1024], n log-uniform "
                               f"in [32, m], U diag(sigma) V^T with sigma_k = 10^(-8(k-1)/(n-1)), dense Philox +-1 "
                               f"sketch, CholQR panel, truncation at ||R22||_F <= 1e-8 ||A||_F, one CUDA graph per "
                               f"step", "batch": a.batch, "trunc_tol": tol, "seed": a.seed,
                   "total_canonical_gflop": flops / 1e9, "matrix_bytes": A0.numel() * 8,
                   "l2": f"inputs larger than L2 (the batch is {A0.numel() * 8 / 1e9:.2f} GB, L2 126 MB)",
                   "block_sizes": "fixed" if a.batch_b > 0 else "autotuned (b, d and trailing tile width)",
                   "classes": classes,
                   "autotune_s": t_tune, "autotune_best_ms": tuned_ms,
                   "parallelism": "replicas" if world > 1 else "single"},
        "latency_ms": {"p50": statistics.median(lat), "p99": p99, "best": lat[0]},
        "own_qr": None, "gpu_launches": launches, "launches_per_step": plan.launches(), "wall_s": t_wall,
        "ranks": {"full_rank": int((ranks == n).sum()), "info_nonzero": int((infos != 0).sum()),
                  "trunc_rank_mean": float(truncs.mean()), "n_mean": float(n.mean())},
        "roofline": roofline, "phases": phases, "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    plan.close()
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------------ serving workload
# (m, n, b, d): b is the fastest of a sweep on this part (8192 x 4096: 128 over 256 and 512; 4096 x 2048: 64 over
# 128 and 256); the two small shapes use b = 32 in the batched lane
SERVING_SHAPES = [(256, 256, 32, 40), (1024, 512, 32, 40), (4096, 2048, 64, 80), (8192, 4096, 128, 160)]
SERVING_WEIGHTS = [0.5, 0.3, 0.15, 0.05]


def run_serving(a, world, rank, local):
    """Poisson-arrival stream of factorization requests of mixed shapes through
    the library's request loop (bqrrp_server_*), at several offered loads."""
    import numpy as np
    import torch

    from paper_2507_00976_b300 import binding as B
    from paper_2507_00976_b300 import workloads as W

    torch.cuda.set_device(local)
    seed = rank_seed(a.seed, rank)
    rng = np.random.Generator(np.random.PCG64(seed))
    tol = 1e-8
    # a pool of distinct inputs per shape (pinned host memory), spectra
    # geometric from 1 down to a decay drawn uniformly in exponent from [1e-14, 1e-4]
    per_shape = [6, 4, 3, 2]
    inputs = []
    for si, ((m, n, b, d), k) in enumerate(zip(SERVING_SHAPES, per_shape)):
        lst = []
        for j in range(k):
            decay = 10.0 ** rng.uniform(-14.0, -4.0)
            sig = decay ** (np.arange(n) / (n - 1))
            Ad = W.spectrum_torch(m, n, sig, seed * 100 + si * 10 + j)
            Ah = torch.empty((n, m), dtype=torch.float64).pin_memory()
            Ah.copy_(Ad.t())
            del Ad
            lst.append(Ah)
        inputs.append(lst)
    torch.cuda.empty_cache()
    outs = []
    for (m, n, b, d) in SERVING_SHAPES:
        outs.append((torch.empty((n, m), dtype=torch.float64).pin_memory(),
                     torch.empty(n, dtype=torch.int64).pin_memory(), torch.empty(n, dtype=torch.float64).pin_memory()))
    budget = 120 << 30
    mixed_lane = a.serving_precision == "mixed"
    S = B.Server(budget, (12 if mixed_lane else 8) << 30, trunc_tol=tol, small_max_elems=1 << 20, mixed=mixed_lane)

    def draw(count, rng_):
        kinds = rng_.choice(len(SERVING_SHAPES), size=count, p=SERVING_WEIGHTS)
        picks = [int(rng_.integers(len(inputs[k]))) for k in kinds]
        return list(zip(kinds.tolist(), picks))

    def run(stream, gaps):
        """Submit stream[i] at cumulative time sum(gaps[:i+1]) after start; returns completions."""
        t_base = S.clock()
        done, sub_t = [], {}
        arrival = t_base
        for i, (k, j) in enumerate(stream):
            arrival += gaps[i]
            while S.clock() < arrival:
                done += S.poll(256, 0.0)
                time.sleep(min(0.0005, max(0.0, arrival - S.clock())))
            m, n, b, d = SERVING_SHAPES[k]
            Ao, jo, to = outs[k]
            rid = len(sub_t) + 1_000_000 * run.calls
            sub_t[rid] = (arrival, k)
            S.submit(rid, m, n, b, d, 7 + i, inputs[k][j], Ao, jo, to)
        S.drain()
        done += S.poll(100000, 0.0)
        run.calls += 1
        return done, sub_t

    run.calls = 0
    # warm-up: one of each shape
    run([(k, 0) for k in range(len(SERVING_SHAPES))], [0.0] * len(SERVING_SHAPES))
    l0 = B.bqrrp_launch_counter()
    sampler = ClockSampler(local)
    sampler.start()
    # capacity: the sample offered all at once
    base_stream = draw(a.requests, rng)
    done, sub = run(base_stream, [0.0] * len(base_stream))
    span = max(c["t_done"] for c in done) - min(c["t_submit"] for c in done)
    capacity = len(done) / span
    flops_per_req = float(np.mean([canonical_flops(*SERVING_SHAPES[k][:2]) for k, _ in base_stream]))
    loads = {}
    for load in a.loads:
        # the same request sample at every load (only the arrival gaps differ), so
        # the levels compare the server, not the shape mix of different samples
        lam = load * capacity
        gaps = rng.exponential(1.0 / lam, size=len(base_stream))
        gaps[0] = 0.0
        done, sub = run(base_stream, gaps)
        lat = np.array([(c["t_done"] - sub[c["id"]][0]) * 1e3 for c in done])
        kinds = np.array([sub[c["id"]][1] for c in done])
        fl = sum(canonical_flops(*SERVING_SHAPES[sub[c["id"]][1]][:2]) for c in done)
        t0 = min(sub[c["id"]][0] for c in done)
        t1 = max(c["t_done"] for c in done)
        per_shape = {}
        for k, (m, n, _, _) in enumerate(SERVING_SHAPES):
            sel = kinds == k
            if sel.any():
                per_shape[f"{m}x{n}"] = {"count": int(sel.sum()), "p50_ms": float(np.percentile(lat[sel], 50)),
                                         "p99_ms": float(np.percentile(lat[sel], 99))}
        loads[str(load)] = {"offered_req_per_s": lam, "completed": len(done),
                            "gflops": fl / (t1 - t0) / 1e9, "p50_ms": float(np.percentile(lat, 50)),
                            "p99_ms": float(np.percentile(lat, 99)),
                            "status_nonzero": int(sum(1 for c in done if c["status"] != 0)),
                            "per_shape": per_shape}
    clocks = sampler.stop()
    st = S.stats()
    launches = B.bqrrp_launch_counter() - l0
    S.close()
    if rank != 0:
        return
    hi = loads[str(max(a.loads))]
    mid = loads[str(sorted(a.loads)[len(a.loads) // 2])]
    line = {
        "metric": METRIC, "value": hi["gflops"], "unit": "GFLOP/s", "n_gpus": world, "steps": len(a.loads),
        "warmup": 1, "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "serving loop: Poisson arrivals of FP64 factorization requests, shapes 256x256 / "
                               "1024x512 / 4096x2048 / 8192x4096 with weights 0.5/0.3/0.15/0.05, spectra geometric "
                               "from 1 to a decay uniform in exponent on [1e-14, 1e-4], truncation 1e-8, admission by "
                               "a 120 GB HBM budget, continuous batching of the small shapes"
                               + ("; large lane in the mixed form (FP64-accurate products on the tensor cores)"
                                  if mixed_lane else ""), "large_lane_precision": a.serving_precision,
                   "requests_per_load": len(base_stream),
                   "sample": (f"{len(base_stream)} requests per load level" +
                              (" (the configured 20000-request stream)" if len(base_stream) >= 20000 else
                               " (a bounded sample of the 20000-request stream)")), "hbm_budget_bytes": budget,
                   "block_sizes": {f"{m}x{n}": [b, d] for m, n, b, d in SERVING_SHAPES},
                   "capacity_req_per_s": capacity, "mean_gflop_per_request": flops_per_req / 1e9,
                   "parallelism": "single"},
        "latency_ms": {"p50": mid["p50_ms"], "p99": mid["p99_ms"], "at_load": sorted(a.loads)[len(a.loads) // 2]},
        "loads": loads, "server": st, "e2e": {"value": hi["gflops"], "unit": "GFLOP/s",
                                             "note": "every request is copied host->device at admission and its "
                                                     "R, reflectors, jpvt and tau device->host at completion"},
        "gpu_launches": launches, "roofline": None, "cpu_baseline": None, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, world, rank)
        return
    if a.workload == "batched":
        run_batched(a, world, rank, local)
        return
    if a.workload == "serving":
        run_serving(a, world, rank, local)
        return
    if a.only in ("gemm", "ozaki"):
        run_gemm(a)
        return
    if a.only == "geqrf":
        run_geqrf(a)
        return

    import torch

    import paper_2507_00976_b300 as bq
    from paper_2507_00976_b300 import binding as B
    from paper_2507_00976_b300 import workloads as W

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    m, n, b, d = a.m, a.n, a.b, a.d
    seed = rank_seed(a.seed, rank)
    if a.family == "gaussian":
        A0 = W.gaussian_torch(m, n, seed)
    else:
        A0 = W.spectrum_torch(m, n, W.geometric_sigma(min(m, n), -a.decay), seed)
    A = bq.colmajor_empty(m, n)
    jpvt = torch.empty(n, dtype=torch.int64, device="cuda")
    tau = torch.empty(n, dtype=torch.float64, device="cuda")
    opts = B.make_opts(B.SKETCH_DENSE if a.sketch == "dense" else B.SKETCH_SPARSE, 8,
                       B.PANEL_CHOLQR if a.panel == "cholqr" else B.PANEL_HQR,
                       B._PRECISIONS[a.precision],
                       B.SCHEDULE_OVERLAP if a.schedule == "overlap" else B.SCHEDULE_SERIAL,
                       1 if (a.panel_tc and a.precision != "fp64") else 0)
    ws = torch.empty(B.bqrrp_workspace_query(m, n, b, d, opts), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    probe = B.bqrrp_probe_fp64_peak(4000)

    def one_factor():
        A.copy_(A0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rk = B.bqrrp_factor(A, b, d, 1, jpvt, tau, opts=opts, workspace=ws)
        e1.record(stream)
        return e0, e1, rk

    for _ in range(a.warmup):
        one_factor()
    torch.cuda.synchronize()

    # ---------------- timed region: exactly K steps
    sampler = ClockSampler(local)
    B.bqrrp_profile_reset()
    B.bqrrp_profile_enable(True)
    launches0 = B.bqrrp_launch_counter()
    barrier()
    sampler.start()
    t_wall0 = time.perf_counter()
    evs = []
    ranks = []
    for _ in range(a.steps):
        e0, e1, rk = one_factor()
        evs.append((e0, e1))
        ranks.append(rk)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    barrier()
    clocks = sampler.stop()
    launches = B.bqrrp_launch_counter() - launches0
    B.bqrrp_profile_enable(False)
    prof = B.bqrrp_profile_read()
    step_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    tot_ms = max_over_ranks(sum(step_ms), dist, "cuda")
    flops = canonical_flops(m, n)
    value = job_gflops(flops, a.steps, world, tot_ms)

    # ---------------- the library's own unpivoted QR on the same input
    qr = None
    if not a.skip_qr:
        qms = time_own_qr(A, A0, a.precision, max(1, a.qr_reps))
        qr_gf = flops / (statistics.mean(qms) * 1e-3) / 1e9
        qr = {"gflops": qr_gf, "ms_mean": statistics.mean(qms), "ms_best": min(qms),
              "bqrrp_over_qr": (flops / (statistics.mean(step_ms) * 1e-3) / 1e9) / qr_gf,
              "precision": a.precision}

    # ---------------- the mixed-precision form on the same input (FP64 headline runs)
    mixed = None
    if a.precision == "fp64" and not a.skip_mixed:
        mopts = B.make_opts(B.SKETCH_DENSE if a.sketch == "dense" else B.SKETCH_SPARSE, 8,
                            B.PANEL_CHOLQR if a.panel == "cholqr" else B.PANEL_HQR, B.PRECISION_MIXED)
        del ws
        torch.cuda.empty_cache()
        ws = torch.empty(B.bqrrp_workspace_query(m, n, b, d, mopts), dtype=torch.uint8, device="cuda")
        def time_mixed(opts_):
            """Two timed solves after one warm-up, with the phase profile."""
            ms_, rank_ = [], None
            B.bqrrp_profile_reset()
            for i in range(3):
                B.bqrrp_profile_enable(i > 0)
                A.copy_(A0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                rank_ = B.bqrrp_factor(A, b, d, 1, jpvt, tau, opts=opts_, workspace=ws)
                e1.record(stream)
                torch.cuda.synchronize()
                if i > 0:
                    ms_.append(e0.elapsed_time(e1))
            B.bqrrp_profile_enable(False)
            prof_ = B.bqrrp_profile_read()
            return ms_, rank_, prof_

        mms, mrank, mprof = time_mixed(mopts)
        mtr_ms, mtr_fl = mprof["trailing"]
        mgf = flops / (statistics.mean(mms) * 1e-3) / 1e9
        mtf = mtr_fl / (mtr_ms * 1e-3) / 1e12 if mtr_ms > 0 else None
        mcalls = max(1, mprof["calls"])
        mixed = {"gflops": mgf, "ms_mean": statistics.mean(mms), "rank": mrank, "roofline": mixed_roofline(mtf),
                 "speedup_vs_fp64": mgf / (flops / (statistics.mean(step_ms) * 1e-3) / 1e9),
                 "arith": "FP64-accurate products on bf16 tensor cores (7 exact balanced 8-bit slices, 28 pair products); "
                          "LU, sketch QR, panel, tau, R in FP64",
                 "phases_ms": {p_: mprof[p_][0] / mcalls for p_ in B.PHASES}}
        # the variant with the sketch's QR factor in FP32 (pivots from the FP64 LU)
        s32 = B.make_opts(B.SKETCH_DENSE if a.sketch == "dense" else B.SKETCH_SPARSE, 8,
                          B.PANEL_CHOLQR if a.panel == "cholqr" else B.PANEL_HQR, B.PRECISION_MIXED_SKETCH32)
        sms, srank, sprof = time_mixed(s32)
        scalls = max(1, sprof["calls"])
        mixed["sketch32"] = {"gflops": flops / (statistics.mean(sms) * 1e-3) / 1e9, "ms_mean": statistics.mean(sms),
                             "rank": srank, "phases_ms": {p_: sprof[p_][0] / scalls for p_ in B.PHASES},
                             "arith": "as above, with the QR that forms R^sk from the sketch's LU factor in FP32"}
        # the variants with the CholQR panel's Gram and tall-solve updates as slice products
        for key, prec, what in (("panel_tc", B.PRECISION_MIXED, "the mixed form"),
                                ("sketch32_panel_tc", B.PRECISION_MIXED_SKETCH32, "the FP32 sketch QR variant")):
            vo = B.make_opts(B.SKETCH_DENSE if a.sketch == "dense" else B.SKETCH_SPARSE, 8,
                             B.PANEL_CHOLQR if a.panel == "cholqr" else B.PANEL_HQR, prec, panel_tc=1)
            vms, vrank, vprof = time_mixed(vo)
            vcalls = max(1, vprof["calls"])
            mixed[key] = {"gflops": flops / (statistics.mean(vms) * 1e-3) / 1e9, "ms_mean": statistics.mean(vms),
                          "rank": vrank, "phases_ms": {p_: vprof[p_][0] / vcalls for p_ in B.PHASES},
                          "arith": what + ", with the CholQR panel's Gram and the block updates of its two tall "
                                          "solves also as slice products (opts.panel_tc = 1); Cholesky, "
                                          "reconstruction LU, tau, R in FP64"}
        if not a.skip_qr:
            mq = time_own_qr(A, A0, "mixed", 3)[1:]   # one warm-up run, two timed
            mixed["own_qr_gflops"] = flops / (statistics.mean(mq) * 1e-3) / 1e9
            mixed["bqrrp_over_qr"] = mgf / mixed["own_qr_gflops"]

    # ---------------- end to end through the host-buffer entry point
    e2e = None
    if not a.skip_e2e:
        Ah0 = torch.empty((n, m), dtype=torch.float64).pin_memory().t()
        Ah0.copy_(A0)
        Ah = torch.empty((n, m), dtype=torch.float64).pin_memory().t()
        jh = torch.empty(n, dtype=torch.int64).pin_memory()
        th = torch.empty(n, dtype=torch.float64).pin_memory()
        del ws
        torch.cuda.empty_cache()
        hws = torch.empty(B.bqrrp_workspace_query_host(m, n, b, d, opts), dtype=torch.uint8, device="cuda")
        ems = []
        k_e2e = max(1, min(a.steps, 3 if m * n <= (1 << 28) else 1))
        for _ in range(k_e2e):
            Ah.copy_(Ah0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.bqrrp_factor_host(Ah, b, d, 1, jh, th, hws, opts=opts)
            e1.record(stream)
            torch.cuda.synchronize()
            ems.append(e0.elapsed_time(e1))
        tot = max_over_ranks(sum(ems), dist, "cuda")
        e2e = {"value": job_gflops(flops, k_e2e, world, tot), "unit": "GFLOP/s",
               "h2d_bytes_per_step": m * n * 8, "d2h_bytes_per_step": m * n * 8 + n * 16, "steps": k_e2e,
               "entry_point": "bqrrp_factor_host (pinned host buffers)"}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # ---------------- roofline of the dominant kernel: the FP64 GEMMs of the trailing update
    tr_ms, tr_fl = prof["trailing"]
    achieved = tr_fl / (tr_ms * 1e-3) / 1e12 if tr_ms > 0 else None
    phases = {}
    for name in B.PHASES:
        ms, fl = prof[name]
        phases[name] = {"ms_per_step": ms / max(1, prof["calls"]),
                        "share": ms / max(1e-9, sum(prof[p][0] for p in B.PHASES)),
                        "tflops": (fl / (ms * 1e-3) / 1e12) if ms > 0 and fl > 0 else None}
    if a.precision.startswith("mixed"):
        roofline = mixed_roofline(achieved)
    else:
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": (achieved / FP64_PEAK_TFLOPS) if achieved else None,
                    "traffic": trailing_traffic(a.m or a.n, a.n, a.b)["bytes"],
                    "traffic_launch": trailing_traffic(a.m or a.n, a.n, a.b),
                    "kernel": "dgemm_kernel (FP64 SIMT GEMMs of the trailing block-reflector update)",
                    "peak_source": "derived: 148 SMs x 2 DFMA/clk/SM x 2 FLOP x 2032 MHz",
                    "dfma_probe_tflops": probe}
        if config(a, world)["schedule"] == "overlap":
            roofline["note"] = ("overlap schedule: the sketch update and the next block's LU and sketch QR run on a "
                                "side stream during the trailing update and share its SMs' FP64 pipes; the "
                                "trailing launches' event times include that sharing")
    cpu = None
    if not a.skip_cpu and world == 1:
        cpu = cpu_plan(a, a.cpu_budget)
        try:
            lapack = host_lapack_context(a)
        except Exception as e:   # context only: never costs the bench line
            lapack = {"unavailable": f"{type(e).__name__}: {e}"}
        cpu["host_lapack"] = lapack
    lat = sorted(step_ms)
    p99 = lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]
    # the metric's comparison: BQRRP over the own unpivoted QR, same input, same GPU
    vs = (value / world) / qr["gflops"] if qr else None
    line = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": tot_ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": vs,
        "vs_baseline_def": "per-GPU BQRRP GFLOP/s / own unpivoted blocked QR GFLOP/s on the same input and GPU "
                           "(target >= 0.65)",
        "dtype": "f64", "data": "synthetic", "config": config(a, world),
        "latency_ms": {"p50": statistics.median(lat), "p99": p99, "best": lat[0]},
        "best_gflops": flops / (lat[0] * 1e-3) / 1e9,
        "own_qr": qr, "rank": ranks[0], "gpu_launches": launches, "wall_s": t_wall,
        "roofline": roofline, "phases": phases, "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu,
        "mixed_precision": mixed,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
