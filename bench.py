#!/usr/bin/env python
"""Gray-code steps/s of the sparse-permanent walk on one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (one "step" = one whole permanent, i.e. every row of the hot path):
the n=36 single real sparse matrix -- Erdos-Renyi nonzeros with p=0.15 plus a
forced diagonal, (0,1] values, columns in random order (seed 2).  A step walks
all 2^35 Gray indices.  Inputs are synthetic (synth.py); the plan (ordering,
partitioning, generated kernel) is built during warm-up, so the matrix is
resident on the device when the timed region starts.

value       whole-job Gray steps/s (all ranks: independent replicas, weak scaling)
e2e         the same metric through the public C ABI from a host CSR matrix
            (plan_create + compute + destroy every step, result read back)
roofline    the walk kernel against the FP64 issue rate: counted FP64 ops per
            step (cost model) x steps / kernel time
cpu_baseline the CPU oracle (Algorithm 1, long double, all host cores) on a
            bounded Gray sub-range of the same matrix
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N36 = dict(n=36, p=0.15, seed=2)
GRAY_STEPS = 1 << 35
NOMINAL_FP64_ISSUE = 2 * 152 * 2.07e9   # 1.25 TFLOP/s nominal = 2 FP64 lane-ops/clk/SM x 152 SMs x 2.07 GHz
L2_FLUSH_BYTES = 256 << 20              # > 129 MB L2
METRIC = "Gray-code steps/s (n=36 single sparse matrix permanent)"


def workload_matrix():
    from paper_2501_15126_gb300 import synth
    return synth.single_er(N36["n"], N36["p"], N36["seed"], values="f64", shuffle_cols=True)


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.proc:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        out.update(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=reasons, samples=len(rows))
        return out


def traffic_record(kernel_hash: str):
    """DRAM bytes per launch of the walk kernel from the committed ncu summary,
    or None when absent or taken on a different kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))
    except Exception:
        return None
    if rec.get("kernel_hash") != kernel_hash:
        return None
    return rec.get("dram_bytes_per_launch")


def kernel_hash() -> str:
    """Identifies the timed kernel: the CUDA C++ the generator emits for the
    workload matrix (which fixes its layout and scheme) and the two headers it
    is compiled with."""
    from paper_2501_15126_gb300 import _abi as A
    h = hashlib.sha256()
    h.update(A.codegen_source(workload_matrix()).encode())
    for name in ("core.cuh", "devmat.h"):
        h.update(open(os.path.join(ROOT, "paper_2501_15126_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def cpu_baseline(a, seconds_hint: float = 15.0):
    """The oracle as it stands (Algorithm 1, long double, every host core) on
    a Gray sub-range of the workload, sized to roughly `seconds_hint` s."""
    import oracle
    cores = os.cpu_count() or 1
    span = 1 << 20
    t0 = time.time()
    oracle.nw_range(a, 0, span, threads=cores)
    dt = max(time.time() - t0, 1e-6)
    k = 20
    while (1 << (k + 1)) * dt / span < seconds_hint and k < 34:
        k += 1
    span = 1 << k
    t0 = time.time()
    oracle.nw_range(a, 0, span, threads=cores)
    dt = time.time() - t0
    return {"value": span / dt, "unit": "steps/s", "cores": cores, "kind": "oracle",
            "sample": "Gray indices [0, 2^%d) of the n=36 matrix (Algorithm 1, long double, %d-bit significand)"
                      % (k, oracle.long_double_bits()),
            "seconds": dt}


def cpu_fp64_baseline(a, seconds_hint: float = 10.0):
    """CPU-SparsePerman (cpu_sparseperman.c beside this file: FP64, degree-sorted
    columns, zero tracking, every host core over aligned Gray chunks) on a
    Gray prefix of the workload sized to about `seconds_hint` s."""
    import ctypes
    src = os.path.join(ROOT, "cpu_sparseperman.c")
    d = tempfile.mkdtemp()
    so = os.path.join(d, "libcpu_sparseperman.so")
    subprocess.check_call(["gcc", "-O3", "-fPIC", "-shared", "-pthread", src, "-o", so, "-lm"])
    L = ctypes.CDLL(so)
    L.cpu_sparseperman_range.restype = ctypes.c_double
    L.cpu_sparseperman_range.argtypes = [ctypes.c_int] + [ctypes.c_void_p] * 4 + [ctypes.c_uint64, ctypes.c_uint64,
                                          ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    n = a.shape[0]
    order = sorted(range(n), key=lambda j: (int(np.count_nonzero(a[:, j])), j))   # ascending degree (Sec. VI-B)
    ao = np.ascontiguousarray(a[:, order])
    colptr, rows, vals = [0], [], []
    for j in range(n):
        nz = np.nonzero(ao[:, j])[0]
        rows += list(nz)
        vals += list(ao[nz, j])
        colptr.append(len(rows))
    colptr = np.array(colptr[:n], dtype=np.int32)
    rows = np.array(rows, dtype=np.int32)
    vals = np.array(vals, dtype=np.float64)
    x0 = ao[:, n - 1] - ao.sum(axis=1) / 2.0
    cores = os.cpu_count() or 1
    K = 12
    ab = ctypes.c_double()

    def run(span):
        t0 = time.perf_counter()
        L.cpu_sparseperman_range(n, colptr.ctypes.data, rows.ctypes.data, vals.ctypes.data, x0.ctypes.data, 0, span,
                                 K, cores, ctypes.byref(ab))
        return time.perf_counter() - t0
    k = 24
    dt = run(1 << k)
    while (1 << (k + 1)) * dt / (1 << k) < seconds_hint and k < n - 2:
        k += 1
        dt = run(1 << k)
    return {"value": (1 << k) / dt, "unit": "steps/s", "cores": cores, "kind": "cpu-sparseperman (FP64)",
            "sample": "Gray indices [0, 2^%d) of the n=%d matrix: FP64 Algorithm 1, degree-sorted columns, zero "
                      "tracking, %d threads over aligned 2^%d-step chunks" % (k, n, cores, K),
            "seconds": dt, "ms_per_permanent_extrapolated": 1e3 * dt * (1 << (n - 1 - k))}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    a = workload_matrix()
    import oracle
    cores = os.cpu_count() or 1
    span = 1 << 24
    for _ in range(args.warmup):
        oracle.nw_range(a, 0, 1 << 16, threads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.time()
        oracle.nw_range(a, 0, span, threads=cores)
        times.append(time.time() - t0)
    total = sum(times)
    value = args.steps * span / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f80/f128 (long double)",
            "data": "synthetic", "config": config_block("oracle", span),
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": cores, "kind": "oracle",
                             "sample": "Gray indices [0, 2^24) of the n=36 matrix per step"},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def extras(A, sh, a, first):
    """What the single-matrix line carries beside its headline (one GPU only):
    the batch and serving workloads, accuracy against the oracle on every
    workload, the first (cold) call on a matrix never seen before, the FP64
    CPU baseline, and the Table II-shaped suite."""
    from paper_2501_15126_gb300 import synth
    out = {}
    out["batch"] = measure_batch(A, sh)
    out["serving"] = measure_serving(A)
    # cold: a new n=36 matrix of the same shape, its kernel generated and compiled
    b = synth.single_er(36, 0.15, 1002, values="f64", shuffle_cols=True)
    t0 = time.perf_counter()
    rb = A.permanent(b, stream=sh, flags=A.PERM_FLAG_NO_KERNEL_CACHE)
    wall = time.perf_counter() - t0
    out["e2e_cold"] = {"seconds": wall, "ms_plan": rb.ms_plan, "ms_compile": rb.ms_compile, "ms_kernel": rb.ms_kernel,
                       "overhead_ms": rb.ms_plan + rb.ms_compile,
                       "note": "a never-seen n=36 matrix through perm_plan_create (ordering, Algorithm 4, code "
                               "generation, NVRTC) + perm_compute + perm_plan_destroy; the paper quotes < 2 s of "
                               "generation and compilation per matrix (Sec. VI-F)"}
    # accuracy against the oracle
    golden = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "er36_f64_perm.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            golden[k] = float(v)
    want2 = golden["perm_hi"] + golden["perm_lo"]
    a01 = synth.single_er(24, 0.2, 1, values="01")
    _, af = synth.single_er_pair(24, 0.2, 1)
    r01, rf = A.permanent(a01, stream=sh), A.permanent(af, stream=sh)
    out["accuracy"] = {
        "target": "exact results bit-identical, FP64 within 1e-9 relative to the oracle's permanent",
        "er24_01_and_f64": {"exact_matches": r01.value == oracle_value(a01), "f64_rel_err": rel(rf.value, oracle_value(af)),
                     "f64_precision": "double-double" if rf.precision == 2 else "fp64"},
        "er36_f64": {"f64_rel_err": rel(first.value, want2),
                     "kappa_sum_abs_terms_over_perm": golden["abs_terms"] / abs(want2),
                     "reference": "oracle value stored in tests/golden/er36_f64_perm.txt"},
        "batch_sampled": out["batch"].get("accuracy_vs_oracle"),
        "serving_sampled": out["serving"].get("accuracy_vs_oracle"),
        "band48": "whole 2^47-step exact walks: bench.py --workload band48 (profiles/band48_whole_permanent.md)"}
    out["exact_roofline"] = exact_roofline(A, sh)
    out["cpu_fp64_baseline"] = cpu_fp64_baseline(a)
    out["table2"] = measure_table2(A)
    return out


def exact_roofline(A, sh):
    """The exact path against the integer issue roofline: counted integer
    multiply operations per Gray step (the ring-op cost model,
    perm_inspect_t.ring_ops_per_step) x steps / kernel time, over the IMAD
    rate measured on this GPU: the n=24 0/1 ER matrix (the plan the library picks) and
    the n=48 band's generated exact kernel on a 2^30-step prefix."""
    from paper_2501_15126_gb300 import synth
    _, imad = A.issue_rates(sh)
    out = {"bound": "alu (IMAD)", "peak_imad_ops_per_s": imad}
    for name, a, kw in (("er24_01", synth.single_er(24, 0.2, 1, values="01"), {}),
                        ("n48_band_01_prefix_2^30", synth.band_plus(48, 3, 2, seed=3, values="01"),
                         dict(g_lo=0, g_hi=1 << 30, engine=A.PERM_ENGINE_CODEGEN))):
        p = A.Plan(a, **kw)
        r = p.compute(sh)
        ms = min(p.compute(sh).ms_kernel for _ in range(5))
        p.close()
        ach = r.fp_ops_per_step * r.steps / (ms / 1e3)
        out[name] = {"engine": "codegen" if r.engine == A.PERM_ENGINE_CODEGEN else "generic", "ms": ms,
                     "gray_steps_per_s": r.steps / (ms / 1e3), "ring_ops_per_step": r.fp_ops_per_step,
                     "achieved_imad_ops_per_s": ach, "frac": ach / imad, "zero_skip_frac": r.zero_skip_frac,
                     "exact_words": r.exact_words, "regs": r.regs_per_thread}
    return out


def config_block(engine, steps_per_step, shard=False):
    return {"workload": "single real sparse matrix n=36: ER p=0.15 + forced diagonal, (0,1] values, shuffled "
                        "columns, seed 2", "n": 36, "gray_steps_per_step": steps_per_step, "engine": engine,
            "l2": "flushed between steps (256 MiB device write)",
            "parallelism": ("Gray-range shards: one permanent split across the GPUs, partial sums combined once"
                            if shard else "replicas (one matrix per GPU)")}


def run_ours(args):
    import torch
    from paper_2501_15126_gb300 import _abi as A

    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream
    a = workload_matrix()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    fp64_rate, imad_rate = A.issue_rates(sh)
    shard = args.shard and world > 1
    if shard:
        # one permanent split across the ranks: each walks its Gray shard (Sec. II-A)
        from paper_2501_15126_gb300 import dist as pd
        lo, hi = pd.shard_range(GRAY_STEPS, world, rank)
        plan = A.Plan(a, g_lo=lo, g_hi=hi)
    else:
        plan = A.Plan(a)                   # ordering, partitioning, NVRTC (warm-up region)
    first = plan.compute(sh)
    for _ in range(max(args.warmup - 1, 0)):
        plan.compute(sh)

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    clocks = Clocks(local_rank)
    clocks.start()
    step_ms, kern_ms, results = [], [], []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)               # evict L2 between steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        r = plan.compute(sh)
        with torch.cuda.stream(stream):
            e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        kern_ms.append(r.ms_kernel)
        results.append(r.value)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    total_ms = sum(step_ms)
    combined = None
    if world > 1:
        from paper_2501_15126_gb300 import dist as pd
        total_ms = pd.max_over_ranks(total_ms, device=dev)
        if shard:   # the shards' partial sums, combined on every rank
            s_hi, s_lo = pd.combine_f64(first.f64, first.f64_lo, device=dev)
            combined = (s_hi + s_lo) * (2.0 if N36["n"] % 2 else -2.0)
        torch.distributed.barrier()

    # end to end through the public API from host memory, every step
    e2e_ms = []
    for _ in range(max(1, min(args.steps, 3))):
        t0 = time.perf_counter()
        rr = A.permanent(a, stream=sh)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
        assert shard or rr.value == first.value
    plan_engine = "codegen" if first.engine == A.PERM_ENGINE_CODEGEN else "generic"

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0
    # replicas: every rank walks a whole permanent; shards: the ranks walk one together
    value = (1 if shard else world) * args.steps * GRAY_STEPS / (total_ms / 1e3)
    mean_kernel_ms = statistics.mean(kern_ms)
    ops = first.fp_ops_per_step * GRAY_STEPS
    achieved = ops / (mean_kernel_ms / 1e3)
    kh = kernel_hash()
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if shard else "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_block(plan_engine, GRAY_STEPS, shard),
        "ms_per_permanent": total_ms / args.steps,
        "permanent": combined if shard else first.value,
        "roofline": {"bound": "alu", "achieved": achieved / 1e9, "peak": NOMINAL_FP64_ISSUE / 1e9,
                     "unit": "G FP64 op/s", "frac": achieved / NOMINAL_FP64_ISSUE,
                     "peak_measured": fp64_rate / 1e9, "frac_of_measured": achieved / fp64_rate,
                     "traffic": traffic_record(kh), "kernel": "perm_walk (generated)", "kernel_hash": kh,
                     "ops_per_step": first.fp_ops_per_step, "kernel_ms": mean_kernel_ms,
                     "peak_note": "peak = 2 FP64 ops/clk/SM x 152 SMs x 2.07 GHz (nominal 1.25 TFLOP/s); "
                                  "peak_measured = DFMA probe on this GPU (perm_issue_rates)"},
        "e2e": {"value": GRAY_STEPS / (statistics.median(e2e_ms) / 1e3), "unit": "steps/s",
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 64,
                "note": "perm_plan_create + perm_compute + perm_plan_destroy from a host CSR matrix; the matrix "
                        "reaches the GPU inside the generated kernel (cached module), the result comes back as "
                        "8 words"},
        "gpu_launches": 2 * args.steps,
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]},
        "plan": {"ms_compile": first.ms_compile, "ms_plan": first.ms_plan, "regs": first.regs_per_thread,
                 "threads": first.threads, "chunk_log2": first.chunk_log2, "reg_rows": first.reg_rows,
                 "ordering": first.ordering},
        "imad_rate_measured": imad_rate,
    }
    if not args.no_cpu_baseline and world == 1:   # the CPU baseline: rank 0 at N=1 only
        line["cpu_baseline"] = cpu_baseline(a, args.cpu_seconds)
    if world == 1 and not args.no_extras:
        line.update(extras(A, sh, a, first))
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def oracle_value(a):
    """The oracle's permanent of a small matrix: Eq. 2 in integers for 0/1
    inputs, Algorithm 1 in long double (all host cores) for real ones."""
    import oracle
    if a.dtype == np.int64:
        return oracle.ryser_gray(a)
    return float(oracle.nw_perm(a, threads=os.cpu_count() or 1)[0])


def accuracy_sample(mats, results, values, max_n=22, count=40):
    """Evenly spaced sample of the results with n <= max_n against the
    oracle: exact mismatches, FP64 max relative error, FP64 results beyond 1e-9,
    and how many of the sampled FP64 results came from double-double reruns."""
    idx = [i for i, a in enumerate(mats) if a.shape[0] <= max_n]
    f64 = [i for i in idx if values[i] != "01"][:: max(1, len([i for i in idx if values[i] != "01"]) // count)][:count]
    ex = [i for i in idx if values[i] == "01"][:: max(1, len([i for i in idx if values[i] == "01"]) // count)][:count]
    errs = [rel(results[i].value, oracle_value(mats[i])) for i in f64]
    return {"f64_sampled": len(f64), "f64_max_rel_err": max(errs, default=0.0),
            "f64_beyond_1e-9": sum(1 for e in errs if e > 1e-9),
            "f64_double_double": sum(1 for i in f64 if results[i].precision == 2),
            "exact_sampled": len(ex), "exact_mismatches": sum(1 for i in ex if results[i].value != oracle_value(mats[i])),
            "sample": "every k-th matrix with n <= %d, up to %d per arithmetic" % (max_n, count)}


def measure_batch(A, stream, count=10_000, steps=2, warmup=1, accuracy=True):
    """The 10,000-matrix workload: one persistent launch per kernel family
    (perm_batch) against one plan and launch per matrix (perm_batch_sequential,
    the paper's policy) and against the best per-matrix form here (the
    allocation-free call per matrix: no allocation, one launch and one sync)."""
    from paper_2501_15126_gb300 import synth
    items = synth.batch(count=count)
    mats = [A.CSRMatrix(it.a) for it in items]
    steps_total = sum(1 << (it.n - 1) for it in items)
    for _ in range(max(warmup, 1)):
        A.batch(mats, stream=stream)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        res = A.batch(mats, stream=stream)
        times.append(time.perf_counter() - t0)
    split = {}
    for vals in ("f64", "01"):
        sub = [m for m, it in zip(mats, items) if it.values == vals]
        sub_steps = sum(1 << (it.n - 1) for it in items if it.values == vals)
        t0 = time.perf_counter()
        A.batch(sub, stream=stream)
        dt = time.perf_counter() - t0
        split[vals] = {"count": len(sub), "seconds": dt, "gray_steps_per_s": sub_steps / dt}
    t0 = time.perf_counter()
    seq = A.batch(mats, sequential=True, stream=stream)
    seq_time = time.perf_counter() - t0
    t0 = time.perf_counter()
    loop = [A.permanent_noalloc(m, stream=stream) for m in mats]
    loop_time = time.perf_counter() - t0
    mism_exact = sum(1 for r, q, it in zip(res, seq, items) if it.values == "01" and r.value != q.value)
    max_rel_f64 = max((rel(r.value, q.value) for r, q, it in zip(res, seq, items) if it.values == "f64"), default=0.0)
    best = min(times)
    out = {"metric": "batched permanents/s (10,000 matrices, n in [12,28])", "perms_per_s": len(items) / best,
           "seconds": best, "gray_steps_total": steps_total, "gray_steps_per_s": steps_total / best,
           "workload": "batch of %d ER matrices, n uniform in [12,28], p uniform in [0.2,0.4] + forced diagonal, "
                       "alternating 0/1 (exact) and (0,1] (FP64), seed 4" % len(items),
           "by_arithmetic": split,
           "double_double_reruns": sum(1 for r in res if r.precision == 2),
           "per_matrix_plans": {"seconds": seq_time, "perms_per_s": len(items) / seq_time,
                                "speedup": seq_time / best,
                                "note": "perm_batch_sequential: plan + launch + sync + destroy per matrix"},
           "per_matrix_noalloc": {"seconds": loop_time, "perms_per_s": len(items) / loop_time,
                                  "speedup": loop_time / best,
                                  "note": "perm_compute_noalloc per matrix: no allocation, one walk launch and "
                                          "one synchronisation per matrix"},
           "agreement_vs_per_matrix": {"exact_mismatches": mism_exact, "f64_max_rel_diff": max_rel_f64}}
    out["speedup_vs_best_per_matrix"] = min(seq_time, loop_time) / best
    if accuracy:
        out["accuracy_vs_oracle"] = accuracy_sample([it.a for it in items], res, [it.values for it in items])
    return out


def measure_serving(A, rate=2000.0, duration=60.0, sequential_seconds=10.0, accuracy=True):
    """Open-loop replay of the Poisson stream against the server (latency from
    each request's arrival), and the same requests' first `sequential_seconds`
    served by one plan + launch per request, back to back (its capacity)."""
    from paper_2501_15126_gb300 import synth
    reqs = synth.serving_stream(rate=rate, duration=duration, seed=5)
    mats = [A.CSRMatrix(r.a) for r in reqs]
    arrivals = [r.t_arrival for r in reqs]
    lat = [None] * len(reqs)
    res = [None] * len(reqs)
    with A.Server() as s:
        for m in mats[:50]:                       # the kernel families set up
            s.poll(s.submit(m), 60000)
        tickets = [None] * len(reqs)

        def collector():
            # every outstanding ticket is checked without blocking, so a request
            # is timed when its own result is ready, not when the ones submitted
            # before it are
            pend, nxt, done = [], 0, 0
            while done < len(reqs):
                while nxt < len(reqs) and tickets[nxt] is not None:
                    pend.append(nxt)
                    nxt += 1
                still = []
                for i in pend:
                    r = s.poll(tickets[i], 0)
                    if r is None:
                        still.append(i)
                    else:
                        res[i] = r
                        lat[i] = time.perf_counter() - (t0 + arrivals[i])
                        done += 1
                pend = still
                time.sleep(0.0002)
        t0 = time.perf_counter()
        th = threading.Thread(target=collector)
        th.start()
        for i, m in enumerate(mats):
            delay = t0 + arrivals[i] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets[i] = s.submit(m)
        th.join()
        wall = time.perf_counter() - t0
        st = s.stats()   # the server's own submit -> result-ready latencies
        # capacity: the first `sequential_seconds` of requests submitted at once
        nseq = sum(1 for t in arrivals if t < sequential_seconds)
        t1 = time.perf_counter()
        for t in [s.submit(m) for m in mats[:nseq]]:
            s.poll(t, -1)
        cap_server = nseq / (time.perf_counter() - t1)
    t1 = time.perf_counter()
    seq = [A.permanent(m) for m in mats[:nseq]]
    cap_seq = nseq / (time.perf_counter() - t1)
    q = lambda v, p: float(np.percentile(np.array(v) * 1e3, p))
    mism = sum(1 for r, z in zip(res[:nseq], seq) if r.status or z.status or
               (r.value != z.value if r.vtype == 1 else rel(r.value, z.value) > 1e-9))
    out = {"metric": "served permanents/s with p50/p99 latency (Poisson %g req/s)" % rate,
           "perms_per_s": len(reqs) / wall, "requests": len(reqs), "seconds": wall,
           "p50_ms": q(lat, 50), "p99_ms": q(lat, 99), "max_ms": q(lat, 100),
           "server_side_ms": {"p50": st.p50_ms, "p99": st.p99_ms, "max": st.max_ms,
                              "note": "perm_server_stats: submit to result ready, inside the library"},
           "failed": sum(1 for r in res if r.status != 0),
           "max_ms_by_n": {str(n): round(max(l for l, rq in zip(lat, reqs) if rq.a.shape[0] == n) * 1e3, 2)
                           for n in sorted({rq.a.shape[0] for rq in reqs})},
           "double_double_reruns": sum(1 for r in res if r.precision == 2),
           "workload": "Poisson arrivals at %g req/s for %g s, n = 16 + m with P(m) ~ 2^-m up to 40, p uniform in "
                       "[0.1,0.3] + diagonal, mixed 0/1 and (0,1], seed 5" % (rate, duration),
           "capacity_perms_per_s": {"server": cap_server, "per_request_plans": cap_seq, "ratio": cap_server / cap_seq,
                                    "requests": nseq,
                                    "note": "the first %g s of requests submitted at once; per_request_plans: "
                                            "plan + launch + sync + destroy per request, back to back"
                                            % sequential_seconds},
           "agreement_vs_per_request": {"mismatches": mism, "compared": nseq}}
    if accuracy:
        out["accuracy_vs_oracle"] = accuracy_sample([r.a for r in reqs], res, [r.values for r in reqs], count=60)
    return out


def run_batch(args):
    import torch
    from paper_2501_15126_gb300 import _abi as A
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    print(json.dumps(measure_batch(A, stream.cuda_stream, args.batch_count, args.steps, args.warmup)))
    return 0


def run_serving(args):
    import torch
    from paper_2501_15126_gb300 import _abi as A
    torch.cuda.set_device(0)
    print(json.dumps(measure_serving(A, args.rate, args.duration)))
    return 0


def run_band48(args):
    """The n=48 band workload in full (2^47 Gray steps per permanent), exact,
    through checkpointed slices: the band |i-j| <= 3 plus 2 off-band nonzeros
    per row (0/1) in the Algorithm 3 order and in the degree order -- the
    permanent does not depend on the column order (Sec. V), so the two must be
    the same integer -- and its band-only sibling, checked against the banded
    dynamic program of the oracle.  Checkpoint files go to --ckpt-dir, so an
    interrupted run resumes where it stopped."""
    import torch
    import oracle
    from paper_2501_15126_gb300 import _abi as A
    from paper_2501_15126_gb300 import synth
    torch.cuda.set_device(0)
    os.makedirs(args.ckpt_dir, exist_ok=True)
    a01 = synth.band_plus(48, 3, 2, seed=3, values="01")
    band = synth.band_plus(48, 3, 0, seed=3, values="01")
    runs = [("band_offband_alg3", a01, A.PERM_ORDER_PAPER), ("band_offband_degree", a01, A.PERM_ORDER_DEGREE),
            ("band_only", band, A.PERM_ORDER_AUTO)]
    out = {"workload": "n=48 band |i-j|<=3 + 2 off-band nonzeros per row, 0/1 values, seed 3 (and its band-only "
                       "sibling); whole 2^47-step walks, exact", "slice_log2": args.slice_log2, "runs": {}}
    for name, a, order in runs:
        path = os.path.join(args.ckpt_dir, "band48_%s.ckpt" % name)
        t0 = time.time()
        st, r = A.checkpoint_run(a, path, slice_log2=args.slice_log2, max_slices=args.max_slices,
                                 ordering=order, engine=A.PERM_ENGINE_CODEGEN)
        rec = {"status": "done" if st == A.PERM_OK else "partial", "gray_steps_done": r.steps,
               "wall_s_this_call": time.time() - t0, "kernel_s_this_call": r.ms_kernel / 1e3,
               "ordering": r.ordering, "exact_words": r.exact_words}
        if st == A.PERM_OK:
            rec["permanent"] = str(r.value)
            if name == "band_only":
                want = oracle.band_dp_int(a, 3)
                rec["band_dp"] = str(want)
                rec["matches_band_dp"] = r.value == want
        out["runs"][name] = rec
        print(json.dumps({name: rec}), flush=True)
    ra, rd = out["runs"]["band_offband_alg3"], out["runs"]["band_offband_degree"]
    if "permanent" in ra and "permanent" in rd:
        out["orders_agree"] = ra["permanent"] == rd["permanent"]
    print(json.dumps(out))
    return 0


def run_ablation(args):
    """The paper's ablation (Sec. VI-B, Table III, Fig. 4) on GB300: the
    library's generated kernel (product chain, two-state chains) against
    CodeGen-PureReg (a full product every step, x in registers) and
    GPU-SparsePerman (x in shared memory, a full product every step, zero
    tracking), on the n=36 workload (whole walk) and an n=40 ER p=0.1 matrix
    (the paper's smallest Table III shape; a 2^36-step prefix).  Kernel time by
    CUDA events (best of 3 after a warm-up), all in FP64; then the host-only
    ordering report of Fig. 4 (register rows k and columns c of Algorithm 4,
    and operations per step, without and with Algorithm 3)."""
    import torch
    from paper_2501_15126_gb300 import _abi as A
    from paper_2501_15126_gb300 import synth
    torch.cuda.set_device(0)
    cases = [("n36_workload", workload_matrix(), 0, 0),
             ("n40_er_p0.1", synth.single_er(40, 0.1, 40, values="f64"), 0, 1 << 36)]
    engines = [("codegen_chain", dict(engine=A.PERM_ENGINE_CODEGEN)),
               ("codegen_pure_reg", dict(engine=A.PERM_ENGINE_CODEGEN, flags=A.PERM_FLAG_PURE_REG)),
               ("generic_chain", dict(engine=A.PERM_ENGINE_GENERIC)),
               ("x_shared", dict(engine=A.PERM_ENGINE_XSHARED, ordering=A.PERM_ORDER_DEGREE))]
    out = {"workload": "ablation", "cases": {}}
    for name, a, lo, hi in cases:
        rec = {}
        for ename, kw in engines:
            p = A.Plan(a, g_lo=lo, g_hi=hi, precision=A.PERM_PREC_F64, **kw)
            r = p.compute()
            ms = min(p.compute().ms_kernel for _ in range(3))
            rec[ename] = {"ms": ms, "gray_steps_per_s": r.steps / (ms / 1e3), "value": r.value,
                          "ops_per_step_model": r.fp_ops_per_step, "regs": r.regs_per_thread,
                          "threads": r.threads, "zero_skip_frac": r.zero_skip_frac}
            p.close()
        base = rec["codegen_chain"]["ms"]
        for ename in rec:
            rec[ename]["chain_speedup_over_this"] = rec[ename]["ms"] / base
        if not hi:   # whole walks agree up to rounding (a prefix's partial sum depends on the column order)
            vals = [rec[e]["value"] for e in rec]
            rec["max_rel_spread_of_values"] = (max(vals) - min(vals)) / abs(vals[0])
        rec["gray_steps"] = (hi - lo) if hi else 1 << (a.shape[0] - 1)
        out["cases"][name] = rec
        print(json.dumps({name: rec}), flush=True)
    fig4 = {}
    for name, a, _, _ in cases:
        rows = {}
        for oname, o in (("none", A.PERM_ORDER_NONE), ("degree", A.PERM_ORDER_DEGREE), ("algorithm3", A.PERM_ORDER_PAPER)):
            ins = A.inspect(a, ordering=o)
            rows[oname] = {"reg_rows_k": ins.reg_rows, "reg_cols_c": ins.reg_cols,
                           "ops_per_step_chain": ins.ops_per_step, "ops_per_step_full_product": ins.ops_per_step_paper,
                           "ops_per_step_walk": ins.ops_per_step_walk}
        fig4[name] = rows
    out["fig4_ordering"] = fig4
    print(json.dumps(out))
    return 0


# Table III: CodeGen-Hybrid on the real matrices, seconds on an A100 (the paper's numbers; other
# matrices with these shapes and another GPU: context only)
PAPER_TABLE3_HYBRID_S = {"bcsstk01": 882.94, "mycielskian6": 477.75, "mesh1e1": 860.19, "d_ss": 21448.17,
                         "curtis54": 47841.18, "bcspwr02": 1317.42}


def zero_product_fraction(a, samples=1 << 16, seed=11):
    """Fraction of the 2^(n-1) Gray-walk terms whose product has a zero factor,
    estimated from uniformly drawn column subsets (host, numpy)."""
    n = a.shape[0]
    a = a.astype(np.float64)
    x0 = a[:, n - 1] - 0.5 * a.sum(axis=1)
    g = np.random.default_rng(seed)
    S = (g.random((samples, n - 1)) < 0.5).astype(np.float64)
    return float(((x0[None, :] + S @ a[:, : n - 1].T) == 0).any(axis=1).mean())


def measure_table2(A, seconds_per_range=0.25, cpu_seconds=1.0):
    """Matrices with the shapes of the paper's real-life set (Table II; values
    as Sec. VI-E describes them): the library's default plan timed by CUDA
    events on four Gray sub-ranges spread over the walk (their sizes picked
    for about `seconds_per_range` each), the fraction of blocks the zero skip
    removed, the fraction of zero products (host sample), the projected time
    of the whole walk, and CPU-SparsePerman (FP64, zero tracking) on a prefix.
    The bcspwr02 shape's whole walk (n = 49) is computed and compared with the
    oracle's row-expansion DP."""
    from paper_2501_15126_gb300 import synth
    out = {"workload": "table2", "note": "random matrices with Table II's n, nnz, symmetry and value structure "
                                         "(not the SuiteSparse matrices)", "matrices": {}}
    for sh in synth.TABLE2_SHAPES:
        a = synth.table2_like(sh.name)
        n = a.shape[0]
        top = 1 << (n - 1)
        p = A.Plan(a, g_lo=0, g_hi=1 << 30)
        p.compute()
        r = p.compute()
        p.close()
        k = int(np.clip(np.floor(np.log2(max(r.steps / (r.ms_kernel / 1e3), 1.0) * seconds_per_range)), 30, n - 3))
        ms, steps, skipped, first = 0.0, 0, 0.0, None
        for i in range(4):
            lo = (i * (top >> 2)) >> k << k
            p = A.Plan(a, g_lo=lo, g_hi=lo + (1 << k))
            p.compute()
            r = p.compute()
            p.close()
            first = first or r
            ms += r.ms_kernel
            steps += r.steps
            skipped += r.zero_skip_frac * r.steps
        rate = steps / (ms / 1e3)
        cpu = cpu_fp64_baseline(a.astype(np.float64), seconds_hint=cpu_seconds)
        rec = {"n": n, "nnz": int(np.count_nonzero(a)), "values": sh.values,
               "arithmetic": "exact (%d-bit ring)" % (64 * first.exact_words) if first.vtype == A.PERM_I64 else "fp64",
               "engine": "codegen" if first.engine == A.PERM_ENGINE_CODEGEN else "generic",
               "regs": first.regs_per_thread, "chunk_log2": first.chunk_log2,
               "ranges": "4 x 2^%d steps at 0, 1/4, 1/2, 3/4 of the walk" % k,
               "gray_steps_per_s": rate, "zero_skip_frac": skipped / steps,
               "zero_product_frac": zero_product_fraction(a),
               "projected_whole_walk_s": top / rate,
               "paper_table3_hybrid_s_a100_real_matrix": PAPER_TABLE3_HYBRID_S[sh.name],
               "cpu_sparseperman_fp64_steps_per_s": cpu["value"], "cpu_cores": cpu["cores"],
               "gpu_over_cpu": rate / cpu["value"]}
        out["matrices"][sh.name] = rec
    import oracle
    a = synth.table2_like("bcspwr02")
    t0 = time.perf_counter()
    r = A.permanent(a)
    wall = time.perf_counter() - t0
    want = oracle.rowdp_int(a)
    out["bcspwr02_whole_walk"] = {"n": 49, "gray_steps": 1 << 48, "value": str(r.value), "oracle_rowdp": str(want),
                                  "matches": r.value == want, "ms_kernel": r.ms_kernel, "seconds_end_to_end": wall,
                                  "zero_skip_frac": r.zero_skip_frac,
                                  "note": "exact walk of all 2^48 Gray steps; oracle: Eq. 1 expanded row by row"}
    return out


def run_table2(args):
    import torch
    from paper_2501_15126_gb300 import _abi as A
    torch.cuda.set_device(0)
    out = measure_table2(A, cpu_seconds=2.0)
    for name, rec in out["matrices"].items():
        print(json.dumps({name: rec}), flush=True)
    print(json.dumps(out))
    return 0


def run_profile_case(args):
    """A small case of the bench kernel for `ncu --set full`: the same matrix,
    plan and generated kernel, walking only the Gray sub-range [0, 2^k)."""
    import torch
    from paper_2501_15126_gb300 import _abi as A
    torch.cuda.set_device(0)
    from paper_2501_15126_gb300 import synth
    vals = "01" if args.profile_exact else "f64"
    if args.profile_matrix == "batch28":
        # the largest class of the batch workload: its first n=28 matrix with these values
        a = next(it.a for it in synth.batch(count=400) if it.a.shape[0] == 28 and it.values == vals)
    elif args.profile_matrix in [t.name for t in synth.TABLE2_SHAPES]:
        a = synth.table2_like(args.profile_matrix)
        vals = "01" if a.dtype == np.int64 else "f64"
    elif args.profile_exact or args.profile_matrix == "band48":
        a = synth.band_plus(48, 3, 2, seed=3, values=vals)
    else:
        a = workload_matrix()
    engine = A.PERM_ENGINE_GENERIC if args.profile_engine == "generic" else A.PERM_ENGINE_CODEGEN
    n = a.shape[0]
    # a prefix of the walk, or (when it covers the range) the whole walk with its own ring width
    g_hi = 0 if args.profile_log2 >= n - 1 else 1 << args.profile_log2
    p = A.Plan(a, g_lo=0, g_hi=g_hi, engine=engine, flags=A.PERM_FLAG_PAIRED_CHAIN if args.profile_paired else 0,
               chunk_log2=args.profile_chunk_log2)
    for _ in range(args.steps):
        r = p.compute()
    print(json.dumps({"profile_case": vals, "matrix": args.profile_matrix, "n": n, "engine": args.profile_engine,
                      "gray_steps": r.steps, "ms_kernel": r.ms_kernel,
                      "ops_per_step": r.fp_ops_per_step, "threads": r.threads, "regs": r.regs_per_thread,
                      "chunk_log2": r.chunk_log2, "zero_skip_frac": r.zero_skip_frac}))
    p.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shard", action="store_true",
                    help="N > 1: split each permanent's Gray range across the ranks (strong scaling) "
                         "instead of one permanent per rank")
    ap.add_argument("--no-extras", action="store_true",
                    help="single workload: only the headline (no batch, serving, accuracy, cold e2e, FP64 CPU baseline)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--workload", default="single", choices=["single", "batch", "serving", "profile", "band48", "ablation",
                                                             "table2"])
    ap.add_argument("--ckpt-dir", default=os.path.join(tempfile.gettempdir(), "perm_band48_ckpt"),
                    help="band48: checkpoint files")
    ap.add_argument("--slice-log2", type=int, default=40, help="band48: Gray indices per checkpointed slice (log2)")
    ap.add_argument("--max-slices", type=int, default=0, help="band48: slices per run per call (0 = all)")
    ap.add_argument("--profile-log2", type=int, default=30)
    ap.add_argument("--profile-exact", action="store_true")
    ap.add_argument("--profile-chunk-log2", type=int, default=0, help="profile: K (0 = the plan's choice)")
    ap.add_argument("--profile-engine", default="codegen", choices=["codegen", "generic"])
    ap.add_argument("--profile-matrix", default="bench", choices=["bench", "batch28", "band48", "bcsstk01",
                                                                  "mycielskian6", "mesh1e1", "bcspwr02", "curtis54",
                                                                  "d_ss"],
                    help="bench: the n=36 bench matrix (the n=48 band with --profile-exact); "
                         "batch28: an n=28 matrix of the batch workload; band48: the n=48 band-plus-off-band matrix; "
                         "the Table II shape names: that suite's matrix")
    ap.add_argument("--profile-paired", action="store_true",
                    help="generated FP64 kernels: the paired chain even where two-state chains are cheaper")
    ap.add_argument("--batch-count", type=int, default=10_000)
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--duration", type=float, default=60.0)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    import __graft_entry__
    __graft_entry__.build()
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "profile":
        return run_profile_case(args)
    if args.workload == "band48":
        return run_band48(args)
    if args.workload == "table2":
        return run_table2(args)
    if args.workload == "ablation":
        return run_ablation(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
