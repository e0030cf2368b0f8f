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
    h = hashlib.sha256()
    # the walk code, the generator, and the host code that picks layout and scheme
    for name in ("core.cuh", "codegen.cpp", "devmat.h", "host.cpp", "api.cpp"):
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


def config_block(engine, steps_per_step):
    return {"workload": "single real sparse matrix n=36: ER p=0.15 + forced diagonal, (0,1] values, shuffled "
                        "columns, seed 2", "n": 36, "gray_steps_per_step": steps_per_step, "engine": engine,
            "l2": "flushed between steps (256 MiB device write)", "parallelism": "replicas (one matrix per GPU)"}


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
    plan = A.Plan(a)                       # ordering, partitioning, NVRTC (warm-up region)
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
    if world > 1:
        from paper_2501_15126_gb300 import dist as pd
        total_ms = pd.max_over_ranks(total_ms, device=dev)
        torch.distributed.barrier()

    # end to end through the public API from host memory, every step
    e2e_ms = []
    for _ in range(max(1, min(args.steps, 3))):
        t0 = time.perf_counter()
        rr = A.permanent(a, stream=sh)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
        assert rr.value == first.value
    plan_engine = "codegen" if first.engine == A.PERM_ENGINE_CODEGEN else "generic"

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0
    value = world * args.steps * GRAY_STEPS / (total_ms / 1e3)
    mean_kernel_ms = statistics.mean(kern_ms)
    ops = first.fp_ops_per_step * GRAY_STEPS
    achieved = ops / (mean_kernel_ms / 1e3)
    kh = kernel_hash()
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_block(plan_engine, GRAY_STEPS),
        "ms_per_permanent": total_ms / args.steps,
        "permanent": first.value,
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
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(a, args.cpu_seconds)
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_batch(args):
    """The 10,000-matrix workload: one persistent launch per kernel family
    (perm_batch) against one plan and launch per matrix (perm_batch_sequential)."""
    import torch
    from paper_2501_15126_gb300 import _abi as A
    from paper_2501_15126_gb300 import synth
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    items = synth.batch(count=args.batch_count)
    mats = [A.CSRMatrix(it.a) for it in items]
    steps_total = sum(1 << (it.n - 1) for it in items)
    for _ in range(max(args.warmup, 1)):
        A.batch(mats, stream=stream.cuda_stream)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        res = A.batch(mats, stream=stream.cuda_stream)
        times.append(time.perf_counter() - t0)
    # the two arithmetic halves on their own (each is its own kernel family)
    split = {}
    for vals in ("f64", "01"):
        sub = [m for m, it in zip(mats, items) if it.values == vals]
        sub_steps = sum(1 << (it.n - 1) for it in items if it.values == vals)
        t0 = time.perf_counter()
        A.batch(sub, stream=stream.cuda_stream)
        dt = time.perf_counter() - t0
        split[vals] = {"count": len(sub), "seconds": dt, "gray_steps_per_s": sub_steps / dt}
    seq_t0 = time.perf_counter()
    seq = A.batch(mats, sequential=True, stream=stream.cuda_stream)
    seq_time = time.perf_counter() - seq_t0
    mism_exact = sum(1 for r, q, it in zip(res, seq, items) if it.values == "01" and r.value != q.value)
    mism_f64 = sum(1 for r, q, it in zip(res, seq, items)
                   if it.values == "f64" and abs(r.value - q.value) > 1e-9 * abs(q.value))
    max_rel_f64 = max((abs(r.value - q.value) / abs(q.value) for r, q, it in zip(res, seq, items)
                       if it.values == "f64"), default=0.0)
    best = min(times)
    line = {"metric": "batched permanents/s (10,000 matrices, n in [12,28])", "value": len(items) / best,
            "unit": "perms/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * best, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64+exact", "data": "synthetic",
            "config": {"workload": "batch of %d ER matrices, n uniform in [12,28], p uniform in [0.2,0.4] + forced "
                                   "diagonal, alternating 0/1 (exact) and (0,1] (FP64), seed 4" % len(items),
                       "gray_steps_total": steps_total, "l2": "inputs re-uploaded every step"},
            "gray_steps_per_s": steps_total / best, "by_arithmetic": split,
            "sequential": {"seconds": seq_time, "perms_per_s": len(items) / seq_time,
                           "note": "perm_batch_sequential: plan + launch + sync + destroy per matrix"},
            "speedup_vs_sequential": seq_time / best,
            "agreement_vs_sequential": {"exact_mismatches": mism_exact, "f64_beyond_1e-9": mism_f64,
                                        "f64_max_rel_diff": max_rel_f64},
            "kernel_ms": res[0].ms_kernel}
    print(json.dumps(line))
    return 0


def run_serving(args):
    """Open-loop replay of the Poisson serving stream against the server, and
    the same arrivals served by one plan + launch per request in order."""
    import torch
    from paper_2501_15126_gb300 import _abi as A
    from paper_2501_15126_gb300 import synth
    torch.cuda.set_device(0)
    reqs = synth.serving_stream(rate=args.rate, duration=args.duration, seed=5)
    mats = [A.CSRMatrix(r.a) for r in reqs]
    arrivals = [r.t_arrival for r in reqs]

    def replay_server():
        lat = [None] * len(reqs)
        res = [None] * len(reqs)
        with A.Server() as s:
            # warm the families up
            for m in mats[:50]:
                s.poll(s.submit(m), 60000)
            tickets = [None] * len(reqs)
            done_evt = threading.Event()

            def collector():
                for i in range(len(reqs)):
                    while tickets[i] is None:
                        time.sleep(0.0001)
                    r = s.poll(tickets[i], -1)
                    lat[i] = time.perf_counter() - (t0 + arrivals[i])
                    res[i] = r
                done_evt.set()
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
        return lat, res, wall

    def replay_sequential():
        lat = [None] * len(reqs)
        res = [None] * len(reqs)
        t0 = time.perf_counter()
        for i, m in enumerate(mats):
            delay = t0 + arrivals[i] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            res[i] = A.permanent(m)
            lat[i] = time.perf_counter() - (t0 + arrivals[i])
        return lat, res, time.perf_counter() - t0

    def capacity_server():
        """Closed loop: every request submitted at once; time until all are done."""
        with A.Server() as s:
            for m in mats[:50]:
                s.poll(s.submit(m), 60000)
            t0 = time.perf_counter()
            tickets = [s.submit(m) for m in mats]
            for t in tickets:
                s.poll(t, -1)
            return len(mats) / (time.perf_counter() - t0)

    def capacity_sequential():
        t0 = time.perf_counter()
        for m in mats:
            A.permanent(m)
        return len(mats) / (time.perf_counter() - t0)

    ls, rs, ws = replay_server()
    lq, rq, wq = replay_sequential()
    cap_s = capacity_server()
    cap_q = capacity_sequential()
    q = lambda v, p: float(np.percentile(np.array(v) * 1e3, p))
    bad = [(i, reqs[i].a.shape[0], reqs[i].values, a.status, a.value, b.value) for i, (a, b) in enumerate(zip(rs, rq))
           if a.status or b.status or (a.value != b.value if a.vtype == 1 else abs(a.value - b.value) > 1e-9 * abs(b.value))]
    mism = len(bad)

    def terms_bound(a):
        # sum of |Nijenhuis-Wilf terms| <= 2^(n-1) prod_i (sum_j |a_ij| / 2) = prod_i rowsum_i / 2
        return float(np.prod(np.abs(a).sum(axis=1))) / 2.0

    # FP64 differences beyond 1e-9 relative that are also beyond 1e-12 of the a-priori bound on
    # sum |terms| (64 n u sum|terms| < 1e-12 sum|terms| for n <= 48): an ill-conditioned permanent
    # (heavy cancellation) cannot be resolved to 1e-9 of itself in FP64 by any summation order
    beyond_bound = sum(1 for i, n, v, _, x, y in bad
                       if v != "01" and abs(x - y) > 1e-12 * terms_bound(reqs[i].a))
    line = {"metric": "served permanents/s with p50/p99 latency (Poisson 2,000 req/s)",
            "value": len(reqs) / ws, "unit": "perms/s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": 1e3 * ws, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64+exact", "data": "synthetic",
            "config": {"workload": "Poisson arrivals at %g req/s for %g s (%d requests), n = 16 + m with P(m) ~ 2^-m "
                                   "up to 40, p uniform in [0.1,0.3] + diagonal, mixed 0/1 and (0,1], seed 5"
                                   % (args.rate, args.duration, len(reqs))},
            "p50_ms": q(ls, 50), "p99_ms": q(ls, 99), "max_ms": q(ls, 100),
            "sequential": {"perms_per_s": len(reqs) / wq, "p50_ms": q(lq, 50), "p99_ms": q(lq, 99),
                           "max_ms": q(lq, 100)},
            "capacity_perms_per_s": {"server": cap_s, "sequential": cap_q, "ratio": cap_s / cap_q,
                                     "note": "closed loop: the same requests submitted all at once"},
            "mismatches_vs_sequential": mism, "mismatch_examples": [list(map(str, b)) for b in bad[:5]],
            "f64_mismatches_beyond_terms_bound": beyond_bound}
    print(json.dumps(line))
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
    elif args.profile_exact or args.profile_matrix == "band48":
        a = synth.band_plus(48, 3, 2, seed=3, values=vals)
    else:
        a = workload_matrix()
    engine = A.PERM_ENGINE_GENERIC if args.profile_engine == "generic" else A.PERM_ENGINE_CODEGEN
    n = a.shape[0]
    # a prefix of the walk, or (when it covers the range) the whole walk with its own ring width
    g_hi = 0 if args.profile_log2 >= n - 1 else 1 << args.profile_log2
    p = A.Plan(a, g_lo=0, g_hi=g_hi, engine=engine, flags=A.PERM_FLAG_PAIRED_CHAIN if args.profile_paired else 0)
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
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--workload", default="single", choices=["single", "batch", "serving", "profile"])
    ap.add_argument("--profile-log2", type=int, default=30)
    ap.add_argument("--profile-exact", action="store_true")
    ap.add_argument("--profile-engine", default="codegen", choices=["codegen", "generic"])
    ap.add_argument("--profile-matrix", default="bench", choices=["bench", "batch28", "band48"],
                    help="bench: the n=36 bench matrix (the n=48 band with --profile-exact); "
                         "batch28: an n=28 matrix of the batch workload; band48: the n=48 band-plus-off-band matrix")
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
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
