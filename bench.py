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
    for name in ("core.cuh", "codegen.cpp", "devmat.h"):
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
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    import __graft_entry__
    __graft_entry__.build()
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
