#!/usr/bin/env python
"""Benchmark of the PACO hot path on GB300.

Workload: one complex64 1-D DFT of N = 2^28 as N1 = N2 = 2^14, radix b = 4,
p = 64 virtual slabs, forward (w^{-kj}); input Re/Im i.i.d. U[-1, 1) from
seed (rank).  One step = one pass of the whole path: Phase I with the fused
twiddle + digit-reversal redistribution (stage 1), then Phase III (stage 2),
exactly the two launches paco_execute makes.  The input (2 GiB) is larger
than L2, so no flush is needed between steps.

Reported: 5 N log2 N GFLOP/s (whole job), effective HBM GB/s (32 N bytes per
step: two reads and two writes of N complex64), the dominant kernel's
roofline against the measured copy bandwidth, an end-to-end number through
paco_execute_host with pinned host buffers, the CPU oracle on a bounded
sample, and SM clocks sampled during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl paco|reference]

Under torchrun each rank runs an independent replica on its own GPU (the
transform does not shard across GPUs on this path); timing is the max over
ranks and `value` is the total over ranks.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "5N·log2N GFLOP/s + HBM GB/s, N=2^28 c64; TC-split vs plain FP32 at matched error"


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["paco", "reference"], default="paco")
    ap.add_argument("--lg1", type=int, default=14, help="log2 N1")
    ap.add_argument("--lg2", type=int, default=14, help="log2 N2")
    ap.add_argument("--b", type=int, default=4)
    ap.add_argument("--p", type=int, default=64)
    ap.add_argument("--dtype", choices=["c64", "c128"], default="c64")
    ap.add_argument("--dir", type=int, default=-1, choices=[-1, 1])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-lg", type=int, default=24, help="log2 size of the oracle sample")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, interval_ms: int = 100):
        self.gpu = gpu_index
        self.interval = interval_ms
        self.proc = None
        self.file = None
        self.t_start = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", str(self.interval)],
                stdout=self.file, stderr=subprocess.DEVNULL)
            self.t_start = time.time()
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self, t_begin: float, t_end: float):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [l.strip().split(",") for l in self.file.read().splitlines() if l.strip()]
        self.file.close()
        os.unlink(self.file.name)
        n = len(rows)
        if n == 0:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        # samples are evenly spaced from t_start; keep those inside the timed region
        dt = self.interval / 1000.0
        idx = [i for i in range(n) if t_begin - dt <= self.t_start + i * dt <= t_end + dt]
        used = [rows[i] for i in idx] or rows
        sm = []
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        mx = None
        for r in used:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(used)}


# ---------------------------------------------------------------------------
# CPU oracle leg
# ---------------------------------------------------------------------------
def oracle_sample(lg: int, seconds: float, dtype: str):
    """Time the CPU oracle (FP64 recursive FFT, as it stands) on one 2^lg
    transform of the same recipe, repeated until `seconds` of work."""
    import numpy as np

    import oracle
    from paco_inputs import uniform

    n = 1 << lg
    x = uniform(n, 0, np.complex64 if dtype == "c64" else np.complex128).astype(np.complex128)
    oracle.fft(x[:16], threads=1)          # build + load outside the timing
    reps, total = 0, 0.0
    while total < seconds or reps == 0:
        t = time.perf_counter()
        oracle.fft(x, threads=1)
        total += time.perf_counter() - t
        reps += 1
    per = total / reps
    gflops = 5.0 * n * lg / per / 1e9
    return gflops, per, reps


def run_reference(args, rank: int, world: int):
    """The reference arm: the CPU oracle as it stands, on the machine's host cores
    (rank 0 only), each step one bounded sample of the workload: a 2^lg-point
    transform of the same recipe, lg chosen so K + W steps take a few minutes."""
    if rank != 0:
        return
    k = max(args.steps, 1) + max(args.warmup, 0)
    lg = 24 if k <= 12 else 22 if k <= 60 else 20 if k <= 300 else 18
    import numpy as np

    import oracle
    from paco_inputs import uniform

    n = 1 << lg
    x = uniform(n, 0, np.complex64).astype(np.complex128)
    for _ in range(max(args.warmup, 0)):
        oracle.fft(x, threads=1)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.fft(x, threads=1)
    el = time.perf_counter() - t
    per = el / max(args.steps, 1)
    v = 5.0 * n * lg / per / 1e9
    sample = (f"one 2^{lg}-point transform per step (same U[-1,1) recipe, seed 0), "
              f"FP64 recursive radix-2 oracle, 1 thread")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "GFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": v, "unit": "GFLOP/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


class Ranks:
    """The rank context of a bench run: one process per GPU under torchrun,
    a single process otherwise.  `barrier`, `max_over_ranks` and
    `job_value` are the only cross-rank operations (no data-path
    collective: every rank runs an independent replica)."""

    def __init__(self, backend: str | None = None, device=None):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None
        self.device = device
        if self.world > 1:
            import torch
            import torch.distributed as dist_mod
            if not dist_mod.is_initialized():
                if backend == "nccl":
                    dist_mod.init_process_group("nccl", device_id=torch.device("cuda", self.local))
                else:
                    dist_mod.init_process_group(backend or "gloo")
            self.dist = dist_mod

    def barrier(self) -> None:
        if self.dist is not None:
            self.dist.barrier()

    def max_over_ranks(self, v: float) -> float:
        if self.dist is None:
            return v
        import torch
        t = torch.tensor([v], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def job_value(self, units_per_rank: float, seconds_per_step: float) -> float:
        """Whole-job throughput: the units every rank processed in one step
        over the slowest rank's step time."""
        return units_per_rank * self.world / self.max_over_ranks(seconds_per_step)

    def close(self) -> None:
        if self.dist is not None:
            self.dist.destroy_process_group()


def workload_config(args):
    N1, N2 = 1 << args.lg1, 1 << args.lg2
    return {
        "workload": f"{args.dtype} 1-D DFT N=2^{args.lg1 + args.lg2} as N1=2^{args.lg1} x N2=2^{args.lg2}, "
                    f"b={args.b}, p={args.p}, {'forward' if args.dir == -1 else 'conjugate'}",
        "N1": N1, "N2": N2, "b": args.b, "p": args.p, "batch": 1, "dir": args.dir,
        "input": "Re, Im i.i.d. U[-1,1), seed = rank",
        "l2": "inputs larger than L2 (no flush)",
    }


def captured_traffic(stage: str, N1: int, N2: int, b: int, p: int, dtype: str, dir: int):
    """DRAM bytes per launch of the panel kernel from the committed ncu
    capture (profiles/roofline_traffic.json), or None when the workload differs
    or the kernel source changed since the counters were taken."""
    import hashlib
    if (N1, N2, b, p, dtype, dir) != (1 << 14, 1 << 14, 4, 64, "c64", -1):
        return None
    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as fh:
            rec = json.load(fh)
        csrc = os.path.join(ROOT, "paper_2609_06449_gb300", "csrc")
        h = hashlib.sha256()
        for name in ("paco_panel.cuh", "paco_common.cuh"):
            with open(os.path.join(csrc, name), "rb") as fh:
                h.update(fh.read())
        if h.hexdigest()[:16] != rec["source_sha16"]:
            return None
        return float(rec["traffic_bytes_per_launch"][stage])
    except (OSError, KeyError, ValueError):
        return None


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------
def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch

    import paper_2609_06449_gb300 as paco
    from paco_inputs import uniform

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    ranks = Ranks("nccl", device="cuda")
    barrier, max_over_ranks = ranks.barrier, ranks.max_over_ranks

    N1, N2 = 1 << args.lg1, 1 << args.lg2
    N = N1 * N2
    lgN = args.lg1 + args.lg2
    dt = paco.C64 if args.dtype == "c64" else paco.C128
    npdt = np.complex64 if args.dtype == "c64" else np.complex128
    esize = 8 if args.dtype == "c64" else 16
    plan = paco.Plan(N1, N2, args.b, 1, dt, p=args.p)

    x_host = torch.from_numpy(uniform(N, rank, npdt)).pin_memory()
    x = x_host.to("cuda", non_blocking=False)
    out = torch.empty_like(x)
    stream = torch.cuda.current_stream()

    for _ in range(max(args.warmup, 3)):
        plan.execute_stage1(x, out, args.dir, stream)
        plan.execute_stage2(out, out, args.dir, stream)
    torch.cuda.synchronize()
    plan.check()

    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    t_begin = time.time()
    for k in range(K):
        ev[k][0].record(stream)
        plan.execute_stage1(x, out, args.dir, stream)
        ev[k][1].record(stream)
        plan.execute_stage2(out, out, args.dir, stream)
        ev[k][2].record(stream)
    torch.cuda.synchronize()
    t_end = time.time()
    barrier()
    clocks = sampler.stop(t_begin, t_end)
    plan.check()

    total_ms = ev[0][0].elapsed_time(ev[K - 1][2])
    s1 = [ev[k][0].elapsed_time(ev[k][1]) for k in range(K)]
    s2 = [ev[k][1].elapsed_time(ev[k][2]) for k in range(K)]
    flop = 5.0 * N * lgN
    value = ranks.job_value(flop / 1e9, total_ms / K * 1e-3)
    ms_step = max_over_ranks(total_ms) / K
    hbm_eff = 4.0 * N * esize * world / (ms_step * 1e-3) / 1e9

    avg1, avg2 = statistics.mean(s1), statistics.mean(s2)
    dom, dom_ms, dom_key = ("stage1 (Phase I + fused PARA-CO-DRP)", avg1, "stage1") if avg1 >= avg2 else \
        ("stage2 (Phase III)", avg2, "stage2")
    traffic = captured_traffic(dom_key, N1, N2, args.b, args.p, args.dtype, args.dir)
    bytes_per_launch = 2.0 * N * esize            # read N + write N elements
    achieved = bytes_per_launch / (dom_ms * 1e-3) / 1e9
    peak, peak_src = measured_peak_hbm()

    # end to end: host buffers through paco_execute_host (H2D + execute + D2H)
    e2e = None
    if not args.no_e2e:
        h_out = torch.empty_like(x_host).pin_memory()
        d_in = torch.empty_like(x)
        for _ in range(2):
            plan.execute_host(x_host, h_out, d_in, out, args.dir, stream)
        torch.cuda.synchronize()
        KE = max(args.e2e_steps, 1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(KE):
            plan.execute_host(x_host, h_out, d_in, out, args.dir, stream)
        b.record(stream)
        torch.cuda.synchronize()
        e_ms = max_over_ranks(a.elapsed_time(b)) / KE
        e2e = {"value": flop * world / (e_ms * 1e-3) / 1e9, "unit": "GFLOP/s",
               "ms_per_step": e_ms,
               "h2d_bytes_per_step": N * esize, "d2h_bytes_per_step": N * esize,
               "api": "paco_execute_host (pinned host buffers)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            import oracle
            g, per, reps = oracle_sample(args.cpu_lg, args.cpu_seconds, args.dtype)
            cpu = {"value": g, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                   "sample": f"{reps} x one 2^{args.cpu_lg}-point transform (same recipe), "
                             f"FP64 recursive radix-2 oracle, 1 thread, {per:.2f} s each"}
        except Exception as e:  # report, do not hide
            cpu = {"value": None, "unit": "GFLOP/s", "cores": 0, "kind": "oracle",
                   "sample": f"failed: {e}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
            "steps": K, "warmup": max(args.warmup, 3), "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.dtype == "c64" else "f64", "data": "synthetic",
            "config": workload_config(args),
            "hbm_gbs_effective": hbm_eff,
            "stage_ms": {"stage1": avg1, "stage2": avg2},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                         "peak_source": peak_src, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic,
                         "algorithmic_bytes_per_launch": bytes_per_launch},
            "e2e": e2e, "cpu_baseline": cpu, "gpu_launches": 2 * K, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    ranks.close()


if __name__ == "__main__":
    main()
