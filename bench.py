#!/usr/bin/env python
"""Benchmark of the PACO hot path on GB300.

Default workload (the headline): one complex64 1-D DFT of N = 2^28 as
N1 = N2 = 2^14, radix b = 4, p = 64 virtual slabs, forward (w^{-kj}); input
Re/Im i.i.d. U[-1, 1) from seed (rank).  One step = one pass of the whole
path: Phase I with the fused twiddle + digit-reversal redistribution
(stage 1), then Phase III (stage 2), exactly the two launches paco_execute
makes.  The input (2 GiB) is larger than L2, so no flush is needed between
steps.  The same line carries the tensor-core sub-DFT forms (BF16x3 split,
FP16 per-block scaled) timed on the same transform, each with its relative
L2 error against the FP64 oracle.

Reported: 5 N log2 N GFLOP/s (whole job), effective HBM GB/s (32 N bytes per
step: two reads and two writes of N complex64), the dominant kernel's
roofline against the measured copy bandwidth, an end-to-end number through
paco_execute_host with pinned host buffers, the CPU oracle on a bounded
sample, SM clocks sampled during the timed region, and cuFFT on the same
input as context.

Other workloads (--workload): A (2^16 as 256 x 256, latency: one cluster
launch), B128 (complex128 N = 2^27), C (the uneven batch in one persistent
launch), D (16 x 2^24 per precision form), E (forward + backward of
256 x 2^20 with the weighted power loss fused into the stage kernels), T
(the 128-point sub-pass of a 2^14 stage on the tcgen05 tensor cores against
the plain FP32 kernel), U (the unfused three-pass pipeline Phase I ->
paco_permute -> Phase III on the headline transform: the ablation of the
fused redistribution), F3 (64 complex64 3-D DFTs of 256 x 64 x 64, the
dims = 3 plan, with cuFFT's fftn as context).  Each prints one line of the
same contract.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl paco|reference]
                  [--workload B|A|B128|C|D|E|T|U|F3] [--dir -1|1]

Under torchrun each rank runs an independent replica on its own GPU (the
sharded form's exchange is not timed on this pool's one-GPU machines); timing
is the max over ranks and `value` is the total over ranks.
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
    ap.add_argument("--workload", choices=["B", "A", "B128", "C", "D", "E", "U", "T", "F3"], default="B")
    ap.add_argument("--small", action="store_true",
                    help="a reduced case of the workload (C: 1024 lengths to 2^26 + 4096 x 2^12; D: batch 2; "
                         "U: N = 2^26; T: 2^24 points), for ncu captures")
    ap.add_argument("--no-autotune", action="store_true", help="C: fixed configuration instead of autotuning")
    ap.add_argument("--form", choices=["all", "plain", "bf16x3", "fp16"], default="all",
                    help="D: time only this precision form")
    ap.add_argument("--no-tc", action="store_true", help="skip the tensor-core forms on the headline line")
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
def oracle_sample(lg: int, seconds: float, dtype: str, threads: int = 1):
    """Time the CPU oracle (FP64 recursive FFT, as it stands) on one 2^lg
    transform of the same recipe, repeated until `seconds` of work, on
    `threads` OpenMP threads (its top recursion levels run as tasks)."""
    import numpy as np

    import oracle
    from paco_inputs import uniform

    n = 1 << lg
    x = uniform(n, 0, np.complex64 if dtype == "c64" else np.complex128).astype(np.complex128)
    oracle.fft(x[:16], threads=1)          # build + load outside the timing
    reps, total = 0, 0.0
    while total < seconds or reps == 0:
        t = time.perf_counter()
        oracle.fft(x, threads=threads)
        total += time.perf_counter() - t
        reps += 1
    per = total / reps
    gflops = 5.0 * n * lg / per / 1e9
    return gflops, per, reps


def host_cores() -> int:
    """The host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover - non-Linux
        return os.cpu_count() or 1


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
    cores = host_cores()
    x = uniform(n, 0, np.complex64).astype(np.complex128)
    for _ in range(max(args.warmup, 0)):
        oracle.fft(x, threads=cores)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.fft(x, threads=cores)
    el = time.perf_counter() - t
    per = el / max(args.steps, 1)
    v = 5.0 * n * lg / per / 1e9
    sample = (f"one 2^{lg}-point transform per step (same U[-1,1) recipe, seed 0), "
              f"FP64 recursive radix-2 oracle, {cores} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "GFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": v, "unit": "GFLOP/s", "cores": cores, "kind": "oracle", "sample": sample},
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


def fp64_peak_measured(paco, gpu_index: int):
    """The FP64 FMA rate of this GPU, measured by the library's DFMA probe
    (paco_probe_fp64_peak: one launch, CUDA events) with the SM clock sampled
    while it runs; returns (GFLOP/s, description)."""
    sampler = ClockSampler(gpu_index)
    sampler.start()
    time.sleep(0.3)
    t0 = time.time()
    g, ms = paco.probe_fp64_peak(iters=8192)
    t1 = time.time()
    clk = sampler.stop(t0, t1)
    return g, (f"measured: DFMA probe (paco_probe_fp64_peak), {ms:.1f} ms at a median SM clock of "
               f"{clk.get('sm_mhz')} MHz (max {clk.get('sm_max_mhz')} MHz), FMA = 2 flops")


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# shared pieces of the GPU leg
# ---------------------------------------------------------------------------
def time_steps(step, K: int, warmup: int, stream):
    """Warm up, then time exactly K steps with one CUDA event pair per step on
    `stream`; returns (total ms from the first step's start to the last
    step's end, list of per-step ms)."""
    import torch
    for _ in range(max(warmup, 3)):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for k in range(K):
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    per = [a.elapsed_time(b) for a, b in ev]
    return ev[0][0].elapsed_time(ev[K - 1][1]), per


def rel_l2_vs_oracle(y, x):
    import numpy as np

    import oracle
    ref = oracle.fft(np.asarray(x, dtype=np.complex128).reshape(1, -1), threads=0)
    got = np.asarray(y, dtype=np.complex128).reshape(ref.shape)
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def tc_split(paco, x, y, N1, N2, b, p, K, warmup, stream, flop, world, max_over_ranks, plain_plan=None):
    """The tensor-core sub-DFT forms on the headline transform: time per step
    and, for each form and for the plain form, the relative L2 error of that
    same timed transform (the same input buffer) against the FP64 oracle."""
    import numpy as np
    res = {}
    KT = max(min(K, 50), 5)
    outs = {}
    for name, dt in (("bf16x3", paco.C64_TC_BF16X3), ("fp16", paco.C64_TC_FP16)):
        pl = paco.Plan(N1, N2, b, 1, dt, p=p)
        tot, per = time_steps(lambda: pl.execute(x, y, -1, stream), KT, warmup, stream)
        pl.check()
        ms = max_over_ranks(tot) / KT
        res[name] = {"ms_per_step": ms, "value": flop * world / (ms * 1e-3) / 1e9, "unit": "GFLOP/s",
                     "steps": KT, "kernel": "paco_stage_kernel, radix-16 passes as mma.sync contractions"}
        torch_sync()
        outs[name] = y.cpu().numpy()
        pl.close()
    if plain_plan is not None:
        plain_plan.execute(x, y, -1, stream)
        torch_sync()
        outs["plain"] = y.cpu().numpy()
    import oracle
    ref = oracle.fft(x.cpu().numpy().astype(np.complex128).reshape(1, -1), threads=0).reshape(-1)
    nref = float(np.linalg.norm(ref))
    for k, v in outs.items():
        res.setdefault(k, {})["rel_l2"] = float(np.linalg.norm(v.astype(np.complex128) - ref) / nref)
    res["error_measured_on"] = (f"the timed transform itself (N = {N1} x {N2}, b={b}, same input), "
                                "vs the FP64 oracle's full FFT")
    return res


def torch_sync():
    import torch
    torch.cuda.synchronize()


def cpu_leg(args, rank, world, dtype="c64", lg=None, threads=None):
    """The oracle timed on the host: all the cores this process may use
    (default), or `threads` of them."""
    if rank != 0 or world != 1 or args.no_cpu_baseline:
        return None
    lg = args.cpu_lg if lg is None else lg
    nt = host_cores() if threads is None else threads
    try:
        g, per, reps = oracle_sample(lg, args.cpu_seconds / 2, dtype, nt)
        return {"value": g, "unit": "GFLOP/s", "cores": nt, "kind": "oracle",
                "sample": f"{reps} x one 2^{lg}-point transform (same recipe), "
                          f"FP64 recursive radix-2 oracle, {nt} thread(s), {per:.2f} s each"}
    except Exception as e:  # report, do not hide
        return {"value": None, "unit": "GFLOP/s", "cores": 0, "kind": "oracle", "sample": f"failed: {e}"}


def hbm_roofline(kernel, bytes_per_launch, ms_per_launch, traffic=None):
    peak, src = measured_peak_hbm()
    achieved = bytes_per_launch / (ms_per_launch * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "peak_source": src,
            "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
            "algorithmic_bytes_per_launch": bytes_per_launch}


def e2e_host(step_host, KE, stream, units, unit, h2d, d2h, api, max_over_ranks, world, barrier):
    import torch
    for _ in range(2):
        step_host()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(KE):
        step_host()
    b.record(stream)
    torch.cuda.synchronize()
    e_ms = max_over_ranks(a.elapsed_time(b)) / KE
    return {"value": units * world / (e_ms * 1e-3), "unit": unit, "ms_per_step": e_ms,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "api": api}


def cufft_context(x, N: int, batch: int, flop: float, reps: int = 20):
    """cuFFT (through torch.fft.fft) on the same input: context only, not
    part of the measured path."""
    import torch
    try:
        xv = x.view(batch, N)
        stream = torch.cuda.current_stream()
        tot, per = time_steps(lambda: torch.fft.fft(xv), reps, 3, stream)
        ms = statistics.median(per)
        return {"cufft_ms_per_step": ms, "cufft_gflops": flop / (ms * 1e-3) / 1e9,
                "source": "torch.fft.fft (cuFFT C2C), same input, median of %d" % reps}
    except Exception as e:  # report, do not hide
        return {"cufft": f"failed: {e}"}


def emit(line):
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# other workloads
# ---------------------------------------------------------------------------
def run_other(args, ranks, local):
    import numpy as np
    import torch

    import paper_2609_06449_gb300 as paco
    from paco_inputs import gaussian, uniform, uneven_lengths

    rank, world = ranks.rank, ranks.world
    stream = torch.cuda.current_stream()
    K = args.steps
    W = max(args.warmup, 3)
    sampler = ClockSampler(local)
    mor = ranks.max_over_ranks
    base = {"n_gpus": world, "steps": K, "warmup": W, "scaling": "weak", "vs_baseline": None,
            "data": "synthetic", "metric": METRIC}

    def timed(step):
        sampler.start()
        time.sleep(0.3)
        ranks.barrier()
        torch.cuda.synchronize()
        t0 = time.time()
        tot, per = time_steps(step, K, 0, stream)
        t1 = time.time()
        ranks.barrier()
        return tot, per, sampler.stop(t0, t1)

    wl = args.workload
    if wl == "A":
        N1 = N2 = 256
        N = N1 * N2
        plan = paco.Plan(N1, N2, 2, 1, paco.C64, p=4)
        fused = bool(plan.info.fused_cluster)
        xh = torch.from_numpy(uniform(N, rank, np.complex64)).pin_memory()
        x = xh.cuda()
        y = torch.empty_like(x)
        for _ in range(W):
            plan.execute(x, y, -1, stream)
        tot, per, clocks = timed(lambda: plan.execute(x, y, -1, stream))
        plan.check()
        us = mor(statistics.median(per)) * 1e3
        acc = {"rel_l2": rel_l2_vs_oracle(y.cpu().numpy(), xh.numpy()),
               "measured_on": "the timed transform, vs the FP64 oracle"}
        ho = torch.empty_like(xh).pin_memory()
        di = torch.empty_like(x)
        e2e = None if args.no_e2e else e2e_host(lambda: plan.execute_host(xh, ho, di, y, -1, stream), max(args.e2e_steps, 20), stream,
                       1.0, "transforms/s", N * 8, N * 8, "paco_execute_host (pinned host buffers)", mor, world,
                       ranks.barrier)
        line = dict(base, value=us, unit="us (median latency per transform)", higher_is_better=False,
                    ms_per_step=mor(tot) / K, dtype="f32",
                    config={"workload": "c64 1-D DFT N=2^16 as 256 x 256, b=2, p=4, forward, latency",
                            "N1": N1, "N2": N2, "b": 2, "p": 4, "batch": 1,
                            "input": "Re, Im i.i.d. U[-1,1), seed = rank",
                            "l2": "input fits in L2: latency-bound by design, no flush"},
                    roofline=dict(hbm_roofline("paco_cluster_kernel (one launch, 16-CTA cluster)" if fused
                                               else "stage kernels (2 launches)",
                                               (16.0 if fused else 32.0) * N, statistics.median(per)),
                                  bound="latency"),
                    gflops=5.0 * N * 16 / (us * 1e-6) / 1e9, accuracy=acc,
                    e2e=e2e, cpu_baseline=cpu_leg(args, rank, world, lg=16),
                    gpu_launches=(1 if fused else 2) * K, clocks=clocks)
    elif wl == "B128":
        N1, N2 = 1 << 13, 1 << 14
        N = N1 * N2
        plan = paco.Plan(N1, N2, 2, 1, paco.C128, p=128)
        xh = torch.from_numpy(uniform(N, rank, np.complex128)).pin_memory()
        x = xh.cuda()
        y = torch.empty_like(x)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]

        def step2(k=[0]):
            i = k[0] % K
            ev[i][0].record(stream)
            plan.execute_stage1(x, y, args.dir, stream)
            ev[i][1].record(stream)
            plan.execute_stage2(y, y, args.dir, stream)
            ev[i][2].record(stream)
            k[0] += 1
        for _ in range(W):
            plan.execute(x, y, args.dir, stream)
        tot, per, clocks = timed(step2)
        plan.check()
        s1 = statistics.mean(ev[k][0].elapsed_time(ev[k][1]) for k in range(K))
        s2 = statistics.mean(ev[k][1].elapsed_time(ev[k][2]) for k in range(K))
        flop = 5.0 * N * 27
        ms = mor(tot) / K
        fp64_peak, fp64_src = fp64_peak_measured(paco, local)
        dom_ms = max(s1, s2)
        ho = torch.empty_like(xh).pin_memory()
        di = torch.empty_like(x)
        e2e = None if args.no_e2e else e2e_host(lambda: plan.execute_host(xh, ho, di, y, args.dir, stream), max(args.e2e_steps, 1), stream,
                       flop / 1e9, "GFLOP/s", N * 16, N * 16, "paco_execute_host (pinned host buffers)", mor,
                       world, ranks.barrier)
        hr = hbm_roofline("stage1" if s1 >= s2 else "stage2", 32.0 * N, dom_ms)
        import oracle
        plan.execute(x, y, args.dir, stream)
        torch.cuda.synchronize()
        ks = np.random.default_rng(5).integers(0, N, 8)
        ref = oracle.dft_at(xh.numpy(), ks, dir=args.dir, threads=0)
        got = y[torch.from_numpy(ks).cuda()].cpu().numpy()
        rms = math.sqrt(float((x.abs() ** 2).sum().item()))     # Parseval: rms of y = sqrt(sum |x|^2)
        acc = {"max_abs_err_over_rms": float(np.max(np.abs(got - ref)) / rms),
               "measured_on": "8 sampled coefficients vs the oracle's single-coefficient DFT"}
        line = dict(base, value=flop * world / (ms * 1e-3) / 1e9, unit="GFLOP/s", higher_is_better=True,
                    ms_per_step=ms, dtype="f64",
                    config={"workload": "c128 1-D DFT N=2^27 as N1=2^13 x N2=2^14, b=2, p=128, "
                                        + ("forward" if args.dir == -1 else "conjugate"), "dir": args.dir,
                            "N1": N1, "N2": N2, "b": 2, "p": 128, "batch": 1,
                            "input": "Re, Im i.i.d. U[-1,1), seed = rank", "l2": "inputs larger than L2"},
                    stage_ms={"stage1": s1, "stage2": s2}, hbm_gbs_effective=64.0 * N * world / (ms * 1e-3) / 1e9,
                    accuracy=acc, context=cufft_context(x, N, 1, flop),
                    roofline={"bound": "alu", "kernel": hr["kernel"],
                              "achieved": flop / 2 / (dom_ms * 1e-3) / 1e12, "peak": fp64_peak / 1e3,
                              "unit": "TFLOP/s (nominal 5N log2 N flops, half per stage)",
                              "peak_source": fp64_src,
                              "frac": flop / 2 / (dom_ms * 1e-3) / 1e12 / (fp64_peak / 1e3),
                              "traffic": None, "hbm": hr},
                    e2e=e2e, cpu_baseline=cpu_leg(args, rank, world, "c128"), gpu_launches=2 * K, clocks=clocks)
    elif wl == "C":
        if args.small:
            e = uneven_lengths(count=1024, seed=0, lo=8, hi=20, total_log2=26)
            lengths = np.concatenate([2 ** e, np.full(2 ** 12, 2 ** 12)]).astype(np.int64)
        else:
            e = uneven_lengths()
            lengths = np.concatenate([2 ** e, np.full(2 ** 14, 2 ** 12)]).astype(np.int64)
        total = int(lengths.sum())
        t_plan = time.time()
        plan = paco.BatchedPlan(lengths, autotune=not args.no_autotune, ctas_per_sm=2, lag=2)
        t_plan = time.time() - t_plan
        xh = torch.from_numpy(gaussian(total, rank, np.complex64)).pin_memory()
        x = xh.cuda()
        y = torch.empty_like(x)
        for _ in range(W):
            plan.execute(x, y, -1, stream)
        tot, per, clocks = timed(lambda: plan.execute(x, y, -1, stream))
        plan.check()
        flop = float(np.sum(5.0 * lengths * np.log2(lengths)))
        ms = mor(tot) / K
        ho = torch.empty_like(xh).pin_memory()
        di = torch.empty_like(x)
        e2e = None if args.no_e2e else e2e_host(lambda: plan.execute_host(xh, ho, di, y, -1, stream), max(args.e2e_steps, 1), stream,
                       flop / 1e9, "GFLOP/s", total * 8, total * 8, "paco_execute_host (pinned host buffers)", mor,
                       world, ranks.barrier)
        cfg = {str(int(n)): dict(zip(("b", "N1", "ctas_per_sm", "lag"), plan.config(int(n))))
               for n in np.unique(lengths)}
        plan.execute(x, y, -1, stream)
        torch.cuda.synchronize()
        offs = np.concatenate([[0], np.cumsum(lengths)])
        rng = np.random.default_rng(3)
        worst = 0.0
        for n in np.unique(lengths):
            for i in rng.choice(np.flatnonzero(lengths == n), size=2, replace=False):
                a_, b_ = int(offs[i]), int(offs[i + 1])
                e_ = rel_l2_vs_oracle(y[a_:b_].cpu().numpy(), xh[a_:b_].numpy())
                worst = max(worst, e_ / (5e-7 * math.log2(n)))
        acc = {"max_rel_l2_over_bound": worst,
               "measured_on": "2 sampled transforms of every length vs the oracle; bound 5e-7*log2(N_i)"}
        line = dict(base, value=flop * world / (ms * 1e-3) / 1e9, unit="GFLOP/s", higher_is_better=True,
                    ms_per_step=ms, dtype="f32",
                    config={"workload": "uneven batch: 4096 c64 transforms, log2 lengths uniform over 8..20 "
                                        "reduced to a 2^28 total, plus 2^14 transforms of 2^12; one persistent "
                                        "launch", "transforms": int(len(lengths)), "total_elements": total,
                            "input": "Re, Im i.i.d. N(0,1), seed = rank", "l2": "inputs larger than L2",
                            "autotuned": cfg, "plan_seconds": t_plan},
                    hbm_gbs_effective=32.0 * total * world / (ms * 1e-3) / 1e9, accuracy=acc,
                    roofline=hbm_roofline("paco_batched_kernel (1 launch)", 16.0 * total, statistics.mean(per)),
                    e2e=e2e, cpu_baseline=cpu_leg(args, rank, world, lg=18), gpu_launches=K, clocks=clocks)
    elif wl == "D":
        N1 = N2 = 4096
        N, B = N1 * N2, (2 if args.small else 16)
        xh = torch.from_numpy(np.concatenate([
            __import__("paco_inputs").loguniform(N, 100 * rank + i, np.complex64) for i in range(B)])).pin_memory()
        x = xh.cuda()
        y = torch.empty_like(x)
        flop = 5.0 * N * 24 * B
        forms = {}
        clocks = None
        for name, dt in (("plain", paco.C64), ("bf16x3", paco.C64_TC_BF16X3), ("fp16", paco.C64_TC_FP16)):
            if args.form not in ("all", name):
                continue
            pl = paco.Plan(N1, N2, 4, B, dt)
            for _ in range(W):
                pl.execute(x, y, -1, stream)
            tot, per, ck = timed(lambda: pl.execute(x, y, -1, stream))
            pl.check()
            ms = mor(tot) / K
            torch.cuda.synchronize()
            err = rel_l2_vs_oracle(y[:N].cpu().numpy(), xh[:N].numpy())
            split = tuple(pl.info.stage_split)
            forms[name] = {"ms_per_step": ms, "value": flop * world / (ms * 1e-3) / 1e9, "unit": "GFLOP/s",
                           "rel_l2_transform0": err, "dominant_launch_ms": statistics.mean(per) / 2,
                           "stage_split": list(split), "launches_per_step": 2 + sum(split)}
            if name == "bf16x3":
                clocks = ck
            pl.close()
        head = "bf16x3" if "bf16x3" in forms else next(iter(forms))
        hdt = {"plain": paco.C64, "bf16x3": paco.C64_TC_BF16X3, "fp16": paco.C64_TC_FP16}[head]
        clocks = clocks or ck
        line = dict(base, value=forms[head]["value"], unit="GFLOP/s", higher_is_better=True,
                    ms_per_step=forms[head]["ms_per_step"],
                    dtype={"plain": "f32", "bf16x3": "bf16x3 operands, f32 accumulate",
                           "fp16": "f16 operands (per-block scaled), f32 accumulate"}[head],
                    config={"workload": f"{B} x c64 1-D DFT N=2^24 (4096 x 4096, b=4), forward; precision forms",
                            "form_of_value": head,
                            "input": "log-uniform magnitudes 1e-4..1e4, uniform phases, seed = 100*rank + i",
                            "l2": "inputs larger than L2"},
                    forms=forms, context=cufft_context(x, N, B, flop),
                    roofline=hbm_roofline(f"stage kernel ({head})" + (", two passes per stage"
                                                                       if sum(forms[head]["stage_split"]) else ""),
                                          16.0 * N * B, forms[head]["dominant_launch_ms"]),
                    e2e=None, cpu_baseline=cpu_leg(args, rank, world),
                    gpu_launches=K * sum(f["launches_per_step"] for f in forms.values()), clocks=clocks)
        # e2e for the form of the line's value
        pl = paco.Plan(N1, N2, 4, B, hdt)
        ho = torch.empty_like(xh).pin_memory()
        di = torch.empty_like(x)
        line["e2e"] = None if args.no_e2e else e2e_host(lambda: pl.execute_host(xh, ho, di, y, -1, stream), max(args.e2e_steps, 1),
                               stream, flop / 1e9, "GFLOP/s", N * B * 8, N * B * 8,
                               "paco_execute_host (pinned host buffers)", mor, world, ranks.barrier)
    elif wl == "T":
        # the 128-point DFT sub-pass of a 2^14 stage: tcgen05 BF16x3 against the plain FP32 kernel
        Bt, Ct = (8, 16384) if args.small else (128, 16384)
        npts = Bt * 128 * Ct
        xh = torch.from_numpy(uniform(npts, rank, np.complex64)).pin_memory()
        x = xh.cuda().reshape(Bt, 128, Ct)
        y = torch.empty_like(x)
        y2 = torch.empty_like(x)
        plan = paco.Plan(128, Ct, 2, Bt, paco.C64)             # Phase I alone: the same column DFTs
        tot, per, clocks = timed(lambda: paco.probe_tc05_dft128(x, y, Bt, Ct, stream))
        ptot, pper = time_steps(lambda: plan.execute_phase1(x, y2, -1, stream), K, 3, stream)
        plan.check()
        torch.cuda.synchronize()
        rng = np.random.default_rng(1234)
        jj = np.arange(128)
        F = np.exp(-2j * np.pi * np.outer(jj, jj) / 128)
        rev = np.array([int(f"{k:07b}"[::-1], 2) for k in range(128)])   # Phase I stores row pi(k) (b = 2)
        e_tc, e_pl = [], []
        for _ in range(64):
            bi, ci = int(rng.integers(Bt)), int(rng.integers(Ct))
            ref = F @ x[bi, :, ci].cpu().numpy().astype(np.complex128)
            e_tc.append(np.linalg.norm(y[bi, :, ci].cpu().numpy() - ref) / np.linalg.norm(ref))
            e_pl.append(np.linalg.norm(y2[bi, rev, ci].cpu().numpy() - ref) / np.linalg.norm(ref))
        ms = mor(statistics.median(per))
        pms = mor(statistics.median(pper))
        gbs = lambda t: 16.0 * npts / (t * 1e-3) / 1e9
        peaks = {}
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
                peaks = json.load(fh)
        except (OSError, ValueError):
            pass
        bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
        mma_tflops = 3072.0 * npts / (ms * 1e-3) / 1e12          # 12 real 128 x 128 products per point, 2 flops each
        line = dict(base, value=gbs(ms), unit="GB/s effective (16 B per point), tcgen05 BF16x3 sub-pass",
                    higher_is_better=True, ms_per_step=ms, dtype="bf16x3 (fp32 in/out)",
                    config={"workload": f"DFT-128 sub-pass of a 2^14 stage: {Bt} x [128 x {Ct}] c64 "
                                        f"({npts} points), tcgen05 BF16x3 vs the plain FP32 stage kernel",
                            "input": "Re, Im i.i.d. U[-1,1), seed = rank", "l2": "inputs larger than L2"},
                    forms={"tcgen05_bf16x3": {"ms": ms, "gbs": gbs(ms), "rel_l2_max": float(max(e_tc))},
                           "plain_fp32": {"ms": pms, "gbs": gbs(pms), "rel_l2_max": float(max(e_pl))}},
                    accuracy={"measured_on": "64 sampled sequences vs their FP64 DFT"},
                    roofline={"bound": "tensor", "kernel": "tc05_dft128_kernel", "achieved": mma_tflops,
                              "peak": bf16_peak, "peak_source": "measured" if peaks else "fallback",
                              "unit": "TFLOP/s (bf16 MMA work)", "frac": mma_tflops / bf16_peak, "traffic": None,
                              "hbm": hbm_roofline("tc05_dft128_kernel", 16.0 * npts, ms)},
                    e2e=None, cpu_baseline=None, gpu_launches=K, clocks=clocks)
    elif wl == "U":
        lg = 13 if args.small else 14
        N1 = N2 = 1 << lg
        N = N1 * N2
        plan = paco.Plan(N1, N2, 4 if lg % 2 == 0 else 2, 1, paco.C64, p=64 if lg % 2 == 0 else 32)
        xh = torch.from_numpy(uniform(N, rank, np.complex64)).pin_memory()
        x = xh.cuda()
        at = torch.empty_like(x)
        w = torch.empty_like(x)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]

        def step3(k=[0]):
            i = k[0] % K
            ev[i][0].record(stream)
            plan.execute_phase1(x, at, -1, stream)
            ev[i][1].record(stream)
            plan.permute(at, w, -1, stream)
            ev[i][2].record(stream)
            plan.execute_stage2(w, w, -1, stream)
            ev[i][3].record(stream)
            k[0] += 1
        for _ in range(W):
            step3()
        tot, per, clocks = timed(step3)
        plan.check()
        sp = [statistics.mean(ev[k][j].elapsed_time(ev[k][j + 1]) for k in range(K)) for j in range(3)]
        flop = 5.0 * N * 2 * lg
        ms = mor(tot) / K
        # the fused two-pass path on the same transform, for the ratio
        yf = torch.empty_like(x)
        ftot, fper = time_steps(lambda: plan.execute(x, yf, -1, stream), K, 3, stream)
        line = dict(base, value=flop * world / (ms * 1e-3) / 1e9, unit="GFLOP/s", higher_is_better=True,
                    ms_per_step=ms, dtype="f32",
                    config={"workload": f"c64 1-D DFT N=2^{2 * lg} unfused: Phase I -> paco_permute -> Phase III",
                            "N1": N1, "N2": N2, "input": "Re, Im i.i.d. U[-1,1), seed = rank",
                            "l2": "inputs larger than L2"},
                    pass_ms={"phase1": sp[0], "permute": sp[1], "phase3": sp[2]},
                    fused_ms_per_step=mor(ftot) / K,
                    hbm_gbs_effective=48.0 * N * world / (ms * 1e-3) / 1e9,
                    roofline=hbm_roofline("paco_permute_kernel", 16.0 * N, sp[1]),
                    e2e=None, cpu_baseline=cpu_leg(args, rank, world), gpu_launches=3 * K, clocks=clocks)
    elif wl == "F3":
        # the 3-D DFT (dims = 3) of 64 arrays of 256 x 64 x 64, with cuFFT's fftn on the same input as context
        N1, N2, N3 = 256, 64, 64
        N, B = N1 * N2 * N3, (8 if args.small else 64)
        xh = torch.from_numpy(uniform(N * B, rank, np.complex64)).pin_memory()
        x = xh.cuda()
        y = torch.empty_like(x)
        plan = paco.Plan(N1, N2, 2, B, paco.C64, dims=3, N3=N3)
        launches = 2 + sum(plan.info.stage_split)
        for _ in range(W):
            plan.execute(x, y, -1, stream)
        tot, per, clocks = timed(lambda: plan.execute(x, y, -1, stream))
        plan.check()
        ms = mor(tot) / K
        flop = 5.0 * N * math.log2(N) * B
        xv = x.view(B, N1, N2, N3)
        ctot, cper = time_steps(lambda: torch.fft.fftn(xv, dim=(1, 2, 3)), min(K, 20), 3, stream)
        ref = torch.fft.fftn(xv, dim=(1, 2, 3)).permute(0, 3, 2, 1).reshape(B * N)
        torch.cuda.synchronize()
        diff = float(torch.linalg.vector_norm(y - ref) / torch.linalg.vector_norm(ref))
        cms = statistics.median(cper)
        ho = torch.empty_like(xh).pin_memory()
        di = torch.empty_like(x)
        line = dict(base, value=flop * world / (ms * 1e-3) / 1e9, unit="GFLOP/s", higher_is_better=True,
                    ms_per_step=ms, dtype="f32",
                    config={"workload": f"{B} x c64 3-D DFT of {N1} x {N2} x {N3} (dims = 3, b = 2), forward, "
                                        "output axes reversed",
                            "N1": N1, "N2": N2, "N3": N3, "batch": B, "input": "Re, Im i.i.d. U[-1,1), seed = rank",
                            "l2": "inputs larger than L2"},
                    stage_split=list(plan.info.stage_split), launches_per_step=launches,
                    hbm_gbs_effective=16.0 * launches * N * B * world / (ms * 1e-3) / 1e9,
                    accuracy={"rel_l2_vs_cufft_fftn": diff,
                              "measured_on": "the whole output vs torch.fft.fftn (parity with the oracle is in the tests)"},
                    context={"cufft_fftn_ms_per_step": cms, "cufft_gflops": flop / (cms * 1e-3) / 1e9,
                             "source": "torch.fft.fftn over the three axes (cuFFT), same input, median of %d"
                                       % min(K, 20)},
                    roofline=hbm_roofline(f"stage kernels, {launches} passes (Phase III split over the "
                                          f"{N2} x {N3} planes)", 16.0 * N * B, statistics.mean(per) / launches),
                    e2e=None if args.no_e2e else e2e_host(lambda: plan.execute_host(xh, ho, di, y, -1, stream),
                                                          max(args.e2e_steps, 1), stream, flop / 1e9, "GFLOP/s",
                                                          N * B * 8, N * B * 8, "paco_execute_host (pinned host buffers)",
                                                          mor, world, ranks.barrier),
                    cpu_baseline=None, gpu_launches=K * launches, clocks=clocks)
    else:  # E
        N1 = N2 = 1024
        N, B = N1 * N2, 256
        xh = torch.from_numpy(gaussian(N * B, rank, np.complex64).reshape(B, N)).pin_memory()
        wh = torch.from_numpy(__import__("paco_inputs").weights(N * B, rank + 1).reshape(B, N)).pin_memory()
        x = xh.cuda().requires_grad_(True)
        w = wh.cuda()

        def loss_of(yv):
            # sum(w |y|^2) on the (re, im) view: the unfused composition, for context
            yr = torch.view_as_real(yv)
            return (w * (yr * yr).sum(-1)).sum()

        def step():
            # the loss summed in the Phase III kernel, its backward fused into
            # the conjugate transform's loads
            x.grad = None
            loss = paco.weighted_power_loss(x, w, N1, N2, 4)
            loss.backward()
            return loss

        def step_unfused():
            x.grad = None
            loss = loss_of(paco.PacoFFT.apply(x, N1, N2, 4))
            loss.backward()
            return loss
        for _ in range(W):
            step()
        tot, per, clocks = timed(step)
        tot_u, _ = time_steps(step_unfused, min(K, 20), 3, stream)
        flop = 2 * 5.0 * N * 20 * B
        import oracle
        step()
        torch.cuda.synchronize()
        x0 = xh[0].numpy().astype(np.complex128)
        w0 = wh[0].numpy().astype(np.float64)
        # d/dx of sum(w |F x|^2) in PyTorch's convention: 2 F^H (w * F x)
        gref = 2.0 * oracle.fft((w0 * oracle.fft(x0.reshape(1, -1))).reshape(1, -1), dir=+1).reshape(-1)
        g0 = x.grad[0].detach().cpu().numpy().astype(np.complex128)
        acc = {"grad_rel_l2": float(np.linalg.norm(g0 - gref) / np.linalg.norm(gref)),
               "measured_on": "gradient of transform 0 vs the analytic adjoint 2 F^H (w F x) from the oracle"}
        ms = mor(tot) / K
        gh = torch.empty_like(xh).pin_memory()

        def step_host():
            xd = xh.to("cuda", non_blocking=True).requires_grad_(True)
            loss = paco.weighted_power_loss(xd, w, N1, N2, 4)
            loss.backward()
            gh.copy_(xd.grad, non_blocking=True)
        e2e = None if args.no_e2e else e2e_host(step_host, max(args.e2e_steps, 1), stream, flop / 1e9, "GFLOP/s", N * B * 8, N * B * 8,
                       "torch.autograd through PacoFFT (pinned host input and gradient)", mor, world, ranks.barrier)
        line = dict(base, value=flop * world / (ms * 1e-3) / 1e9, unit="GFLOP/s (forward + backward transforms)",
                    higher_is_better=True, ms_per_step=ms, dtype="f32",
                    config={"workload": "256 x c64 1-D DFT N=2^20 (1024 x 1024, b=4): loss = sum(w |FFT(x)|^2), "
                                        "forward + backward (conjugate transform) through torch.autograd, "
                                        "the loss and its backward fused into the stage kernels",
                            "input": "x Re, Im i.i.d. N(0,1); w U[0,1)", "l2": "inputs larger than L2"},
                    accuracy=acc,
                    context=dict(cufft_context(x.detach(), N, B, flop / 2),
                                 unfused_ms_per_step=mor(tot_u) / min(K, 20),
                                 unfused="PacoFFT + the loss and its gradient as PyTorch element-wise ops"),
                    roofline=hbm_roofline("stage kernels (4 launches; w read by the loss epilogue and the "
                                          "backward's loads)", (4 * 16.0 + 2 * 4.0) * N * B, ms),
                    e2e=e2e, cpu_baseline=cpu_leg(args, rank, world, lg=20), gpu_launches=4 * K, clocks=clocks)
    if rank == 0:
        emit(line)


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
    if args.workload != "B":
        run_other(args, ranks, local)
        ranks.close()
        return

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

    tc = None
    if args.dtype == "c64" and not args.no_tc:
        tc = tc_split(paco, x, out, N1, N2, args.b, args.p, K, args.warmup, stream, flop, world, max_over_ranks,
                      plain_plan=plan)
        tc["plain"].update({"ms_per_step": ms_step, "value": value, "unit": "GFLOP/s"})

    cpu = cpu_leg(args, rank, world, args.dtype)
    cpu1 = cpu_leg(args, rank, world, args.dtype, threads=1)
    context = cufft_context(x, N, 1, flop)

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
            "e2e": e2e, "cpu_baseline": cpu, "cpu_baseline_1core": cpu1, "gpu_launches": 2 * K,
            "clocks": clocks, "tc_split": tc, "context": context,
        }
        print(json.dumps(line), flush=True)
    ranks.close()


if __name__ == "__main__":
    main()
