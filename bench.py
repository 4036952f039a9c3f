#!/usr/bin/env python
"""Throughput of the GB300 k-means hot path on five seeded synthetic workloads.

Every workload prints one JSON line (rank 0).  The metric is assign+update GFLOP/s with the
algorithmic flop count 2nkd + nd per Lloyd iteration (padding, rechecks and fallbacks are not
counted), and the roofline of the dominant kernel beside it.

  highdim (default)  n = 200,000 points, d = 1,024, k = 100, 100-component Gaussian mixture
                     (weights Dirichlet(1), means U[-10,10]^d, sigma log-uniform in [0.5, 2]).
                     A step is one Lloyd iteration: kmeans_assign (distance GEMM, fused top-2
                     epilogue, exact recheck of certified near-ties) + kmeans_update (stable
                     counting sort, segmented CF sums, FP64 centroids and costs).  Seeding, row
                     norms and the operand copy are per-dataset preparation, timed separately
                     in "pipeline".  X (819 MB FP32, 410 MB BF16) is larger than L2.
  small              n = 10,000, d = 64, k = 10, 10 components, FP32: a step is a whole run
                     (row norms, k-means++, 20 Lloyd iterations); L2 is flushed between steps
                     (X is 2.56 MB).  Latency-bound.
  stream             2,000,000 points in d = 2,048 from a 500-component mixture in a random
                     rank-64 subspace plus N(0, 0.1^2) noise; 31 chunks of 65,536 rows projected
                     to r = 64 by the BF16 projection GEMM, then k = 1,000 k-means++ and Lloyd on
                     the coordinates in BF16 (step), FP8 and FP32 (forms), 20 iterations.
  batch              512 problems (n log-uniform in [1e3, 1e5], d in {32, 128, 512}, k
                     log-uniform in [4, 256], k components each), 4 k-means++ seeds each,
                     20 Lloyd iterations, in one recorded CUDA graph; a step is one replay.
  learned            n = 4,000,000, d = 256, k = 16,384 (16,384 components; 200,000 held-out
                     points train the proposal network).  Centers: k-means++ on the first
                     200,000 points, then 5 FP32 Lloyd iterations, frozen.  A step is the learned
                     assignment (MLP 256-256-256-16384, top-32 candidates, certified exact check,
                     full-scan fallback) + the CF update; the BF16 and FP32 full scans run beside.

``--impl reference`` times the FP64 CPU oracle on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

UNIT = "GFLOP/s"
METRICS = {
    "highdim": "assign+update GFLOP/s (Lloyd iteration, 200k x 1024, k=100)",
    "small": "assign+update GFLOP/s (whole k-means++ + 20-iteration run, 10k x 64, k=10)",
    "stream": "assign+update GFLOP/s (Lloyd iteration on projected coordinates, 2M x 64, k=1000)",
    "batch": "assign+update GFLOP/s (512 problems x 4 seeds x 20 iterations per replay)",
    "learned": "assign+update GFLOP/s, exact-method flops (learned assignment, 4M x 256, k=16384)",
    "swn": "assign+update GFLOP/s (Lloyd iteration, StructuredWithNoise 50 sets x 5000 points, d=1000, k=50)",
    "svd": "randomised truncated SVD GFLOP/s (one piece 65,536 x 2,048, l=64, s=80)",
    "bico": "nearest-reference query GFLOP/s (1,000,000 x 128 points against 20,000 features)",
    "piecy": "per-piece basis + lift GFLOP/s (8 pieces of 65,536 x 2,048, l=64, s=80)",
}
DEFAULT_STEPS = {"highdim": 30, "small": 20, "stream": 20, "batch": 5, "learned": 5, "swn": 30, "svd": 20,
                 "bico": 10, "piecy": 5}
SWN_X = 20   # signal dimensions per hidden set (Section 3 leaves the count open)
# FP32 SIMT peak: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (maximum SM clock)
FFMA_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
TF32_OVER_BF16 = 1.1 / 2.25   # nominal dense ratios, applied to the measured BF16 peak
FP8_OVER_BF16 = 4.5 / 2.25
FP64_NOMINAL_TFLOPS = 1.25    # GB300's dense FP64 figure (the FP64 pipe is about 1/64 of the FP32 one)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gbkm", choices=["gbkm", "reference"])
    ap.add_argument("--workload", default="highdim", choices=list(METRICS))
    ap.add_argument("--form", default="auto", choices=["auto", "f32", "bf16"])
    ap.add_argument("--engine", default="auto", choices=["auto", "simt", "tcgen05"])
    ap.add_argument("--center-terms", type=int, default=1, choices=[1, 2],
                    help="BF16 form: centers as one BF16 term, or two (head + tail, a narrower certified band)")
    ap.add_argument("--n", type=int, default=None, help="override n (highdim / learned / swn)")
    ap.add_argument("--d", type=int, default=None, help="override d (highdim / swn)")
    ap.add_argument("--k", type=int, default=None, help="override k (highdim; swn: the number of hidden sets)")
    ap.add_argument("--problems", type=int, default=512, help="batch: number of problems")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-probe", action="store_true", help="skip the compute-peak probes")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-compare", action="store_true", help="skip the other forms")
    a = ap.parse_args()
    if a.steps is None:
        a.steps = DEFAULT_STEPS[a.workload]
    if a.warmup < 3:
        ap.error("--warmup must be >= 3")
    return a


# ---------------------------------------------------------------------------- shared helpers
def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return {"hbm_gbs": j["hbm_gbs"], "bf16_tflops": j["bf16_tflops"],
                "bf16_tflops_sustained": j.get("bf16_tflops_sustained", j["bf16_tflops"]),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "source": "fallback"}


def source_hash(files):
    """Hash of the given kernel source files (relative to csrc/), to tell whether stored ncu
    counters still apply."""
    import hashlib

    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1502_04265_gb300", "csrc")
    for f in sorted(files):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def stored_traffic(key):
    """DRAM bytes per launch of `key` from a committed ncu capture (profiles/traffic.json), or
    None when its kernel sources changed since the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        table = json.load(f)
    e = table.get(key)
    if not e or e.get("source_hash") != source_hash(e.get("sources", [])):
        return None
    return e["dram_bytes_per_launch"]


class Ranks:
    """The rank bookkeeping of a replicated run (one process per GPU, launched by torchrun): the
    launcher's RANK / LOCAL_RANK / WORLD_SIZE, a barrier and the maximum of a host value over the
    ranks.  The bench uses NCCL tensors on each rank's GPU; the same logic runs on gloo and CPU
    tensors for the multi-process tests."""

    def __init__(self, backend="nccl", device=None):
        import torch.distributed as dist

        self.dist = dist
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.device = device
        if self.world > 1 and not dist.is_initialized():
            if backend == "nccl":
                dist.init_process_group(backend, device_id=device)
            else:
                dist.init_process_group(backend)

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()

    def max_over_ranks(self, v):
        if self.world == 1:
            return v
        import torch

        t = torch.tensor([v], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def whole_job(self, work_per_rank, ms):
        """Throughput of all ranks' work (each rank does work_per_rank units) in the slowest rank's
        time: the weak-scaling value of the JSON line."""
        return self.world * work_per_rank / (ms * 1e-3)

    def close(self):
        if self.world > 1 and self.dist.is_initialized():
            self.dist.destroy_process_group()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, flags in rows for i, f in enumerate(flags)
                          if f.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


class Env:
    """Rank, device, library context and peaks of this process."""

    def __init__(self, args):
        import torch
        import torch.distributed as dist

        from paper_1502_04265_gb300 import _binding as B

        self.args = args
        self.torch, self.dist, self.B = torch, dist, B
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        self.dev = torch.device("cuda", local)
        self.ranks = Ranks("nccl", self.dev)
        self.world, self.rank, self.local = self.ranks.world, self.ranks.rank, self.ranks.local
        B.load(build_if_missing=True)
        self.ctx = B.Context(self.local)
        self.peaks = load_peaks()
        # the compute peaks the copy + cuBLAS figures do not cover, probed on this GPU by the
        # library's own kernels (tcgen05 kind::tf32 / kind::f8f6f4 at the engine's tile shape,
        # CUDA-core FMA chains); every roofline takes the larger of a probe and its nominal ratio
        self.peaks["probed"] = {}
        if not args.no_probe:
            for u in ("bf16", "tf32", "fp8", "ffma", "fp64"):
                try:
                    self.peaks["probed"][u] = self.ctx.probe_peak(u)
                except Exception:
                    self.peaks["probed"][u] = None

    @property
    def stream(self):
        return self.torch.cuda.current_stream(self.dev)

    def barrier(self):
        self.ranks.barrier()

    def max_over_ranks(self, v):
        return self.ranks.max_over_ranks(v)

    def event(self):
        return self.torch.cuda.Event(enable_timing=True)

    def timed(self, step, steps, warmup, clocks=False, flush=None, profile=True):
        """`warmup` untimed and `steps` timed calls of step(i), CUDA events on the launching
        stream, barrier + synchronize on both sides; with `flush`, L2 is overwritten before
        every step and only the steps are timed.  Returns ms per step (max over ranks), our
        kernel launches in the timed region, the library's per-kernel profile and the clocks."""
        torch = self.torch
        for i in range(warmup):
            if flush:
                flush()
            step(i)
        self.ctx.sync()
        sampler = ClockSampler(self.local) if clocks and self.rank == 0 and not self.args.no_clocks else None
        if sampler:
            sampler.start()
            time.sleep(0.5)
        def run_steps(first):
            pairs = []
            if flush is None:
                a, b = self.event(), self.event()
                a.record(self.stream)
                for i in range(steps):
                    step(first + i)
                b.record(self.stream)
                pairs.append((a, b))
            else:
                for i in range(steps):
                    flush()
                    a, b = self.event(), self.event()
                    a.record(self.stream)
                    step(first + i)
                    b.record(self.stream)
                    pairs.append((a, b))
            torch.cuda.synchronize(self.dev)
            return sum(a.elapsed_time(b) for a, b in pairs)

        # the timed pass runs without the library's per-kernel events (they add a few percent to a
        # short step); a second pass of the same steps, with them, gives the per-kernel times
        l0 = self.ctx.launch_count()
        self.barrier()
        torch.cuda.synchronize(self.dev)
        ms_total = run_steps(warmup)
        self.barrier()
        launches = self.ctx.launch_count() - l0
        clk = sampler.stop() if sampler else None
        ms_prof, prof = None, {}
        if profile:
            self.ctx.profile(True)
            ms_prof = run_steps(warmup + steps) / max(steps, 1)
            prof = self.ctx.profile_read()
            self.ctx.profile(False)
        return {"ms": self.max_over_ranks(ms_total / max(steps, 1)), "launches": int(launches), "prof": prof,
                "clocks": clk, "total_s": ms_total * 1e-3, "ms_profiled": ms_prof}

    def once(self, fn, warmup=1):
        """Device time of one call of fn() after `warmup` calls, with the per-kernel profile."""
        for _ in range(warmup):
            fn()
        R = self.timed(lambda i: fn(), 1, 0)
        return R


def kernel_avg_s(prof, name):
    launches, ms = prof.get(name, (0, float("nan")))
    return ms / max(launches, 1) * 1e-3


def roofline(peaks, kernel, avg_s, bytes_, flops, unit_tflops, total_s, bound=None, note=None, traffic=None):
    """Roofline object of one kernel: algorithmic bytes / flops per launch over its average launch
    duration, against the measured HBM copy bandwidth or the compute unit's peak (the burst BF16
    figure for a kernel timed for under a second, the sustained one otherwise)."""
    if bound is None:
        t_hbm = bytes_ / (peaks["hbm_gbs"] * 1e9)
        t_c = flops / (unit_tflops * 1e12) if flops else 0.0
        bound = "hbm" if t_hbm >= t_c else "tensor"
    if bound == "hbm":
        ach, peak, unit = bytes_ / avg_s / 1e9, peaks["hbm_gbs"], "GB/s"
    else:  # "tensor" or "alu": flops against the compute unit's peak
        ach, peak, unit = flops / avg_s / 1e12, unit_tflops, "TFLOP/s"
    r = {"bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak, "traffic": traffic,
         "kernel": kernel, "kernel_ms": avg_s * 1e3, "algorithmic_bytes": int(bytes_),
         "algorithmic_flops": float(flops), "peak_source": f"{peaks['source']} ({'of measured' if peaks['source'] == 'measured' else 'of fallback'})"}
    if note:
        r["note"] = note
    return r


def bf16_peak(peaks, total_s):
    return peaks["bf16_tflops_sustained"] if total_s > 1.0 else peaks["bf16_tflops"]


def _probed(peaks, unit):
    return (peaks.get("probed") or {}).get(unit) or 0.0


def fp64_peak(peaks):
    """FP64 FMA peak: the larger of the probe and the nominal figure."""
    return max(FP64_NOMINAL_TFLOPS, _probed(peaks, "fp64"))


def ffma_peak(peaks):
    """FP32 FMA peak: the larger of the probe and 152 SMs x 128 lanes x 2 x 2.07 GHz."""
    return max(FFMA_PEAK_TFLOPS, _probed(peaks, "ffma"))


def unit_peak(peaks, compute, engine_tc, total_s):
    """Peak of the unit a form runs on: BF16 the measured cuBLAS figure; FP8 and 3xTF32 (three
    kind::tf32 MMAs per product) the larger of the probe and the measured BF16 figure times the
    nominal dense ratio; the SIMT form the FFMA peak."""
    b = bf16_peak(peaks, total_s)
    if compute == "bf16":
        return b
    if compute == "fp8":
        return max(b * FP8_OVER_BF16, _probed(peaks, "fp8"))
    return max(b * TF32_OVER_BF16, _probed(peaks, "tf32")) / 3.0 if engine_tc else ffma_peak(peaks)


def peaks_report(peaks):
    """The denominators in use, with their sources, for the JSON line."""
    b = peaks["bf16_tflops"]
    return {"hbm_gbs": peaks["hbm_gbs"], "bf16_tflops": b, "bf16_tflops_sustained": peaks["bf16_tflops_sustained"],
            "source": peaks["source"], "probed_tflops": peaks.get("probed"),
            "tf32_nominal_tflops": b * TF32_OVER_BF16, "fp8_nominal_tflops": b * FP8_OVER_BF16,
            "ffma_nominal_tflops": FFMA_PEAK_TFLOPS,
            "fp64_nominal_tflops": FP64_NOMINAL_TFLOPS,
            "rule": "tf32 / fp8 / ffma / fp64 peak = max(probe, nominal); 3xTF32 = tf32 / 3"}


def gen_pool(jobs, fn, workers=None):
    """Run the seeded generators of many independent pieces in spawned processes (started before
    any CUDA use in this process); returns the results in job order."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    workers = workers or max(1, min(8, (os.cpu_count() or 2) - 1))
    ex = ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
    return ex, [ex.submit(fn, j) for j in jobs]


def primary_form(requested, d):
    """The form of a workload's primary line: the one requested, or the faster exact form at the
    shape (driver.exact_form: FP32 3xTF32 below 256 dimensions, BF16 with the certified recheck
    from 256 up)."""
    if requested in ("bf16", "f32"):
        return requested
    from paper_1502_04265_gb300 import driver

    return driver.exact_form(d)


def lloyd_timed(env, X, Xop, scales, xnorm, C0, compute, engine, steps, warmup, clocks=False, center_terms=1):
    """`warmup` + `steps` Lloyd iterations from C0 (assign + update per step); the timed steps'
    ms, launches, profile, the FP64 cost trace and recheck counts."""
    torch, B = env.torch, env.B
    n = X.shape[0]
    labels = torch.empty(n, dtype=torch.int32, device=env.dev)
    Cs = [C0.clone(), torch.empty_like(C0)]
    # indices: warm-up, the timed pass, then the profiled pass of the same number of steps
    cost = torch.zeros((2 * steps + warmup, 2), dtype=torch.float64, device=env.dev)
    nre = torch.zeros(2 * steps + warmup, dtype=torch.int64, device=env.dev)

    def step(i):
        B.kmeans_assign(X, Cs[0], Xop=Xop, Xop_scales=scales, xnorm=xnorm, compute=compute, engine=engine,
                        labels=labels, n_rechecked=nre[i:i + 1], center_terms=center_terms, ctx=env.ctx)
        B.kmeans_update(X, labels, Cs[0], C_new=Cs[1], cost_old=cost[i, 0:1], cost_new=cost[i, 1:2], ctx=env.ctx)
        Cs.reverse()

    R = env.timed(step, steps, warmup, clocks=clocks)
    env.ctx.sync()
    R.update({"costs": cost.cpu().numpy(), "rechecked": nre.cpu().numpy(), "C": Cs[0], "labels": labels})
    return R


def assign_kernel(prof):
    return "assign_tc" if "assign_tc" in prof else "assign_simt"


def base_line(env, workload, value, ms, steps, warmup, dtype, config):
    return {"metric": METRICS[workload], "value": value, "unit": UNIT, "n_gpus": env.world, "steps": steps,
            "warmup": warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": config,
            "peaks": peaks_report(env.peaks),
            "kernel_timing": "per-kernel CUDA events on the launching stream, recorded by the library around "
                             "each kernel during a second pass of the same steps right after the timed one (the "
                             "timed pass runs without them: they add a few percent to a short step)"}


def kernels_ms(prof):
    return {name: prof[name][1] / max(prof[name][0], 1) for name in prof}


# ---------------------------------------------------------------------------- CPU oracle samples
def oracle_assign_update_rate(X, C, cpu_seconds, threads=None, label=""):
    """The FP64 oracle's assign + update on a bounded row sample of X, repeated for about
    cpu_seconds; GFLOP/s of the sample (2 m k d + m d per pass)."""
    import numpy as np

    import oracle

    oracle.build()
    cores = oracle.set_threads(threads or os.cpu_count() or 1)
    n, d = X.shape
    k = C.shape[0]
    Cd = np.ascontiguousarray(C, dtype=np.float64)
    rows = min(n, 512)
    t0 = time.perf_counter()
    lab, _, _ = oracle.assign(X[:rows], Cd)
    oracle.update(X[:rows], lab, Cd)
    dt = time.perf_counter() - t0
    rows = int(min(n, max(rows, rows * cpu_seconds / 3 / max(dt, 1e-3))))
    reps, t0 = 0, time.perf_counter()
    while True:
        lab, _, _ = oracle.assign(X[:rows], Cd)
        oracle.update(X[:rows], lab, Cd)
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= cpu_seconds or reps >= 64:
            break
    flops = reps * (2.0 * rows * k * d + rows * d)
    return {"value": flops / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{label}first {rows} of {n} rows x {reps} passes: assign over all k={k} + update, "
                      f"FP64 C loops (OpenMP over points), {dt:.1f} s"}


def oracle_lloyd_rate(problems, iters, cpu_seconds, threads=None, label=""):
    """The oracle's k-means++ + `iters` Lloyd iterations over (X, k, u) runs until about
    cpu_seconds; GFLOP/s counting iters x (2nkd + nd) per run."""
    import numpy as np

    import oracle

    oracle.build()
    cores = oracle.set_threads(threads or os.cpu_count() or 1)
    flops, runs, t0 = 0.0, 0, time.perf_counter()
    for X, k, u in problems:
        _, C0, _, _ = oracle.seed_pp(X, k, u)
        oracle.lloyd(X, C0, iters)
        n, d = X.shape
        flops += iters * (2.0 * n * k * d + n * d)
        runs += 1
        if time.perf_counter() - t0 >= cpu_seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": flops / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{label}{runs} whole runs (k-means++ + {iters} Lloyd iterations), FP64 C loops, {dt:.1f} s"}


# ---------------------------------------------------------------------------- workloads
def mixture(n, d, comps, seed):
    from paper_1502_04265_gb300 import synth

    X, _ = synth.gaussian_mixture(n, d, comps, seed=seed)
    return X


def swn_shape(args):
    """StructuredWithNoise: ell hidden sets of y points in d dimensions, k = ell."""
    ell = args.k or 50
    y = (args.n or 250_000) // ell
    return ell, y, args.d or 1000


def workload_data(args, seed):
    """(X, hidden labels or None, n, d, k) of the highdim or swn workload."""
    from paper_1502_04265_gb300 import synth

    if args.workload == "swn":
        ell, y, d = swn_shape(args)
        X, z = synth.structured_with_noise(ell, y, d, SWN_X, seed=seed)
        return X, z, ell * y, d, ell
    n, d, k = args.n or 200_000, args.d or 1024, args.k or 100
    return mixture(n, d, k, seed=seed), None, n, d, k


def run_highdim(env, args):
    import numpy as np

    torch, B = env.torch, env.B
    from paper_1502_04265_gb300 import synth

    X, hidden, n, d, k = workload_data(args, env.rank)
    F = 2.0 * n * k * d + n * d
    u = synth.seed_uniforms(k, seed=env.rank)
    Xg = torch.from_numpy(X).to(env.dev)
    ug = torch.from_numpy(u).to(env.dev)
    ctx = env.ctx
    xnorm = B.kmeans_row_norms(Xg, ctx=ctx)
    _, C0 = B.kmeans_seed_pp(Xg, k, ug, ctx=ctx)
    form, engine, Xop, Xr = args.form, args.engine, None, None
    if form in ("auto", "bf16"):
        # the BF16 copy and the rows' rounding residuals (the certified band's side data)
        Xb, Xrb = B.kmeans_quantize(Xg, "bf16", ctx=ctx)
        try:
            B.kmeans_assign(Xg, C0, Xop=Xb, Xop_scales=Xrb, xnorm=xnorm, compute="bf16", engine=engine, ctx=ctx)
            form, Xop, Xr = "bf16", Xb, Xrb
        except B.GbkmError:
            if form == "bf16":
                raise
            form = "f32"
            del Xb, Xrb
    else:
        form = "f32"
    ctx.sync()

    R = lloyd_timed(env, Xg, Xop, Xr, xnorm, C0, form, engine, args.steps, args.warmup, clocks=True,
                    center_terms=args.center_terms if form == "bf16" else 1)
    ms, prof = R["ms"], R["prof"]
    value = env.ranks.whole_job(F, ms) / 1e9
    peaks = env.peaks
    kname = assign_kernel(prof)
    tc = kname == "assign_tc"
    es = 2 if form == "bf16" else 4
    bytes_k = n * d * es + k * d * es + n * 4
    roof = roofline(peaks, kname, kernel_avg_s(prof, kname), bytes_k, 2.0 * n * k * d,
                    unit_peak(peaks, form, tc, R["total_s"]), R["total_s"],
                    bound=None if form == "bf16" else ("tensor" if tc else "alu"),
                    note=None if form == "bf16" else ("3xTF32: max(probed kind::tf32, measured BF16 x nominal TF32/BF16 ratio) / 3" if tc
                                                      else "FFMA peak = 152 SMs x 128 lanes x 2 x 2.07 GHz"),
                    traffic=stored_traffic(f"{kname}/{form}/{n}x{d}_k{k}"))
    # the update's segmented sums: one FP32 read of X in cluster order (+ the permutation)
    rooflines = {kname: roof}
    if "segsum" in prof:
        rooflines["segsum"] = roofline(peaks, "segsum", kernel_avg_s(prof, "segsum"), n * d * 4 + n * 4, 0.0,
                                       FFMA_PEAK_TFLOPS, R["total_s"], bound="hbm",
                                       note="update: sums of x - s per (cluster, item) in FP32 blocks with "
                                            "double-float accumulation, one read of X gathered in cluster order",
                                       traffic=stored_traffic(f"segsum/{n}x{d}_k{k}"))
    # the roofline object is the dominant kernel's (the longest average launch)
    roof = max(rooflines.values(), key=lambda r: r["kernel_ms"])
    p_unit = unit_peak(peaks, form, tc, R["total_s"]) * 1e12
    # the algorithmic floor of one iteration: one read of X at the operand dtype, the centers, the
    # labels and the FP64 clustering features; for comparison, one FP32 read of X (what exact FP32
    # centroid sums need at least) and this design's traffic (the operand copy in the assign, FP32
    # in the update)
    B_alg = n * d * es + k * d * 4 + n * 4 + k * (d + 2) * 8
    B_f32 = n * d * 4 + k * d * 4 + n * 4 + k * (d + 2) * 8
    B_design = B_f32 + n * d * es
    hbm = peaks["hbm_gbs"] * 1e9
    t_roof = max(B_alg / hbm, 2.0 * n * k * d / p_unit)
    t_f32 = max(B_f32 / hbm, 2.0 * n * k * d / p_unit)
    t_design = max(B_design / hbm, 2.0 * n * k * d / p_unit)
    step_roof = {"t_roof_ms": t_roof * 1e3, "frac": t_roof / (ms * 1e-3),
                 "t_f32_read_ms": t_f32 * 1e3, "frac_f32_read": t_f32 / (ms * 1e-3),
                 "t_design_ms": t_design * 1e3, "frac_design": t_design / (ms * 1e-3),
                 "note": "T_roof = max(bytes / HBM, flops / unit peak) over the whole iteration with one read of "
                         "X at the operand dtype (the algorithmic floor); T_f32_read with one FP32 read; "
                         "T_design with this design's two reads (operand copy in the assign, FP32 in the update)"}

    # the whole run (per-dataset preparation included): norms, operand copy, k-means++, 30 iterations
    iters = 30
    labels = torch.empty(n, dtype=torch.int32, device=env.dev)
    Ca, Cb = torch.empty_like(C0), torch.empty_like(C0)
    tr = torch.zeros((iters, 2), dtype=torch.float64, device=env.dev)

    def whole():
        # norms, BF16 copy and residuals in one read of X
        B.kmeans_ingest(Xg, copy=False, xnorm=xnorm, Xq=Xop, resid=Xr, quantize=form == "bf16", ctx=ctx)
        B.kmeans_seed_pp(Xg, k, ug, C_out=Ca, ctx=ctx)
        cur, nxt = Ca, Cb
        for t in range(iters):
            B.kmeans_assign(Xg, cur, Xop=Xop, Xop_scales=Xr, xnorm=xnorm, compute=form, engine=engine,
                            labels=labels, ctx=ctx)
            B.kmeans_update(Xg, labels, cur, C_new=nxt, cost_old=tr[t, 0:1], cost_new=tr[t, 1:2], ctx=ctx)
            cur, nxt = nxt, cur

    W = env.once(whole)
    pipeline = {"iterations": iters, "total_ms": W["ms"],
                "gflops_whole_run": iters * F / (W["ms"] * 1e-3) / 1e9,
                "stage_ms": {nm: W["prof"][nm][1] for nm in ("ingest", "seed") if nm in W["prof"]},
                "note": "one whole run from raw X: the k-means++ time is included, its flops are not"}
    if hidden is not None:
        # the planted partition's cost (its own means, through the library's update) against the run's
        zt = torch.from_numpy(hidden).to(env.dev)
        hc = torch.zeros(2, dtype=torch.float64, device=env.dev)
        B.kmeans_update(Xg, zt, Ca, C_new=torch.empty_like(C0), cost_old=hc[0:1], cost_new=hc[1:2], ctx=ctx)
        ctx.sync()
        lab = labels.cpu().numpy()
        tab = np.zeros((k, k), dtype=np.int64)
        np.add.at(tab, (lab, hidden), 1)
        planted, final = float(hc[1]), float(tr[iters - 1, 1])
        pipeline["hidden_sets"] = {"planted_cost": planted, "final_cost": final, "cost_ratio": final / planted,
                                   "purity": float(tab.max(axis=1).sum()) / n,
                                   "note": "purity = share of points whose cluster's most common hidden set is "
                                           "their own, after the whole run's last assignment"}
        del zt

    e2e = None
    if not args.no_e2e:
        Xh = torch.from_numpy(X).pin_memory()
        hb = B.HostBlock((n, d))
        hb.tensor.copy_(torch.from_numpy(X))
        Ch_out = torch.empty((k, d), dtype=torch.float32).pin_memory()
        cost_h = torch.empty(1, dtype=torch.float64).pin_memory()
        Xd = torch.empty_like(Xg)
        xn2 = torch.empty(n, dtype=torch.float32, device=env.dev)
        Xb2 = torch.empty((n, d), dtype=torch.bfloat16, device=env.dev) if form == "bf16" else None
        Xr2 = torch.empty(n, dtype=torch.float32, device=env.dev) if form == "bf16" else None
        Ce, Cen = R["C"].clone(), torch.empty_like(C0)
        lab2 = torch.empty(n, dtype=torch.int32, device=env.dev)
        co2 = torch.empty(2, dtype=torch.float64, device=env.dev)
        st = {"C": Ce, "Cn": Cen}

        def lloyd_and_readback(Xs=None, xns=None, Xbs=None, Xrs=None):
            Xs = Xd if Xs is None else Xs
            xns, Xbs, Xrs = (xn2, Xb2, Xr2) if xns is None else (xns, Xbs, Xrs)
            B.kmeans_assign(Xs, st["C"], Xop=Xbs, Xop_scales=Xrs, xnorm=xns, compute=form, engine=engine,
                            labels=lab2, ctx=ctx)
            B.kmeans_update(Xs, lab2, st["C"], C_new=st["Cn"], cost_old=co2[0:1], cost_new=co2[1:2], ctx=ctx)
            Ch_out.copy_(st["Cn"], non_blocking=True)
            cost_h.copy_(co2[1:2], non_blocking=True)
            st["C"], st["Cn"] = st["Cn"], st["C"]

        def e2e_step(i):
            # one read of X from the mapped host block: device copy, norms, BF16 copy and residuals
            B.kmeans_ingest(hb.tensor, X_dev=Xd, xnorm=xn2, Xq=Xb2, resid=Xr2, quantize=Xb2 is not None,
                            device=env.dev, ctx=ctx)
            lloyd_and_readback()

        def e2e_step_copy_engine(i):
            Xd.copy_(Xh, non_blocking=True)
            B.kmeans_row_norms(Xd, xnorm=xn2, ctx=ctx)
            if Xb2 is not None:
                B.kmeans_quantize(Xd, "bf16", Xq=Xb2, scales=Xr2, ctx=ctx)
            lloyd_and_readback()

        # pipelined: step i's ingest runs on a second stream (its own context and a second set of
        # buffers) while step i - 1's Lloyd iteration and read-back run on the main one
        s_ing = torch.cuda.Stream(device=env.dev)
        ctx_ing = B.Context(env.dev.index)
        pbuf = [(torch.empty_like(Xg), torch.empty(n, dtype=torch.float32, device=env.dev),
                 torch.empty((n, d), dtype=torch.bfloat16, device=env.dev) if Xb2 is not None else None,
                 torch.empty(n, dtype=torch.float32, device=env.dev) if Xb2 is not None else None)
                for _ in range(2)]
        ev_ready = [torch.cuda.Event() for _ in range(2)]
        ev_free = [torch.cuda.Event() for _ in range(2)]

        def e2e_step_pipelined(i):
            b = i % 2
            Xs, xns, Xbs, Xrs = pbuf[b]
            with torch.cuda.stream(s_ing):
                s_ing.wait_event(ev_free[b])  # the Lloyd step that last read this buffer
                B.kmeans_ingest(hb.tensor, X_dev=Xs, xnorm=xns, Xq=Xbs, resid=Xrs, quantize=Xbs is not None,
                                device=env.dev, ctx=ctx_ing)
                ev_ready[b].record(s_ing)
            torch.cuda.current_stream(env.dev).wait_event(ev_ready[b])
            lloyd_and_readback(Xs, xns, Xbs, Xrs)
            ev_free[b].record(torch.cuda.current_stream(env.dev))

        E = env.timed(e2e_step, args.e2e_steps or 5, 1, profile=False)
        Ec = env.timed(e2e_step_copy_engine, args.e2e_steps or 5, 1, profile=False)
        Ep = env.timed(e2e_step_pipelined, args.e2e_steps or 5, 2, profile=False)
        e2e = {"value": env.ranks.whole_job(F, E["ms"]) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(n * d * 4), "d2h_bytes_per_step": int(k * d * 4 + 8),
               "ms_per_step": E["ms"],
               "pipelined": {"value": env.ranks.whole_job(F, Ep["ms"]) / 1e9, "ms_per_step": Ep["ms"],
                             "note": "step i's ingest on a second stream and context (two buffer sets) issued "
                                     "while step i - 1's Lloyd iteration runs: no faster, since the ingest "
                                     "kernel holds every SM while it waits on the host link"},
               "copy_engine": {"value": env.ranks.whole_job(F, Ec["ms"]) / 1e9, "ms_per_step": Ec["ms"],
                               "note": "X copied by the copy engine from torch-pinned memory, then norms and "
                                       "the operand copy as separate passes"},
               "note": "every step: X read from a mapped host block (kmeans_ingest: device copy, norms, BF16 "
                       "copy and residuals in one pass, at the host link's rate: 209 GB/s here, as fast as a "
                       "copy-engine copy of pinned memory), assign, update, and D2H of the centers and the cost"}
        del hb, pbuf

    forms = None
    if form == "bf16" and not args.no_compare:
        s32 = max(3, min(args.steps, args.steps // 2))
        R32 = lloyd_timed(env, Xg, None, None, xnorm, C0, "f32", "tcgen05", s32, args.warmup)
        v32 = env.ranks.whole_job(F, R32["ms"]) / 1e9
        it = args.warmup + min(s32, args.steps) - 1
        c16, c32 = float(R["costs"][it, 1]), float(R32["costs"][it, 1])
        forms = {"bf16": {"value": value, "ms_per_step": ms},
                 "f32_3xtf32": {"value": v32, "ms_per_step": R32["ms"],
                                "assign_ms": kernel_avg_s(R32["prof"], "assign_tc") * 1e3},
                 "speedup_vs_f32": value / v32, "final_cost_rel_gap": abs(c16 - c32) / c32,
                 "note": "both forms run the same Lloyd iterations from the same seeds; labels are exact in "
                         "both (certified near-ties re-resolved), so costs agree to rounding"}

    cpu = None
    if env.rank == 0 and env.world == 1 and not args.no_cpu_baseline:
        cpu = oracle_assign_update_rate(X, R["C"].cpu().numpy(), args.cpu_seconds)

    if hidden is None:
        wdesc = f"gaussian mixture n={n} d={d} k={k} ({k} components, seed = rank), one Lloyd iteration per step"
    else:
        wdesc = (f"StructuredWithNoise: {k} hidden sets x {n // k} points, d={d}, {SWN_X} signal dimensions per "
                 f"set in [-10, 10], the rest in [-1/2, 1/2] (seed = rank), k={k}, one Lloyd iteration per step")
    line = base_line(env, args.workload, value, ms, args.steps, args.warmup, form, {
        "workload": wdesc,
        "form": form + ("x2 (two-term centers)" if form == "bf16" and args.center_terms == 2 else ""),
        "engine": engine,
        "l2": f"inputs larger than L2 (X is {n * d * 4 / 1e6:.0f} MB FP32 / {n * d * 2 / 1e6:.0f} MB BF16)",
        "parallelism": "replicas" if env.world > 1 else "single GPU"})
    line.update({"roofline": roof, "rooflines": rooflines, "step_roofline": step_roof, "pipeline": pipeline,
                 "forms": forms,
                 "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": R["launches"], "clocks": R["clocks"],
                 "kernels_ms": kernels_ms(prof), "points_per_s": env.ranks.whole_job(n, ms),
                 "rechecked_per_step": float(np.mean(R["rechecked"][args.warmup:])),
                 "cost_last": float(R["costs"][-1, 1])})
    return line


def run_small(env, args):
    import numpy as np

    torch, B = env.torch, env.B
    from paper_1502_04265_gb300 import synth

    n, d, k, iters = 10_000, 64, 10, 20
    F = iters * (2.0 * n * k * d + n * d)
    X = mixture(n, d, 10, seed=env.rank)
    u = synth.seed_uniforms(k, seed=env.rank)
    Xg = torch.from_numpy(X).to(env.dev)
    ug = torch.from_numpy(u).to(env.dev)
    ctx = env.ctx
    xn = torch.empty(n, dtype=torch.float32, device=env.dev)
    idx = torch.empty(k, dtype=torch.int64, device=env.dev)
    Ca, Cb = torch.empty((k, d), dtype=torch.float32, device=env.dev), torch.empty((k, d), dtype=torch.float32, device=env.dev)
    labels = torch.empty(n, dtype=torch.int32, device=env.dev)
    tr = torch.zeros((iters, 2), dtype=torch.float64, device=env.dev)
    flush_buf = torch.empty(64 << 20, dtype=torch.float32, device=env.dev)   # 256 MB > L2

    def run(i):
        B.kmeans_row_norms(Xg, xnorm=xn, ctx=ctx)
        B.kmeans_seed_pp(Xg, k, ug, idx_out=idx, C_out=Ca, ctx=ctx)
        cur, nxt = Ca, Cb
        for t in range(iters):
            B.kmeans_assign(Xg, cur, xnorm=xn, compute="f32", engine=args.engine, labels=labels, ctx=ctx)
            B.kmeans_update(Xg, labels, cur, C_new=nxt, cost_old=tr[t, 0:1], cost_new=tr[t, 1:2], ctx=ctx)
            cur, nxt = nxt, cur

    R = env.timed(run, args.steps, args.warmup, clocks=True, flush=lambda: flush_buf.fill_(1.0))
    ms, prof = R["ms"], R["prof"]
    value = env.ranks.whole_job(F, ms) / 1e9
    kname = max((nm for nm in prof), key=lambda nm: prof[nm][1])
    bytes_per = {"assign_tc": n * d * 4 + k * d * 4 + n * 4, "assign_simt": n * d * 4 + k * d * 4 + n * 4,
                 "update": n * d * 4 + n * 4 + k * (d + 2) * 8, "seed": (k - 1) * n * d * 4,
                 "recheck": n * 4, "center_prep": k * d * 4, "row_norms": n * d * 4}
    roof = roofline(env.peaks, kname, kernel_avg_s(prof, kname), bytes_per.get(kname, n * d * 4), 0.0,
                    FFMA_PEAK_TFLOPS, R["total_s"], bound="hbm",
                    note="latency-bound: X (2.56 MB) is in L2 after its first read within a run and every "
                         "kernel is a few microseconds; the fraction is not meaningful")
    us_iter = sum(prof[nm][1] for nm in prof if nm in ("assign_tc", "assign_simt", "recheck", "center_prep",
                                                         "update")) / max(args.steps, 1) / iters * 1e3

    e2e = None
    if not args.no_e2e:
        Xh = torch.from_numpy(X).pin_memory()
        Ch = torch.empty((k, d), dtype=torch.float32).pin_memory()
        Lh = torch.empty(n, dtype=torch.int32).pin_memory()
        Xd = torch.empty_like(Xg)

        def e2e_step(i):
            Xd.copy_(Xh, non_blocking=True)
            B.kmeans_row_norms(Xd, xnorm=xn, ctx=ctx)
            B.kmeans_seed_pp(Xd, k, ug, idx_out=idx, C_out=Ca, ctx=ctx)
            cur, nxt = Ca, Cb
            for t in range(iters):
                B.kmeans_assign(Xd, cur, xnorm=xn, compute="f32", engine=args.engine, labels=labels, ctx=ctx)
                B.kmeans_update(Xd, labels, cur, C_new=nxt, cost_old=tr[t, 0:1], cost_new=tr[t, 1:2], ctx=ctx)
                cur, nxt = nxt, cur
            Ch.copy_(cur, non_blocking=True)
            Lh.copy_(labels, non_blocking=True)

        E = env.timed(e2e_step, args.e2e_steps or 10, 2, flush=lambda: flush_buf.fill_(1.0), profile=False)
        e2e = {"value": env.ranks.whole_job(F, E["ms"]) / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(n * d * 4),
               "d2h_bytes_per_step": int(k * d * 4 + n * 4), "ms_per_step": E["ms"]}

    cpu = None
    if env.rank == 0 and env.world == 1 and not args.no_cpu_baseline:
        reps = [(X, k, u)] * 1000
        cpu = oracle_lloyd_rate(reps, iters, min(args.cpu_seconds, 5.0))

    line = base_line(env, "small", value, ms, args.steps, args.warmup, "f32", {
        "workload": f"gaussian mixture n={n} d={d} k={k} (10 components, seed = rank); a step is row norms + "
                    f"k-means++ + {iters} Lloyd iterations, FP32", "form": "f32", "engine": args.engine,
        "l2": "L2 flushed (256 MB written) before every timed step",
        "parallelism": "replicas" if env.world > 1 else "single GPU"})
    line.update({"roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": R["launches"],
                 "clocks": R["clocks"], "kernels_ms": kernels_ms(prof), "us_per_iteration": us_iter,
                 "run_ms": ms, "points_per_s": env.world * n * iters / (ms * 1e-3),
                 "cost_last": float(tr[-1, 1].item())})
    return line


def _stream_chunk(job):
    d, r, seed, row0, rows, comps = job
    from paper_1502_04265_gb300 import synth

    Q = synth.orthonormal_basis(d, r, seed)
    X, _ = synth.subspace_mixture_chunk(Q, row0, rows, comps, seed)
    return X


def run_stream(env_args):
    env, args = env_args
    import numpy as np

    torch, B = env.torch, env.B
    from paper_1502_04265_gb300 import synth

    n, d, r, k, comps, iters, chunk = 2_000_000, 2048, 64, 1000, 500, 20, 65536
    seed = env.rank
    chunks = [(r0, min(n, r0 + chunk)) for r0 in range(0, n, chunk)]
    ex, futs = env.pool
    ctx = env.ctx
    Xg = torch.empty((n, d), dtype=torch.float32, device=env.dev)
    Xb = torch.empty((n, d), dtype=torch.bfloat16, device=env.dev)
    pinned = []
    for (r0, r1), f in zip(chunks, futs):
        Xc = torch.from_numpy(f.result()).pin_memory()
        pinned.append(Xc)
        Xg[r0:r1].copy_(Xc, non_blocking=True)
        B.kmeans_quantize(Xg[r0:r1], "bf16", Xq=Xb[r0:r1], residuals=False, ctx=ctx)
    ex.shutdown()
    Q = synth.orthonormal_basis(d, r, seed)
    V = torch.from_numpy(Q.astype(np.float32)).to(env.dev)
    u = synth.seed_uniforms(k, seed=seed)
    ug = torch.from_numpy(u).to(env.dev)
    Y = torch.empty((n, r), dtype=torch.float32, device=env.dev)
    ctx.sync()

    def project(src):
        for r0, r1 in chunks:
            B.kmeans_project_block(src[r0:r1], V, Y=Y[r0:r1], ctx=ctx)

    P32 = env.once(lambda: project(Xg))
    P16 = env.once(lambda: project(Xb))          # Y from the BF16 projection feeds the rest
    yn = B.kmeans_row_norms(Y, ctx=ctx)
    Yb, Yr = B.kmeans_quantize(Y, "bf16", ctx=ctx)
    Y8, s8 = B.kmeans_quantize(Y, "fp8", ctx=ctx)
    idx = torch.empty(k, dtype=torch.int64, device=env.dev)
    C0 = torch.empty((k, r), dtype=torch.float32, device=env.dev)
    S = env.once(lambda: B.kmeans_seed_pp(Y, k, ug, idx_out=idx, C_out=C0, ctx=ctx))
    ctx.sync()

    F = 2.0 * n * k * r + n * r
    # the primary form: the faster exact one at this shape (FP32 3xTF32 below 256 dimensions, where
    # BF16's certified band holds most points and their recheck costs more than the halved read)
    pf = primary_form(args.form, r)
    R = lloyd_timed(env, Y, Yb if pf == "bf16" else None, Yr if pf == "bf16" else None, yn, C0, pf,
                    args.engine if pf == "bf16" else "tcgen05",
                    args.steps, args.warmup, clocks=True, center_terms=args.center_terms if pf == "bf16" else 1)
    ms, prof = R["ms"], R["prof"]
    value = env.ranks.whole_job(F, ms) / 1e9
    peaks = env.peaks
    es = 2 if pf == "bf16" else 4
    roof = roofline(peaks, "assign_tc", kernel_avg_s(prof, "assign_tc"), n * r * es + k * r * es + n * 4,
                    2.0 * n * k * r, unit_peak(peaks, pf, True, R["total_s"]), R["total_s"],
                    bound=None if pf == "bf16" else "tensor",
                    note=None if pf == "bf16" else "3xTF32: max(probed kind::tf32, measured BF16 x nominal TF32/BF16 ratio) / 3",
                    traffic=stored_traffic(f"assign_tc/{pf}/{n}x{r}_k{k}"))

    def proj_roof(P, es):
        nl = len(chunks)
        avg = kernel_avg_s(P["prof"], "project")
        bytes_ = (n * d * es + n * r * 4) / nl + d * r * es
        return {"ms_all_chunks": P["ms"], "launches": nl, "kernel_ms": avg * 1e3,
                "achieved_gbs": bytes_ / avg / 1e9, "frac_hbm": bytes_ / avg / 1e9 / peaks["hbm_gbs"],
                "tflops": 2.0 * n * d * r / nl / avg / 1e12}

    forms = None
    if not args.no_compare:
        s2 = max(3, args.steps // 2)
        R8 = lloyd_timed(env, Y, Y8, s8, yn, C0, "fp8", args.engine, s2, args.warmup)
        if pf == "bf16":
            R16, R32 = R, lloyd_timed(env, Y, None, None, yn, C0, "f32", "tcgen05", s2, args.warmup)
        else:
            R16, R32 = lloyd_timed(env, Y, Yb, Yr, yn, C0, "bf16", args.engine, s2, args.warmup), R
        # BF16 with two-term centers: the band then grows with the rows' own rounding residuals and
        # the two centers' distances, not with max ||c||
        R16x2 = lloyd_timed(env, Y, Yb, Yr, yn, C0, "bf16", args.engine, s2, args.warmup, center_terms=2)
        it = args.warmup + s2 - 1
        c16, c8, c32 = (float(x["costs"][it, 1]) for x in (R16, R8, R32))
        v16, v8, v32 = (env.ranks.whole_job(F, x["ms"]) / 1e9 for x in (R16, R8, R32))
        forms = {"bf16": {"value": v16, "ms_per_step": R16["ms"], "assign_ms": kernel_avg_s(R16["prof"], "assign_tc") * 1e3,
                          "rechecked_per_step": float(np.mean(R16["rechecked"][args.warmup:]))},
                 "fp8": {"value": v8, "ms_per_step": R8["ms"], "assign_ms": kernel_avg_s(R8["prof"], "assign_tc") * 1e3,
                         "rechecked_per_step": float(np.mean(R8["rechecked"][args.warmup:])),
                         "final_cost_rel_gap_vs_f32": abs(c8 - c32) / c32},
                 "f32_3xtf32": {"value": v32, "ms_per_step": R32["ms"],
                                "assign_ms": kernel_avg_s(R32["prof"], "assign_tc") * 1e3},
                 "bf16x2": {"value": env.ranks.whole_job(F, R16x2["ms"]) / 1e9, "ms_per_step": R16x2["ms"],
                            "assign_ms": kernel_avg_s(R16x2["prof"], "assign_tc") * 1e3,
                            "rechecked_per_step": float(np.mean(R16x2["rechecked"][args.warmup:])),
                            "final_cost_rel_gap_vs_f32": abs(float(R16x2["costs"][it, 1]) - c32) / c32},
                 "primary": pf, "speedup_bf16_vs_f32": v16 / v32, "speedup_fp8_vs_f32": v8 / v32,
                 "speedup_bf16x2_vs_f32": env.ranks.whole_job(F, R16x2["ms"]) / 1e9 / v32,
                 "final_cost_rel_gap_bf16_vs_f32": abs(c16 - c32) / c32,
                 "note": "the three forms run the same Lloyd iterations from the same k-means++ centers"}

    # whole run from the device-resident BF16 points: projection, norms, operand copy, k-means++, iterations
    labels = torch.empty(n, dtype=torch.int32, device=env.dev)
    Ca, Cb = torch.empty_like(C0), torch.empty_like(C0)
    tr = torch.zeros((iters, 2), dtype=torch.float64, device=env.dev)

    def whole(src_chunks=None):
        if src_chunks is None:
            project(Xb)
        else:
            for (r0, r1), Xc in zip(chunks, src_chunks):
                Xg[r0:r1].copy_(Xc, non_blocking=True)
                B.kmeans_quantize(Xg[r0:r1], "bf16", Xq=Xb[r0:r1], residuals=False, ctx=ctx)
                B.kmeans_project_block(Xb[r0:r1], V, Y=Y[r0:r1], ctx=ctx)
        B.kmeans_row_norms(Y, xnorm=yn, ctx=ctx)
        if pf == "bf16":
            B.kmeans_quantize(Y, "bf16", Xq=Yb, scales=Yr, ctx=ctx)
        B.kmeans_seed_pp(Y, k, ug, idx_out=idx, C_out=Ca, ctx=ctx)
        cur, nxt = Ca, Cb
        for t in range(iters):
            B.kmeans_assign(Y, cur, Xop=Yb if pf == "bf16" else None, Xop_scales=Yr if pf == "bf16" else None,
                            xnorm=yn, compute=pf,
                            engine=args.engine if pf == "bf16" else "tcgen05", labels=labels, ctx=ctx)
            B.kmeans_update(Y, labels, cur, C_new=nxt, cost_old=tr[t, 0:1], cost_new=tr[t, 1:2], ctx=ctx)
            cur, nxt = nxt, cur
        return cur

    W = env.once(whole)
    Fw = iters * F
    pipeline = {"projection_bf16": proj_roof(P16, 2), "projection_tf32": proj_roof(P32, 4),
                "seed_ms": S["ms"], "iterations": iters, "total_ms": W["ms"],
                "gflops_whole_run": Fw / (W["ms"] * 1e-3) / 1e9,
                "note": "whole run from device-resident BF16 points: 31 projections, norms, (BF16 copy of Y for "
                        "the BF16 form), k-means++ (k=1000 rounds over Y), 20 Lloyd iterations in the primary form; "
                        "seeding time counted, its flops not"}

    e2e = None
    if not args.no_e2e:
        Ch = torch.empty((k, r), dtype=torch.float32).pin_memory()
        Lh = torch.empty(n, dtype=torch.int32).pin_memory()

        def e2e_step(i):
            C = whole(pinned)
            Ch.copy_(C, non_blocking=True)
            Lh.copy_(labels, non_blocking=True)

        E = env.timed(e2e_step, args.e2e_steps or 2, 1, profile=False)
        e2e = {"value": env.ranks.whole_job(Fw, E["ms"]) / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(n * d * 4),
               "d2h_bytes_per_step": int(k * r * 4 + n * 4), "ms_per_step": E["ms"],
               "note": "a step is the whole job from FP32 chunks in pinned host memory: H2D, BF16 copy, "
                       "projection, norms, k-means++, 20 iterations, D2H of centers and labels"}

    cpu = None
    if env.rank == 0 and env.world == 1 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        Xs = pinned[0].numpy()[:16384]
        Ys = oracle.project(Xs, Q).astype(np.float32)
        Cs = Ys[(u * Ys.shape[0]).astype(np.int64) % Ys.shape[0]]
        cpu = oracle_assign_update_rate(Ys, Cs, args.cpu_seconds,
                                        label="coordinates of chunk 0 projected by the oracle; ")

    line = base_line(env, "stream", value, ms, args.steps, args.warmup, "bf16" if pf == "bf16" else "f32", {
        "workload": f"{n} points, d={d}, {comps}-component mixture in a random rank-{r} subspace + N(0, 0.1^2) "
                    f"noise, {len(chunks)} chunks of {chunk} projected in BF16; k={k} on the r={r} coordinates, one "
                    f"Lloyd iteration per step", "form": pf if pf == "bf16" else "f32_3xtf32",
        "form_policy": "the faster exact form at the shape: FP32 (3xTF32) below d=256, BF16 + recheck above; "
                       "every form is listed under forms", "engine": args.engine,
        "l2": "inputs larger than L2 (Y BF16 256 MB; X 16.4 GB FP32 / 8.2 GB BF16)",
        "parallelism": "replicas" if env.world > 1 else "single GPU"})
    line.update({"roofline": roof, "pipeline": pipeline, "forms": forms, "cpu_baseline": cpu, "e2e": e2e,
                 "gpu_launches": R["launches"], "clocks": R["clocks"], "kernels_ms": kernels_ms(prof),
                 "points_per_s": env.ranks.whole_job(n, ms), "cost_last": float(R["costs"][-1, 1])})
    return line


def _batch_problem(job):
    n, d, k, seed = job
    from paper_1502_04265_gb300 import synth

    X, _ = synth.gaussian_mixture(n, d, k, seed=seed)
    return X


def batch_jobs(count, rank):
    from paper_1502_04265_gb300 import synth

    shapes = synth.batch_problem_list(count, seed=rank)
    return shapes, [(s["n"], s["d"], s["k"], 1_000_000 * rank + s["seed"]) for s in shapes]


def run_batch(env_args):
    env, args = env_args
    import numpy as np

    torch, B = env.torch, env.B
    from paper_1502_04265_gb300 import synth

    S, iters = 4, 20
    shapes, jobs = env.batch_shapes
    ex, futs = env.pool
    ctx = env.ctx
    hostX, probs = [], []
    for s, f in zip(shapes, futs):
        Xh = torch.from_numpy(f.result()).pin_memory()
        hostX.append(Xh)
        U = np.stack([synth.seed_uniforms(s["k"], seed=s["seed"] * S + j) for j in range(S)])
        probs.append({"X": Xh.to(env.dev, non_blocking=True), "k": s["k"], "u": torch.from_numpy(U).to(env.dev)})
    ex.shutdown()
    ctx.sync()
    F = sum(S * iters * (2.0 * s["n"] * s["k"] * s["d"] + s["n"] * s["d"]) for s in shapes)
    n_tot = sum(s["n"] for s in shapes)
    xbytes = sum(s["n"] * s["d"] * 4 for s in shapes)

    def record(compute):
        t0 = time.perf_counter()
        B.kmeans_batch_run(probs, S, iters, compute=compute, graph=True, autotune=True, ctx=ctx)
        ctx.sync()
        return time.perf_counter() - t0

    # one form for the whole batched launch: the faster exact form for its smallest dimension
    pf = primary_form(args.form, min(s["d"] for s in shapes))
    first_s = record(pf)
    costs_p = [p["cost_out"].clone() for p in probs]
    R = env.timed(lambda i: B.kmeans_batch_replay(ctx=ctx), args.steps, args.warmup - 1, clocks=True, profile=False)
    ms = R["ms"]
    value = env.ranks.whole_job(F, ms) / 1e9
    ok = all(torch.equal(p["cost_out"], c) for p, c in zip(probs, costs_p))

    # per-kernel times from one run that is not recorded into a graph
    Pn = env.once(lambda: B.kmeans_batch_run(probs, S, iters, compute=pf, graph=False, ctx=ctx), warmup=0)
    prof = Pn["prof"]
    peaks = env.peaks
    es = 2 if pf == "bf16" else 4
    a_bytes = sum(s["n"] * s["d"] * es + S * s["k"] * s["d"] * es + S * s["n"] * 4 for s in shapes)
    a_flops = sum(2.0 * s["n"] * S * s["k"] * s["d"] for s in shapes)
    roof = roofline(peaks, "assign_batched", kernel_avg_s(prof, "assign_batched"), a_bytes, a_flops,
                    unit_peak(peaks, pf, True, R["total_s"]), R["total_s"],
                    traffic=stored_traffic(f"assign_batched/{pf}/c{len(shapes)}"),
                    note="per-launch time from a run outside the graph (the graph itself is timed as a whole)"
                         + ("" if pf == "bf16" else "; 3xTF32: measured BF16 peak x nominal TF32/BF16 ratio / 3"))
    per_iter = {nm: prof[nm][1] / max(prof[nm][0], 1) for nm in prof}

    forms = None
    if not args.no_compare:
        other = "bf16" if pf == "f32" else "f32"
        first_o = record(other)
        Ro = env.timed(lambda i: B.kmeans_batch_replay(ctx=ctx), max(2, args.steps // 2), 1, profile=False)
        gaps = []
        for p, cp in zip(probs, costs_p):
            a, b = cp[:, 1].cpu().numpy(), p["cost_out"][:, 1].cpu().numpy()
            gaps.append(float(np.max(np.abs(a - b) / b)))
        vo = env.ranks.whole_job(F, Ro["ms"]) / 1e9
        v16, ms16, f16 = (value, ms, first_s) if pf == "bf16" else (vo, Ro["ms"], first_o)
        v32, ms32, f32_ = (vo, Ro["ms"], first_o) if pf == "bf16" else (value, ms, first_s)
        forms = {"bf16": {"value": v16, "ms_per_step": ms16, "first_call_s": f16},
                 "f32_3xtf32": {"value": v32, "ms_per_step": ms32, "first_call_s": f32_},
                 "primary": pf, "speedup_bf16_vs_f32": v16 / v32, "max_final_cost_rel_gap": max(gaps),
                 "note": "same seeds in both forms; k-means++ is exact in both, so the runs agree up to "
                         "rounding of the FP32/FP64 sums"}

    e2e = None
    if not args.no_e2e:
        outs = [(torch.empty_like(p["C_out"], device="cpu").pin_memory(),
                 torch.empty_like(p["cost_out"], device="cpu").pin_memory()) for p in probs]

        def e2e_step(i):
            for p, Xh in zip(probs, hostX):
                p["X"].copy_(Xh, non_blocking=True)
            B.kmeans_batch_run(probs, S, iters, compute=pf, graph=True, autotune=True, ctx=ctx)
            for p, (Co, co) in zip(probs, outs):
                Co.copy_(p["C_out"], non_blocking=True)
                co.copy_(p["cost_out"], non_blocking=True)

        E = env.timed(e2e_step, args.e2e_steps or 2, 1, profile=False)
        e2e = {"value": env.ranks.whole_job(F, E["ms"]) / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(xbytes),
               "d2h_bytes_per_step": int(sum(p["C_out"].numel() * 4 + p["cost_out"].numel() * 8 for p in probs)),
               "ms_per_step": E["ms"], "note": "H2D of every problem's X, planning + recording + launch of "
                                               "the graph (tile widths cached), D2H of centers and costs"}

    cpu = None
    if env.rank == 0 and env.world == 1 and not args.no_cpu_baseline:
        runs = []
        for s, Xh in zip(shapes, hostX):
            for j in range(S):
                runs.append((Xh.numpy(), s["k"], synth.seed_uniforms(s["k"], seed=s["seed"] * S + j)))
        cpu = oracle_lloyd_rate(runs, iters, args.cpu_seconds, label="problems in list order; ")

    line = base_line(env, "batch", value, ms, args.steps, args.warmup, "bf16" if pf == "bf16" else "f32", {
        "workload": f"{len(shapes)} gaussian-mixture problems (n log-uniform [1e3, 1e5], d in {{32, 128, 512}}, "
                    f"k log-uniform [4, 256]; sum n = {n_tot}), {S} k-means++ seeds each, {iters} Lloyd "
                    f"iterations; a step is one replay of the recorded graph",
        "form": pf if pf == "bf16" else "f32_3xtf32",
        "form_policy": "one form per batched launch, the faster exact form for the smallest dimension in the "
                       "batch (FP32 3xTF32 below d=256); both forms are listed under forms",
        "l2": f"inputs larger than L2 ({xbytes / 1e9:.1f} GB FP32 points)",
        "parallelism": "replicas" if env.world > 1 else "single GPU"})
    line.update({"roofline": roof, "forms": forms, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": R["launches"],
                 "gpu_launches_note": "the kernels recorded in the graph, counted at every replay (one graph launch per step)",
                 "clocks": R["clocks"], "kernels_ms_outside_graph": per_iter, "first_call_s": first_s,
                 "replay_deterministic": bool(ok), "points_per_s": env.world * n_tot * S * iters / (ms * 1e-3)})
    return line


def run_learned(env, args):
    import numpy as np

    torch, B = env.torch, env.B
    from paper_1502_04265_gb300 import driver, synth
    from paper_1502_04265_gb300.learned import ProposalNet

    n, d, k, h, ntrain, nsub, topm = args.n or 4_000_000, 256, 16384, 256, 200_000, 200_000, 32
    ctx = env.ctx
    Xall = mixture(n + ntrain, d, k, seed=env.rank)
    Xg = torch.from_numpy(Xall[:n]).to(env.dev)
    Xtg = torch.from_numpy(Xall[n:]).to(env.dev)
    Xh, Xhr = B.kmeans_quantize(Xg, "bf16", ctx=ctx)
    u = synth.seed_uniforms(k, seed=env.rank)
    ug = torch.from_numpy(u).to(env.dev)
    t0 = time.perf_counter()
    fit = driver.lloyd(Xg[:nsub], k, 5, ug, compute="f32", ctx=ctx)
    C = fit["C"].contiguous()
    ctx.sync()
    centers_s = time.perf_counter() - t0
    lt = B.kmeans_assign(Xtg, C, compute="f32", ctx=ctx)
    net = ProposalNet(d, h, k, seed=env.rank, device=env.dev)
    Xtb, _ = B.kmeans_quantize(Xtg, "bf16", residuals=False, ctx=ctx)
    ctx.sync()
    t0 = time.perf_counter()
    losses = net.train(Xtb, lt, epochs=10, batch=4096, lr=3e-3, ctx=ctx)
    ctx.sync()
    train_s = time.perf_counter() - t0
    s2 = B.kmeans_center_separation(C, ctx=ctx)
    xnorm = B.kmeans_row_norms(Xg, ctx=ctx)
    exact = B.kmeans_assign(Xg, C, xnorm=xnorm, compute="f32", engine="tcgen05", ctx=ctx)
    ctx.sync()

    F = 2.0 * n * k * d + n * d
    K = args.steps
    lab = torch.empty(n, dtype=torch.int32, device=env.dev)
    nf = torch.zeros(2 * K + args.warmup, dtype=torch.int64, device=env.dev)
    cost = torch.zeros((2 * K + args.warmup, 2), dtype=torch.float64, device=env.dev)
    Cn = torch.empty_like(C)

    def step_learned(i):
        B.kmeans_learned_assign(net, Xg, Xh, C, s2, topm=topm, labels=lab, n_fallback=nf[i:i + 1], ctx=ctx)
        B.kmeans_update(Xg, lab, C, C_new=Cn, cost_old=cost[i, 0:1], cost_new=cost[i, 1:2], ctx=ctx)

    R = env.timed(step_learned, K, args.warmup, clocks=True)
    ms, prof = R["ms"], R["prof"]
    value = env.ranks.whole_job(F, ms) / 1e9
    mis = int((lab != exact).sum().item())
    nfb = nf.cpu().numpy()[args.warmup:]
    c_learn = float(cost[-1, 0].item())
    peaks = env.peaks
    fl_top = 2.0 * n * h * k
    roof = roofline(peaks, "mlp_topm", kernel_avg_s(prof, "mlp_topm"), n * h * 2 + k * h * 2 + n * topm * 4, fl_top,
                    bf16_peak(peaks, R["total_s"]), R["total_s"],
                    traffic=stored_traffic(f"mlp_topm/bf16/{n}x{h}_k{k}"),
                    note="the output layer (h=256 -> k logits) with the fused grouped top-32 proposal (the best "
                         "center of each 16-center group competes); the logits are never stored")

    def full_scan(compute, Xop, Xres, steps):
        lab2 = torch.empty(n, dtype=torch.int32, device=env.dev)
        c2 = torch.zeros((2 * steps + 1, 2), dtype=torch.float64, device=env.dev)
        Cn2 = torch.empty_like(C)

        def st(i):
            B.kmeans_assign(Xg, C, Xop=Xop, Xop_scales=Xres, xnorm=xnorm, compute=compute, engine="tcgen05",
                            labels=lab2, ctx=ctx)
            B.kmeans_update(Xg, lab2, C, C_new=Cn2, cost_old=c2[i, 0:1], cost_new=c2[i, 1:2], ctx=ctx)

        Rf = env.timed(st, steps, 1)
        Rf["cost"] = float(c2[steps, 0].item())
        Rf["mis"] = int((lab2 != exact).sum().item())
        return Rf

    forms = None
    if not args.no_compare:
        Rb = full_scan("bf16", Xh, Xhr, max(2, min(K, 3)))
        Rf = full_scan("f32", None, None, 2)
        vb, vf = (env.ranks.whole_job(F, x["ms"]) / 1e9 for x in (Rb, Rf))
        forms = {"learned": {"value": value, "ms_per_step": ms, "misassigned": mis, "cost": c_learn},
                 "bf16_full_scan": {"value": vb, "ms_per_step": Rb["ms"], "misassigned": Rb["mis"], "cost": Rb["cost"],
                                    "assign_ms": kernel_avg_s(Rb["prof"], "assign_tc") * 1e3},
                 "f32_full_scan_3xtf32": {"value": vf, "ms_per_step": Rf["ms"], "misassigned": Rf["mis"],
                                          "cost": Rf["cost"], "assign_ms": kernel_avg_s(Rf["prof"], "assign_tc") * 1e3},
                 "speedup_learned_vs_f32": Rf["ms"] / ms, "speedup_bf16_vs_f32": Rf["ms"] / Rb["ms"],
                 "cost_ratio_learned_vs_f32": c_learn / Rf["cost"],
                 "note": "misassigned = labels differing from the FP32 full scan's (exact) labels; costs are "
                         "cost(C, labels) from the FP64 CF sums with the frozen centers"}

    e2e = None
    if not args.no_e2e:
        Xhost = torch.from_numpy(Xall[:n]).pin_memory()
        Lh = torch.empty(n, dtype=torch.int32).pin_memory()
        ch = torch.empty(1, dtype=torch.float64).pin_memory()
        Xd = torch.empty_like(Xg)
        Xhd = torch.empty_like(Xh)

        def e2e_step(i):
            Xd.copy_(Xhost, non_blocking=True)
            B.kmeans_quantize(Xd, "bf16", Xq=Xhd, residuals=False, ctx=ctx)
            B.kmeans_learned_assign(net, Xd, Xhd, C, s2, topm=topm, labels=lab, ctx=ctx)
            B.kmeans_update(Xd, lab, C, C_new=Cn, cost_old=cost[0, 0:1], cost_new=cost[0, 1:2], ctx=ctx)
            Lh.copy_(lab, non_blocking=True)
            ch.copy_(cost[0, 0:1], non_blocking=True)

        E = env.timed(e2e_step, args.e2e_steps or 2, 1, profile=False)
        e2e = {"value": env.ranks.whole_job(F, E["ms"]) / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(n * d * 4),
               "d2h_bytes_per_step": int(n * 4 + 8), "ms_per_step": E["ms"]}

    cpu = None
    if env.rank == 0 and env.world == 1 and not args.no_cpu_baseline:
        Cs = Xall[(u * n).astype(np.int64) % n]
        cpu = oracle_assign_update_rate(Xall[:n], Cs, args.cpu_seconds)

    line = base_line(env, "learned", value, ms, K, args.warmup, "bf16", {
        "workload": f"gaussian mixture n={n} d={d} k={k} ({k} components, seed = rank) + {ntrain} held-out "
                    f"training points; centers: k-means++ on the first {nsub} points + 5 FP32 Lloyd iterations; "
                    f"MLP {d}-{h}-{h}-{k} GELU, top-{topm}; a step is the learned assignment + CF update",
        "form": "learned (BF16 MLP, FP32 exact candidates)", "l2": "inputs larger than L2 (X 4.1 GB FP32)",
        "parallelism": "replicas" if env.world > 1 else "single GPU"})
    line.update({"roofline": roof, "forms": forms, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": R["launches"],
                 "clocks": R["clocks"], "kernels_ms": kernels_ms(prof),
                 "fallback_rate": float(np.mean(nfb)) / n, "misassignment_rate": mis / n,
                 "training": {"epochs": 10, "batch": 4096, "train_s": train_s, "loss_first": losses[0],
                              "loss_last": losses[-1]},
                 "centers_s": centers_s, "points_per_s": env.ranks.whole_job(n, ms)})
    return line


# ---------------------------------------------------------------------------- randomised SVD of a piece
def svd_shape(args):
    return args.n or 65536, args.d or 2048, 64, 80


def svd_flops(n, d, s, ell):
    """Y = A Omega and Bt = A^T Q (2 n d s each), the two CholeskyQR passes (n s^2 for each Gram,
    2 n s^2 for each Y R^-1), the Gram of Bt (d s^2) and V = Bt T (2 d s l)."""
    return 4.0 * n * d * s + 6.0 * n * s * s + d * s * s + 2.0 * d * s * ell


def svd_piece(n, d, seed):
    from paper_1502_04265_gb300 import synth

    Qp = synth.orthonormal_basis(d, 64, seed)
    A, _ = synth.subspace_mixture_chunk(Qp, 0, n, 500, seed)
    return A, Qp


def oracle_svd_rate(A, Om, ell, cpu_seconds):
    """The FP64 oracle's randomised SVD on the first rows of the piece, repeated for about
    cpu_seconds; GFLOP/s by the same flop count."""
    import numpy as np

    from oracle import rsvd as orsvd

    d, s = Om.shape
    rows = min(A.shape[0], 8192)
    Ad, Omd = A[:rows].astype(np.float64), Om.astype(np.float64)
    reps, t0 = 0, time.perf_counter()
    while True:
        orsvd.rsvd(Ad, Omd, ell)
        reps += 1
        if time.perf_counter() - t0 >= cpu_seconds:
            break
    dt = time.perf_counter() - t0
    threads = os.environ.get("OMP_NUM_THREADS") or str(os.cpu_count() or 1)
    return {"value": reps * svd_flops(rows, d, s, ell) / dt / 1e9, "unit": UNIT, "cores": int(threads),
            "kind": "oracle",
            "sample": f"first {rows} of {A.shape[0]} rows x {reps} runs: numpy FP64 (BLAS threads = {threads}), "
                      f"{dt:.1f} s"}


def svd_rooflines(peaks, prof, n, d, s, total_s):
    """The SVD's two passes over the piece (sketch Y = A' Omega, row reduction Bt = A'^T Q): 3xTF32
    GEMMs on the tensor cores, one read of the piece each; the roofline takes the larger of the HBM
    time and the 3xTF32 time."""
    note = ("3xTF32 on tcgen05; peak max(probed kind::tf32, measured BF16 x nominal TF32/BF16 ratio) / 3; "
            "bound = the larger of the HBM and tensor times")
    out = {}
    for name in ("rsvd_sketch", "rsvd_rows"):
        if name in prof:
            out[name] = roofline(peaks, name, kernel_avg_s(prof, name), n * d * 4 + n * s * 4, 2.0 * n * d * s,
                                 unit_peak(peaks, "f32", True, total_s), total_s, note=note)
    return out


def run_svd(env, args):
    import numpy as np

    torch, B = env.torch, env.B
    from paper_1502_04265_gb300 import synth

    n, d, ell, s = svd_shape(args)
    A, Qp = svd_piece(n, d, env.rank)
    Om = synth.gaussian_sketch(d, s, seed=env.rank)
    Ag, Omg = torch.from_numpy(A).to(env.dev), torch.from_numpy(Om).to(env.dev)
    ctx = env.ctx
    V = torch.empty((d, ell), dtype=torch.float32, device=env.dev)
    sig = torch.empty(ell, dtype=torch.float32, device=env.dev)
    info = torch.zeros(1, dtype=torch.int32, device=env.dev)

    def step(i):
        B.kmeans_rsvd(Ag, Omg, ell, V=V, sigma=sig, info=info, ctx=ctx)

    R = env.timed(step, args.steps, args.warmup, clocks=True)
    ms, prof = R["ms"], R["prof"]
    F = svd_flops(n, d, s, ell)
    value = env.ranks.whole_job(F, ms) / 1e9
    rooflines = svd_rooflines(env.peaks, prof, n, d, s, R["total_s"])
    roof = max(rooflines.values(), key=lambda r: r["kernel_ms"])
    Vh = V.cpu().numpy().astype(np.float64)
    quality = {"info": int(info.item()) & 0xFF, "jacobi_sweeps": int(info.item()) >> 8,
               "orthonormality": float(np.max(np.abs(Vh.T @ Vh - np.eye(ell)))),
               "planted_subspace_distance": float(np.linalg.norm(Vh @ Vh.T - Qp @ Qp.T, 2)),
               "sigma_first_last": [float(sig[0]), float(sig[-1])]}

    e2e = None
    if not args.no_e2e:
        hb = B.HostBlock((n, d))
        hb.tensor.copy_(torch.from_numpy(A))
        Ad = torch.empty_like(Ag)
        xn = torch.empty(n, dtype=torch.float32, device=env.dev)
        Vh_out = torch.empty((d, ell), dtype=torch.float32).pin_memory()
        sh_out = torch.empty(ell, dtype=torch.float32).pin_memory()

        def e2e_step(i):
            B.kmeans_ingest(hb.tensor, X_dev=Ad, xnorm=xn, quantize=False, device=env.dev, ctx=ctx)
            B.kmeans_rsvd(Ad, Omg, ell, V=V, sigma=sig, info=info, ctx=ctx)
            Vh_out.copy_(V, non_blocking=True)
            sh_out.copy_(sig, non_blocking=True)

        E = env.timed(e2e_step, args.e2e_steps or 5, 1, profile=False)
        e2e = {"value": env.ranks.whole_job(F, E["ms"]) / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(n * d * 4),
               "d2h_bytes_per_step": int(d * ell * 4 + ell * 4), "ms_per_step": E["ms"],
               "note": "every step: the piece read from a mapped host block (kmeans_ingest), the SVD, and D2H "
                       "of V and the singular values"}
        del hb

    cpu = None
    if env.rank == 0 and env.world == 1 and not args.no_cpu_baseline:
        cpu = oracle_svd_rate(A, Om, ell, args.cpu_seconds)

    line = base_line(env, "svd", value, ms, args.steps, args.warmup, "f32", {
        "workload": f"one piece of the rank-64-subspace workload (n={n}, d={d}, 500-component mixture in a random "
                    f"64-dim subspace + N(0, 0.1^2) noise, seed = rank), top l={ell} right singular vectors with "
                    f"s={s} (16 oversampling columns), Gaussian Omega",
        "l2": f"inputs larger than L2 (A is {n * d * 4 / 1e6:.0f} MB)",
        "parallelism": "replicas" if env.world > 1 else "single GPU"})
    line.update({"roofline": roof, "rooflines": rooflines, "quality": quality, "cpu_baseline": cpu, "e2e": e2e,
                 "gpu_launches": R["launches"], "clocks": R["clocks"], "kernels_ms": kernels_ms(prof)})
    return line


# ---------------------------------------------------------------------------- BICO-style query
BICO_N, BICO_D, BICO_M = 1_000_000, 128, 20_000


def bico_inputs(seed, n=BICO_N):
    """The features' reference points (a 100-component mixture in R^128, the shape of the paper's
    Caltech128 SIFT vectors), their members and a batch of n arriving points with integer weights."""
    from paper_1502_04265_gb300 import synth

    refs, _ = synth.gaussian_mixture(BICO_M, BICO_D, 100, seed=seed)
    P, f = synth.bico_members(refs, seed)
    X = synth.bico_batch(refs, n, seed)
    w = synth.integer_weights(n, seed=seed, max_w=20)
    return refs, P, f, X, w


def bico_snapshot_torch(torch, P, f, m, dev):
    """The features' (N, S, Q) from their members, FP64 on the device (input preparation)."""
    Pd = torch.from_numpy(P).to(dev).double()
    fi = torch.from_numpy(f).to(dev).long()
    N = torch.zeros(m, dtype=torch.float64, device=dev).index_add_(0, fi, torch.ones_like(fi, dtype=torch.float64))
    S = torch.zeros((m, P.shape[1]), dtype=torch.float64, device=dev).index_add_(0, fi, Pd)
    Q = torch.zeros(m, dtype=torch.float64, device=dev).index_add_(0, fi, (Pd * Pd).sum(1))
    return N, S, Q


def oracle_bico_rate(X, w, refs, N, S, Q, T, cpu_seconds):
    """The FP64 oracle on a bounded sample of the batch: the nearest reference by the C full scan
    (OpenMP over points), then the insertion rule per point (oracle/bico.py)."""
    import numpy as np

    import oracle
    from oracle import bico as OB

    oracle.build()
    cores = oracle.set_threads(os.cpu_count() or 1)
    m, d = refs.shape
    cerr = np.array([OB.cf_error(N[j], S[j], Q[j]) for j in range(m)])
    Rd = refs.astype(np.float64)
    rows, t0, done = 256, time.perf_counter(), 0
    while True:
        Xs = X[done % X.shape[0]: done % X.shape[0] + rows]
        j, _, _ = oracle.assign(Xs, Rd)
        for i in range(Xs.shape[0]):
            mu = S[j[i]] / N[j[i]]
            diff = Xs[i].astype(np.float64) - mu
            OB.insertable(N[j[i]], cerr[j[i]], T, float(diff @ diff), float(w[(done + i) % X.shape[0]]))
        done += Xs.shape[0]
        dt = time.perf_counter() - t0
        if dt >= cpu_seconds:
            break
    flops = done * (2.0 * m * d + 3.0 * d)
    return {"value": flops / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{done} points of the batch against all {m} features in chunks of {rows}: FP64 C full scan "
                      f"(OpenMP over points) + the insertion rule per point, {dt:.1f} s"}


def run_bico(env, args):
    import numpy as np

    torch, B = env.torch, env.B
    from paper_1502_04265_gb300 import driver

    refs, P, f, X, w = bico_inputs(env.rank)
    n, d, m = X.shape[0], BICO_D, BICO_M
    dev = env.dev
    N, S, Q = bico_snapshot_torch(torch, P, f, m, dev)
    cerr = (Q - (S * S).sum(1) / N).cpu().numpy()
    T = float(np.quantile(cerr, 0.8))
    Xg, Rg, wg = torch.from_numpy(X).to(dev), torch.from_numpy(refs).to(dev), torch.from_numpy(w).to(dev)
    ctx = env.ctx
    xnorm = B.kmeans_row_norms(Xg, ctx=ctx)
    ref = torch.empty(n, dtype=torch.int32, device=dev)
    d2 = torch.empty(n, dtype=torch.float64, device=dev)
    take = torch.empty(n, dtype=torch.float64, device=dev)
    F = 2.0 * n * m * d + 3.0 * n * d

    def run_form(form, steps, clocks):
        Xop, Xr = B.kmeans_quantize(Xg, "bf16", ctx=ctx) if form == "bf16" else (None, None)

        def step(i):
            B.kmeans_bico_query(Xg, Rg, N, S, Q, T, w=wg, Xop=Xop, Xop_scales=Xr, xnorm=xnorm, compute=form,
                                ref_out=ref, d2_out=d2, take_out=take, ctx=ctx)

        return env.timed(step, steps, args.warmup, clocks=clocks)

    form = primary_form(args.form, d)
    R = run_form(form, args.steps, True)
    ms, prof = R["ms"], R["prof"]
    value = env.ranks.whole_job(F, ms) / 1e9
    wn = w.astype(np.float64)
    tk = take.cpu().numpy()
    outcome = {"whole": int((tk == wn).sum()), "part": int(((tk > 0) & (tk < wn)).sum()), "none": int((tk == 0).sum()),
               "threshold": T}
    peaks = env.peaks
    kname = assign_kernel(prof)
    es = 2 if form == "bf16" else 4
    rooflines = {kname: roofline(peaks, kname, kernel_avg_s(prof, kname), n * d * es + m * d * es + n * 4,
                                 2.0 * n * m * d, unit_peak(peaks, form, kname == "assign_tc", R["total_s"]),
                                 R["total_s"], bound="tensor",
                                 note=None if form == "bf16" else
                                 "3xTF32: max(probed kind::tf32, measured BF16 x nominal TF32/BF16 ratio) / 3"),
                 "bico_take": roofline(peaks, "bico_take", kernel_avg_s(prof, "bico_take"),
                                       n * d * 4 + n * (4 + 4 + 8 + 8) + m * d * 8 * 2, 3.0 * n * d + 8.0 * n,
                                       fp64_peak(peaks), R["total_s"], bound="alu",
                                       note="FP64-bound (ncu: FP64 pipe 87% busy, DRAM 9%): per element of "
                                            "||x - mu||^2 one subtraction and one FMA (3 flops; the FP32 -> FP64 "
                                            "conversions occupy the pipe too, uncounted), per point the rule's "
                                            "divisions and products; peak = max(probed FP64, 1.25 TFLOP/s)")}
    roof = max(rooflines.values(), key=lambda r: r["kernel_ms"])
    forms = {form: {"value": value, "ms_per_step": ms}}
    if not args.no_compare:
        other = "bf16" if form == "f32" else "f32"
        R2 = run_form(other, max(3, args.steps // 2), False)
        forms[other] = {"value": env.ranks.whole_job(F, R2["ms"]) / 1e9, "ms_per_step": R2["ms"],
                        "note": "the same query in the other exact form (labels exact in both)"}

    e2e = None
    if not args.no_e2e:
        hb = B.HostBlock((n, d))
        hb.tensor.copy_(torch.from_numpy(X))
        Xd = torch.empty_like(Xg)
        take_h = torch.empty(n, dtype=torch.float64).pin_memory()
        ref_h = torch.empty(n, dtype=torch.int32).pin_memory()

        def e2e_step(i):
            B.kmeans_ingest(hb.tensor, X_dev=Xd, xnorm=xnorm, quantize=False, device=dev, ctx=ctx)
            B.kmeans_bico_query(Xd, Rg, N, S, Q, T, w=wg, xnorm=xnorm, compute="f32" if form == "f32" else form,
                                Xop=None if form == "f32" else B.kmeans_quantize(Xd, "bf16", ctx=ctx)[0],
                                ref_out=ref, d2_out=d2, take_out=take, ctx=ctx)
            take_h.copy_(take, non_blocking=True)
            ref_h.copy_(ref, non_blocking=True)

        E = env.timed(e2e_step, args.e2e_steps or 5, 3, profile=False)
        e2e = {"value": env.ranks.whole_job(F, E["ms"]) / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(n * d * 4),
               "d2h_bytes_per_step": int(n * (8 + 4)), "ms_per_step": E["ms"],
               "note": "every step: the batch read from a mapped host block (kmeans_ingest), the query, and D2H of "
                       "every point's reference and insertable count"}
        del hb

    cpu = None
    if env.rank == 0 and env.world == 1 and not args.no_cpu_baseline:
        cpu = oracle_bico_rate(X, w, refs, N.cpu().numpy(), S.cpu().numpy(), Q.cpu().numpy(), T, args.cpu_seconds)

    line = base_line(env, "bico", value, ms, args.steps, args.warmup, form, {
        "workload": f"a batch of n={n} weighted points (integer weights 1..20) arriving at a BICO-style summary of "
                    f"m={m} features (200 k for k = 100) in d={d} (the shape of the paper's Caltech128 SIFT "
                    f"vectors; references from a 100-component mixture, 1..8 members per feature), threshold T = "
                    f"the 0.8 quantile of the features' errors; seed = rank",
        "l2": f"inputs larger than L2 (X is {n * d * 4 / 1e6:.0f} MB)",
        "parallelism": "replicas" if env.world > 1 else "single GPU"})
    line.update({"roofline": roof, "rooflines": rooflines, "forms": forms, "outcome": outcome, "cpu_baseline": cpu,
                 "e2e": e2e, "gpu_launches": R["launches"], "clocks": R["clocks"], "kernels_ms": kernels_ms(prof)})
    return line


# ---------------------------------------------------------------------------- per-piece bases + lift
PIECY_PIECES, PIECY_ROWS, PIECY_D, PIECY_ELL, PIECY_S = 8, 65536, 2048, 64, 80


def piecy_flops(pieces, rows, d, s, ell):
    """Flops of the method: per piece the randomised SVD, the projection X V and the lift Y V^T."""
    return pieces * (svd_flops(rows, d, s, ell) + 2.0 * rows * d * ell * 2)


def run_piecy(env, args):
    import numpy as np

    torch, B = env.torch, env.B
    from paper_1502_04265_gb300 import synth

    P, rows, d, ell, s = PIECY_PIECES, PIECY_ROWS, PIECY_D, PIECY_ELL, PIECY_S
    n = P * rows
    Q = synth.orthonormal_basis(d, 64, env.rank)
    Xg = torch.empty((n, d), dtype=torch.float32, device=env.dev)
    for q in range(P):
        Xq, _ = synth.subspace_mixture_chunk(Q, q * rows, rows, 500, env.rank)
        Xg[q * rows:(q + 1) * rows].copy_(torch.from_numpy(Xq))
    Om = torch.from_numpy(np.stack([synth.gaussian_sketch(d, s, seed=1000 * env.rank + q) for q in range(P)])).to(env.dev)
    L = torch.empty_like(Xg)
    ctx = env.ctx

    def step(i):
        B.kmeans_piecy_lift(Xg, rows, Om, ell, X_lift=L, ctx=ctx)

    R = env.timed(step, args.steps, args.warmup, clocks=True)
    ms, prof = R["ms"], R["prof"]
    F = piecy_flops(P, rows, d, s, ell)
    value = env.ranks.whole_job(F, ms) / 1e9
    peaks = env.peaks
    tf = unit_peak(peaks, "f32", True, R["total_s"])
    note3 = "3xTF32: max(probed kind::tf32, measured BF16 x nominal TF32/BF16 ratio) / 3"
    rooflines = {
        "project": roofline(peaks, "project", kernel_avg_s(prof, "project"), rows * d * 4 + rows * ell * 4 + d * ell * 4,
                            2.0 * rows * d * ell, tf, R["total_s"], note=note3),
        "lift": roofline(peaks, "lift", kernel_avg_s(prof, "lift"), rows * d * 4 + rows * ell * 4 + d * ell * 4,
                         2.0 * rows * d * ell, tf, R["total_s"], note=note3),
        **svd_rooflines(peaks, prof, rows, d, s, R["total_s"])}
    rooflines = {k_: v for k_, v in rooflines.items() if k_ in prof or k_ in ("project", "lift")}
    roof = max(rooflines.values(), key=lambda r: r["kernel_ms"])
    # the intrinsic dimension the pieces add: the rank of the first two pieces' lifted rows
    sub = L[: 2 * rows: 64].double().cpu().numpy()
    sv = np.linalg.svd(sub, compute_uv=False)
    quality = {"rank_first_two_pieces": int((sv > 1e-4 * sv[0]).sum()), "expected": 2 * ell}

    cpu = None
    if env.rank == 0 and env.world == 1 and not args.no_cpu_baseline:
        cpu = oracle_piecy_rate(Xg[:rows].cpu().numpy(), Om[0].cpu().numpy(), ell, args.cpu_seconds)

    e2e = None
    if not args.no_e2e:
        hb = B.HostBlock((n, d))
        hb.tensor.copy_(Xg.cpu())
        Xd = torch.empty_like(Xg)
        xn = torch.empty(n, dtype=torch.float32, device=env.dev)
        Lh = torch.empty((n, d), dtype=torch.float32).pin_memory()

        def e2e_step(i):
            B.kmeans_ingest(hb.tensor, X_dev=Xd, xnorm=xn, quantize=False, device=env.dev, ctx=ctx)
            B.kmeans_piecy_lift(Xd, rows, Om, ell, X_lift=L, ctx=ctx)
            Lh.copy_(L, non_blocking=True)

        E = env.timed(e2e_step, args.e2e_steps or 3, 3, profile=False)
        e2e = {"value": env.ranks.whole_job(F, E["ms"]) / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(n * d * 4),
               "d2h_bytes_per_step": int(n * d * 4), "ms_per_step": E["ms"],
               "note": "every step: the pieces read from a mapped host block (kmeans_ingest), the per-piece bases "
                       "and lifts, and D2H of the lifted points"}
        del hb

    line = base_line(env, "piecy", value, ms, args.steps, args.warmup, "f32", {
        "workload": f"{P} pieces of {rows} rows of the rank-64-subspace workload (d={d}, 500-component mixture in a "
                    f"random 64-dim subspace + N(0, 0.1^2) noise, seed = rank), each replaced by its projection onto "
                    f"its own top l={ell} basis (randomised SVD, s={s}, one Gaussian Omega per piece), d-dim lift",
        "l2": f"inputs larger than L2 (X is {n * d * 4 / 1e9:.1f} GB)",
        "parallelism": "replicas" if env.world > 1 else "single GPU"})
    line.update({"roofline": roof, "rooflines": rooflines, "quality": quality, "cpu_baseline": cpu, "e2e": e2e,
                 "gpu_launches": R["launches"], "clocks": R["clocks"], "kernels_ms": kernels_ms(prof)})
    return line


def oracle_piecy_rate(A, Om, ell, cpu_seconds):
    """The FP64 oracle (oracle/piecy.py: numpy QR and SVD as library steps) on row samples of one
    piece, repeated for about cpu_seconds."""
    import numpy as np

    from oracle import piecy as OP

    rows = 8192
    s = Om.shape[1]
    t0, reps = time.perf_counter(), 0
    while True:
        OP.lift_pieces(A[:rows], rows, [Om], ell)
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= cpu_seconds:
            break
    F = reps * piecy_flops(1, rows, A.shape[1], s, ell)
    return {"value": F / dt / 1e9, "unit": UNIT, "cores": os.cpu_count() or 1, "kind": "oracle",
            "sample": f"{reps} x one piece of {rows} rows x {A.shape[1]} (basis + lift, FP64 numpy with its "
                      f"threaded BLAS / LAPACK), {dt:.1f} s"}


# ---------------------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The FP64 CPU oracle timed on the host cores, on bounded samples of the same workload."""
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_1502_04265_gb300 import synth

    oracle.build()
    cores = oracle.set_threads(os.cpu_count() or 1)
    budget = min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup))
    wl = args.workload
    if wl == "bico":
        import torch as _t

        refs, P, f, X, w = bico_inputs(0, n=65536)
        N, S, Q = (a.numpy() for a in bico_snapshot_torch(_t, P, f, BICO_M, "cpu"))
        T = float(np.quantile(Q - (S * S).sum(1) / N, 0.8))
        vals, dts = [], []
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            r = oracle_bico_rate(X, w, refs, N, S, Q, T, budget)
            if i >= args.warmup:
                vals.append(r["value"])
                dts.append(time.perf_counter() - t0)
        val, sample, cores = statistics.median(vals), r["sample"], r["cores"]
    elif wl == "piecy":
        Qb = synth.orthonormal_basis(PIECY_D, 64, 0)
        A, _ = synth.subspace_mixture_chunk(Qb, 0, 8192, 500, 0)
        Om = synth.gaussian_sketch(PIECY_D, PIECY_S, seed=0)
        vals, dts = [], []
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            r = oracle_piecy_rate(A, Om, PIECY_ELL, budget)
            if i >= args.warmup:
                vals.append(r["value"])
                dts.append(time.perf_counter() - t0)
        val, sample, cores = statistics.median(vals), r["sample"], r["cores"]
    elif wl == "svd":
        n, d, ell, s_ = svd_shape(args)
        A, _ = svd_piece(n, d, 0)
        Om = synth.gaussian_sketch(d, s_, seed=0)
        vals, dts = [], []
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            r = oracle_svd_rate(A, Om, ell, budget)
            if i >= args.warmup:
                vals.append(r["value"])
                dts.append(time.perf_counter() - t0)
        val, sample, cores = statistics.median(vals), r["sample"], r["cores"]
    elif wl in ("small", "batch"):
        if wl == "small":
            X = mixture(10_000, 64, 10, 0)
            runs = [(X, 10, synth.seed_uniforms(10, 0))]
            desc = "the whole run (k-means++ + 20 Lloyd iterations) per step"
        else:
            shapes, jobs = batch_jobs(args.problems, 0)
            runs = []
            for s in shapes[:8]:
                X = _batch_problem((s["n"], s["d"], s["k"], s["seed"]))
                runs.append((X, s["k"], synth.seed_uniforms(s["k"], seed=s["seed"] * 4)))
            desc = "whole runs of the first problems (one seed each), in list order, per step"
        vals, dts = [], []
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            r = oracle_lloyd_rate(runs * 1000, 20, budget)
            if i >= args.warmup:
                vals.append(r["value"])
                dts.append(time.perf_counter() - t0)
        val = statistics.median(vals)
        sample = desc + "; " + r["sample"]
    else:
        if wl in ("highdim", "swn"):
            X, _, n, d, k = workload_data(args, 0)
            u = synth.seed_uniforms(k, 0)
            C = X[(u * n).astype(np.int64) % n]
        elif wl == "stream":
            Q = synth.orthonormal_basis(2048, 64, 0)
            Xc, _ = synth.subspace_mixture_chunk(Q, 0, 16384, 500, 0)
            X = oracle.project(Xc, Q).astype(np.float32)
            u = synth.seed_uniforms(1000, 0)
            C = X[(u * X.shape[0]).astype(np.int64) % X.shape[0]]
        else:
            X = mixture(65536, 256, 16384, 0)
            u = synth.seed_uniforms(16384, 0)
            C = X[(u * X.shape[0]).astype(np.int64) % X.shape[0]]
        vals, dts = [], []
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            r = oracle_assign_update_rate(X, C, budget)
            if i >= args.warmup:
                vals.append(r["value"])
                dts.append(time.perf_counter() - t0)
        val = statistics.median(vals)
        sample = r["sample"]
    ms = 1e3 * statistics.mean(dts)
    line = {"impl": "reference", "metric": METRICS[wl], "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{wl}: the FP64 oracle on a bounded sample per step ({sample})"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- main
def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    # the seeded generators of the large workloads run in spawned processes, started before CUDA
    pool, shapes = None, None
    if args.workload == "stream":
        n, d, r, chunk = 2_000_000, 2048, 64, 65536
        jobs = [(d, r, rank, r0, min(n, r0 + chunk) - r0, 500) for r0 in range(0, n, chunk)]
        pool = gen_pool(jobs, _stream_chunk)
    elif args.workload == "batch":
        shapes = batch_jobs(args.problems, rank)
        pool = gen_pool(shapes[1], _batch_problem)
    env = Env(args)
    env.pool, env.batch_shapes = pool, shapes
    if args.workload in ("highdim", "swn"):
        line = run_highdim(env, args)
    elif args.workload == "small":
        line = run_small(env, args)
    elif args.workload == "stream":
        line = run_stream((env, args))
    elif args.workload == "batch":
        line = run_batch((env, args))
    elif args.workload == "svd":
        line = run_svd(env, args)
    elif args.workload == "bico":
        line = run_bico(env, args)
    elif args.workload == "piecy":
        line = run_piecy(env, args)
    else:
        line = run_learned(env, args)
    if env.rank == 0:
        print(json.dumps(line), flush=True)
    env.ranks.close()


if __name__ == "__main__":
    main()
