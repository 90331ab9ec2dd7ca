#!/usr/bin/env python3
"""Throughput of the IB-LBM step on one GB300: million lattice updates per
second (MLUPS) of the full step -- the 10-iteration distribution-function
correction (arXiv 1803.09380, Eqs. 22-29) plus the fused BGK collide + AA
stream -- on the 4096 x 4096 cylindrical Couette lattice (radii 0.156 N and
0.39 N, 4015 + 10037 markers, tau = 0.8, inner wall speed 0.01), FP32.

One benchmark step is one time step of the method.  The lattice (604 MB in
FP32) is larger than the 129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (under torchrun) every rank runs its own independent lattice
(replicas: the method has no cross-lattice exchange), timing is the max over
ranks and the value is the aggregate.  --impl reference times the FP64 CPU
oracle on the host cores instead (a bounded sample per step).
"""
from __future__ import annotations

import argparse
import json
import os

# 32 hardware work queues instead of CUDA's default 8, before any CUDA
# context exists: the serving section keeps dozens of cases' streams busy.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS (D2Q9+IB correction) vs HBM roofline; batched solves/s, p50/p99 latency"
BYTES_PER_POP = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}
DTYPE = {"fp64": "f64", "fp32": "f32", "fp16": "f16-storage/f32", "bf16": "bf16-storage/f32"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=500)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=4096)
    p.add_argument("--prec", choices=list(BYTES_PER_POP), default="fp32")
    p.add_argument("--n-corr", type=int, default=10)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--cpu-budget", type=float, default=12.0,
                   help="seconds of oracle work for each cpu_baseline sample (one thread, all cores)")
    p.add_argument("--cpu-sample-set", action="store_true",
                   help="also time the oracle on the 64^2 ring case in full (5000 steps), the 1024^2 "
                        "and 4096^2 Couette lattices and the 1600x800 cylinder for 100 steps each, "
                        "one thread and all cores (minutes of host time)")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--ib-ctas", type=int, default=0,
                   help="CTAs of the correction kernel (0: the library's choice)")
    p.add_argument("--no-autotune", action="store_true",
                   help="keep the library's default correction grid instead of timing candidates")
    p.add_argument("--ib-threads", type=int, default=0,
                   help="threads per correction-kernel CTA (0: the library's choice)")
    p.add_argument("--ib-phases", type=int, choices=[-1, 0, 1, 2], default=-1,
                   help="correction loop as one persistent kernel (0), phase kernels (1), or "
                        "persistent kernels around a Jacobi cluster (2); -1: the library's default")
    p.add_argument("--serve-requests", type=int, default=512)
    p.add_argument("--serve-steps", type=int, default=500)
    p.add_argument("--serve-prec", choices=list(BYTES_PER_POP), default="fp32")
    p.add_argument("--serve-rate", type=float, default=2000.0, help="request arrivals per second")
    p.add_argument("--serve-active", type=int, default=128, help="cases resident at once")
    return p.parse_args()


def workload_config(args, case):
    return {
        "workload": f"cylindrical Couette {case.nx}x{case.ny}, D2Q9 BGK tau={case.tau}, "
                    f"radii {case.meta['r1']:.3f}/{case.meta['r2']:.3f}, "
                    f"{case.n_markers} markers, {args.n_corr} correction iterations, {args.prec}",
        "nx": case.nx, "ny": case.ny, "markers": case.n_markers, "n_corr": args.n_corr,
        "precision": args.prec,
        "l2": "inputs larger than L2 (populations %.0f MB > 129 MB), no flush"
              % (9 * case.nx * case.ny * BYTES_PER_POP[args.prec] / 1e6),
    }


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9 or parts[0] != str(self.idx):
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- oracle timing
def host_info():
    """Host cores and CPU model of the machine the oracle runs on."""
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu model")):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for ln in out.splitlines():
                if ln.startswith("Model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return {"nproc": os.cpu_count() or 1, "cpu_model": model or "unknown"}


def oracle_lattice(case, threaded):
    import oracle
    L = oracle.Lattice(case.nx, case.ny, case.tau, rho0=case.rho0, bc=case.bc, wall_u=case.wall_u,
                       inlet_u=case.inlet_u, n_corr=case.n_corr, mrt=case.mrt, threaded=threaded)
    for b in case.bodies:
        L.add_body(b.xy, b.ds, **b.as_kwargs())
    return L


def time_oracle(case, steps: int, threaded: bool) -> float:
    L = oracle_lattice(case, threaded)
    t = time.perf_counter()
    L.step(steps)
    dt = time.perf_counter() - t
    L.close()
    return dt


def oracle_threads(threaded: bool) -> int:
    import oracle
    return oracle.set_threads(0) if threaded else 1


def oracle_sample(budget_s: float, n_max: int, n_corr: int, threaded: bool):
    """Pick the largest Couette size (<= n_max, halving) whose oracle step
    fits the budget, from a calibration on 128^2; returns (n, steps)."""
    from paper_1803_09380_gb300 import workloads as wl
    per_node = time_oracle(wl.couette(128, n_corr=n_corr), 2, threaded) / (2 * 128 * 128)
    n = n_max
    while n > 64 and per_node * n * n > budget_s:
        n //= 2
    steps = max(1, int(budget_s / (per_node * n * n)))
    return n, min(steps, 1000)


def cpu_baseline(args):
    """The oracle as it stands on a bounded sample of the workload (the same
    geometry scaled down until a step fits the budget): all host cores (the
    -fopenmp build; the reported value) and one thread."""
    import oracle
    from paper_1803_09380_gb300 import workloads as wl
    info = host_info()
    runs = {}
    for threaded in ([False, True] if oracle.threaded_available() else [False]):
        n, steps = oracle_sample(args.cpu_budget, args.n, args.n_corr, threaded)
        dt = time_oracle(wl.couette(n, n_corr=args.n_corr), steps, threaded)
        runs[threaded] = {"value": n * n * steps / dt / 1e6, "cores": oracle_threads(threaded),
                          "sample": f"Couette {n}x{n} (same geometry scaled), {steps} step(s), {dt:.1f} s"}
    best = runs.get(True, runs[False])
    out = {"value": best["value"], "unit": "MLUPS", "cores": best["cores"], "kind": "oracle",
           "sample": f"FP64 C oracle, {best['cores']} thread(s), {best['sample']}, "
                     f"{args.n_corr} correction iterations",
           "single_thread": {"value": runs[False]["value"], "sample": runs[False]["sample"]}}
    out.update(info)
    if args.cpu_sample_set:
        out["sample_set"] = cpu_sample_set(args)
    return out


def cpu_sample_set(args):
    """The oracle, one thread and all cores, on a fixed sample set: the
    64^2 ring case in full, the 1024^2 and 4096^2 Couette lattices and the
    1600 x 800 cylinder channel for 100 steps each."""
    import oracle
    from paper_1803_09380_gb300 import workloads as wl
    cases = [("ring 64x64 (radii 10, 25), 5000 steps", wl.couette_64(), 5000),
             ("Couette 1024x1024, 100 steps", wl.couette(1024, n_corr=args.n_corr), 100),
             ("Couette 4096x4096, 100 steps", wl.couette(4096, n_corr=args.n_corr), 100),
             ("cylinder 1600x800 (D 40, 126 markers, Re 20), 100 steps",
              wl.cylinder(nx=1600, ny=800, diameter=40.0, center=(400.0, 400.0), u_in=0.05, re=20.0,
                          markers=126), 100)]
    out = []
    for name, case, steps in cases:
        rec = {"case": name}
        for threaded in ([False, True] if oracle.threaded_available() else [False]):
            dt = time_oracle(case, steps, threaded)
            key = f"mlups_{oracle_threads(threaded)}_threads" if threaded else "mlups_1_thread"
            rec[key] = case.nx * case.ny * steps / dt / 1e6
        out.append(rec)
    return out


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The oracle as it stands, timed like our arm: W untimed steps, then K
    timed steps, each one time step of the workload's geometry scaled down
    so that the whole run ends within minutes, on all host cores."""
    if rank != 0:
        return
    import oracle
    from paper_1803_09380_gb300 import workloads as wl
    case = wl.couette(args.n, n_corr=args.n_corr)
    threaded = oracle.threaded_available()
    total = args.steps + args.warmup
    n, _ = oracle_sample(150.0 / max(total, 1), args.n, args.n_corr, threaded)
    L = oracle_lattice(wl.couette(n, n_corr=args.n_corr), threaded)
    L.step(args.warmup)
    t = time.perf_counter()
    L.step(args.steps)
    dt = time.perf_counter() - t
    value = n * n * args.steps / dt / 1e6
    cores = oracle_threads(threaded)
    sample = (f"FP64 C oracle, {cores} thread(s); each step one time step of the Couette lattice "
              f"scaled to {n}x{n} (same geometry, {args.n_corr} correction iterations)")
    cfg = workload_config(args, case)
    cfg["timed_sample"] = f"{n}x{n} lattice, FP64 oracle"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": dict({"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                                  "sample": sample}, **host_info()),
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
# DRAM bytes (read + write) per collide+stream launch from one ncu capture,
# the mean of the two AA step kinds, with the sha256 prefix of the kernel
# sources the capture ran; the figure is reported only while the sources
# still hash to that value.
TRAFFIC = {
    ("fp32", 4096): (1141.1e6, "3e99c95b0c6971f9"),
    ("fp16", 4096): (541.5e6, "3e99c95b0c6971f9"),
    ("fp64", 4096): (2313.4e6, "3e99c95b0c6971f9"),
}
KERNEL_SOURCES = ("ibm_k1.cuh", "ibm_lbm.cu", "ibm_device.cuh")


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1803_09380_gb300", "csrc")
    for name in KERNEL_SOURCES:
        with open(os.path.join(here, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(prec: str, n: int):
    t = TRAFFIC.get((prec, n))
    if t is None or kernel_source_hash() != t[1]:
        return None, None
    return t[0], (f"ncu dram__bytes_read.sum + dram__bytes_write.sum of k_collide_stream, "
                  f"mean of both step kinds, kernel sources sha256 {t[1]}")


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over all ranks: a replica job takes as long as its
    slowest rank.  dist is torch.distributed (or None for one rank)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(nodes: int, steps: int, world: int, ms: float) -> float:
    """Lattice updates of all replicas over the job's time (weak scaling:
    every rank runs the same lattice)."""
    return nodes * steps * world / (ms * 1e-3) / 1e6


def run_ours(args, rank, world, local_rank, dist):
    import numpy as np
    import torch
    from paper_1803_09380_gb300 import ibm
    from paper_1803_09380_gb300 import workloads as wl

    torch.cuda.set_device(local_rank)
    case = wl.couette(args.n, n_corr=args.n_corr)
    N2 = case.nx * case.ny
    lat = ibm.Lattice.from_case(case, prec=args.prec, device=local_rank)
    tuned = None
    if args.ib_phases >= 0:
        ibm.ibm_set_option(lat.h, ibm.IBM_OPT_IB_PHASES, args.ib_phases)
    if args.ib_ctas:
        lat.set_ib_ctas(args.ib_ctas)
    elif not args.no_autotune:
        # the library's measured choice of the correction grid (its runs are
        # real steps and count as warm-up)
        sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
        tuned = lat.autotune_ib([sms * k // 8 for k in (2, 3, 4, 5, 6, 7, 8)], steps_each=50)
    if args.ib_threads:
        lat.set_ib_threads(args.ib_threads)
    stream = lat._stream
    flags = ibm.STEP_TIME_KERNELS | ibm.STEP_NO_MACRO

    lat.step(max(args.warmup, 3), flags)
    lat.sync()
    lat.kernel_times()
    l0, _ = lat.counters()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(local_rank) if rank == 0 else None
    barrier()
    if sampler:
        sampler.start()
        time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.step(args.steps, flags)
    e1.record(stream)
    barrier()
    clocks = sampler.stop() if sampler else None
    ms = e0.elapsed_time(e1)
    k1_ms, k1_n = lat.kernel_times()
    l1, _ = lat.counters()
    launches = l1 - l0
    ms = max_over_ranks(ms, dist, "cuda")
    value = whole_job_mlups(N2, args.steps, world, ms)

    peak, peak_src = measured_peak_hbm()
    bytes_per_update = 18 * BYTES_PER_POP[args.prec]
    _, _, _, band_nodes, band_segs = lat.sizes()
    main_nodes = N2 - 32 * band_segs           # nodes of the band-free row segments
    k1_avg_s = (k1_ms / max(k1_n, 1)) * 1e-3
    achieved = bytes_per_update * main_nodes / k1_avg_s / 1e9
    traffic, traffic_src = measured_traffic(args.prec, args.n)
    limiter = {"fp64": "FP64 arithmetic (ncu: FP64 pipe 84 % active in k_collide_stream)",
               "fp16": "instruction issue (ncu: issue slots busy in k_collide_stream)",
               "bf16": "instruction issue (ncu: issue slots busy in k_collide_stream)"}.get(args.prec)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_src,
                "kernel": "k_collide_stream (band-free row segments, both AA step kinds)",
                "peak_source": f"hbm_gbs of {peak_src} (MEASURED_PEAKS.json)",
                "bytes_per_launch": bytes_per_update * main_nodes,
                "avg_launch_us": k1_avg_s * 1e6, "launches_timed": k1_n,
                "band_nodes": band_nodes, "band_segment_nodes": 32 * band_segs,
                "step_frac": (bytes_per_update * N2 * args.steps / (ms * 1e-3) / 1e9) / peak}
    if limiter:
        roofline["limited_by"] = limiter
    lat.close()
    roofline["alone"] = k1_alone(args, local_rank, peak, bytes_per_update)

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, case, local_rank, dist, world)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args)

    serving = None
    if rank == 0 and not args.no_serving:
        serving = run_serving(args, local_rank)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": DTYPE[args.prec], "data": "synthetic",
                "config": workload_config(args, case),
                "correction_ctas": tuned[0] if tuned else (args.ib_ctas or "library default"),
                "timed_path": "ibm_step with IBM_STEP_TIME_KERNELS | IBM_STEP_NO_MACRO: every step "
                              "corrects, collides and streams; rho and u are not written out on the "
                              "last step of the call (the optional output fields)",
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": e2e, "gpu_launches": launches, "clocks": clocks, "serving": serving}
        print(json.dumps(line), flush=True)


def k1_alone(args, local_rank, peak, bytes_per_update, steps=200):
    """The same collide+stream kernel with nothing beside it: a marker-free
    periodic lattice of the benchmark's size and precision (every node in
    one launch per step), kernel durations from CUDA events."""
    from paper_1803_09380_gb300 import ibm
    lat = ibm.Lattice(args.n, args.n, 0.8, 1.0, args.prec, device=local_rank)
    try:
        flags = ibm.STEP_TIME_KERNELS | ibm.STEP_NO_MACRO
        lat.step(20, flags)
        lat.sync()
        lat.kernel_times()
        lat.step(steps, flags)
        lat.sync()
        k_ms, k_n = lat.kernel_times()
    finally:
        lat.close()
    us = 1e3 * k_ms / max(k_n, 1)
    achieved = bytes_per_update * args.n * args.n / (us * 1e-6) / 1e9
    return {"avg_launch_us": us, "achieved": achieved, "frac": achieved / peak, "launches_timed": k_n,
            "what": f"k_collide_stream alone: marker-free {args.n}x{args.n} lattice, every node, {steps} steps"}


def run_serving(args, local_rank):
    """Continuous batching on the serving stream (512 requests with seeded
    Poisson arrivals; a uniform mix of Couette with N log-uniform in 64-2048,
    fixed cylinders on 2ny x ny lattices with ny in 200-800 and Re 10-100,
    and one or two settling disks of D 10-30 in a 200 x 600 box),
    `serve_steps` time steps per request, arrivals fast enough to keep the
    server saturated.  Two one-at-a-time baselines run the same requests at
    the same precision, so every solve has the same result and accuracy:
    each case as its own ibm.Lattice (the library's default correction grid,
    graph replays of 8-step blocks), one after another; and the same server
    with one slot."""
    from paper_1803_09380_gb300 import ibm
    from paper_1803_09380_gb300 import workloads as wl
    stream = wl.serving_stream(n_requests=args.serve_requests, seed=1803, rate_hz=args.serve_rate,
                               steps=args.serve_steps)
    prec = args.serve_prec
    out = {"requests": len(stream), "steps_per_request": args.serve_steps, "precision": prec,
           "mix": "Couette N 64-2048 log-uniform, cylinder 2ny x ny (ny 200-800, Re 10-100), "
                  f"1-2 settling disks D 10-30 in 200x600; Poisson arrivals at {args.serve_rate:g}/s, "
                  "seed 1803",
           "solve": f"{args.serve_steps} time steps of the case, residual history read back"}

    def serve(max_active, paced, batched=False, tune=False, prec=prec, preset=None):
        with ibm.Server(device=local_rank, max_active=max_active, steps_per_launch=16,
                        batched=batched, **(preset or {})) as srv:
            tuned = None
            if tune:
                # the autotuner times tile size, markers per correction CTA and
                # task order on the stream's first 24 requests (64 steps each)
                t, m, o, _ = srv.autotune([c for _, c, _ in stream[:24]], 64, prec=prec)
                tuned = {"tile_nodes": t, "markers_per_cta": m, "corr_first": o}
            t0 = time.perf_counter()
            k = 0
            while k < len(stream):
                if paced:
                    while k < len(stream) and stream[k][0] > time.perf_counter() - t0:
                        srv.progress()
                srv.submit(stream[k][1], stream[k][2], prec=prec, outputs=ibm.OUT_RESIDUAL)
                k += 1
                if not paced:
                    srv.wait()
            srv.wait()
            wall = time.perf_counter() - t0
            return srv.stats(), wall, tuned

    def lattice_one_at_a_time():
        t0 = time.perf_counter()
        for _, case, steps in stream:
            with ibm.Lattice.from_case(case, prec=prec, device=local_rank) as lat:
                lat.step(steps)
                lat.resid
        return time.perf_counter() - t0

    st, wall, tuned = serve(args.serve_active, True, batched=True, tune=True)
    out.update({"mode": "batched: one persistent kernel per round over a task queue of all resident "
                        "cases' correction tasks and collide+stream tiles",
                "solves_per_s": st["solves_per_s"], "p50_ms": st["p50_ms"], "p95_ms": st["p95_ms"],
                "p99_ms": st["p99_ms"], "mlups": st["mlups"], "failed": st["failed"],
                "max_active": args.serve_active, "wall_s": wall, "autotuned": tuned,
                "host_admit_s": st["host_admit_s"], "host_launch_s": st["host_launch_s"]})
    if prec == "fp32":
        # the same stream with FP16 deviation storage, batched, with the
        # parameters the autotuner chose for FP32
        preset = {"tile_nodes": tuned["tile_nodes"], "corr_first": tuned["corr_first"],
                  "ib_markers_per_cta": tuned["markers_per_cta"]}
        sth, wallh, _ = serve(args.serve_active, True, batched=True, prec="fp16", preset=preset)
        out["fp16_storage"] = {"solves_per_s": sth["solves_per_s"], "p50_ms": sth["p50_ms"],
                               "p99_ms": sth["p99_ms"], "failed": sth["failed"], "wall_s": wallh,
                               "vs_fp32_batched": sth["solves_per_s"] / st["solves_per_s"],
                               "what": "batched server, FP16 deviation storage, the FP32 run's tuned parameters"}
    # per-case streams peak at about 64 resident cases (more streams than
    # that cost more than they overlap)
    active_s = min(args.serve_active, 64)
    stp, wallp, _ = serve(active_s, True)
    out["per_case_streams"] = {"solves_per_s": stp["solves_per_s"], "p50_ms": stp["p50_ms"],
                               "p99_ms": stp["p99_ms"], "failed": stp["failed"], "wall_s": wallp,
                               "max_active": active_s,
                               "what": "each resident case stepped by its own graph launches on its own stream"}
    wall_l = lattice_one_at_a_time()
    out["solves_per_s_one_at_a_time"] = len(stream) / wall_l
    out["speedup_vs_one_at_a_time"] = out["solves_per_s"] / out["solves_per_s_one_at_a_time"]
    out["one_at_a_time"] = "each case as its own ibm.Lattice, one after another (the best single-case path)"
    _, wall1, _ = serve(1, False)
    out["solves_per_s_server_one_slot"] = len(stream) / wall1
    out["speedup_vs_server_one_slot"] = out["solves_per_s"] / out["solves_per_s_server_one_slot"]
    return out


def run_e2e(args, case, local_rank, dist, world):
    """The whole job through the public API: create the lattice, upload the
    markers from pinned host memory, run the timed number of steps, read the
    corrected density and velocity back into pinned host memory."""
    import numpy as np
    import torch
    from paper_1803_09380_gb300 import ibm

    nx, ny = case.nx, case.ny
    pinned = []
    for b in case.bodies:
        t = torch.empty((b.xy.shape[0], 3), dtype=torch.float64, pin_memory=True)
        t[:, :2] = torch.from_numpy(b.xy)
        t[:, 2] = torch.from_numpy(b.ds)
        pinned.append(t)
    outs = [torch.empty((ny, nx), dtype=torch.float64, pin_memory=True) for _ in range(3)]
    h2d = sum(t.numel() * 8 for t in pinned)
    d2h = sum(t.numel() * 8 for t in outs)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat = ibm.Lattice(nx, ny, case.tau, case.rho0, args.prec, case.bc, case.wall_u, case.inlet_u,
                      case.n_corr, device=local_rank)
    for b, t in zip(case.bodies, pinned):
        a = t.numpy()
        lat.add_markers(np.ascontiguousarray(a[:, :2]), np.ascontiguousarray(a[:, 2]), **b.as_kwargs())
    lat.step(args.steps)
    for fld, o in zip((ibm.FIELD_RHO, ibm.FIELD_UX, ibm.FIELD_UY), outs):
        lat.read(fld, out=o.numpy())
    dt = time.perf_counter() - t0
    lat.close()
    dt = max_over_ranks(dt, dist, "cuda")
    return {"value": whole_job_mlups(nx * ny, args.steps, world, dt * 1e3), "unit": "MLUPS",
            "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
            "wall_s": dt,
            "what": "create lattice + upload markers (pinned) + steps + read rho, ux, uy (pinned)"}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
        dist = tdist
    try:
        run_ours(args, rank, world, local_rank, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
