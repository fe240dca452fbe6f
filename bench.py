#!/usr/bin/env python
"""Benchmark of the phi+mu time step (arXiv:1506.01684, Algorithm 1) on GB300.

Workload: the single large domain, 256x256x1024 cells, FP32 stencil arithmetic and
storage, the symmetric parameter set, 64 Voronoi grains in the bottom 8 planes with
liquid above, moving-window trigger at z = 512 (synthetic inputs; the paper's Ag-Al-Cu
data is not available).  A "step" is one full explicit step over the domain: phi-sweep,
mu-sweep, FP64 reductions, window check.  The fields (1.6 GB FP32) are larger than L2,
so no cache flush is needed between steps.

Printed: one JSON line with MLUP/s (value), the FP64 GPU path on the same workload, the
FP32-vs-FP64 error, the dominant kernel's roofline, an end-to-end figure through host
buffers, the oracle's CPU baseline, clocks and launch counts.

The timed steps start from the configuration's own state: 2000 untimed steps (--pre-steps) take the
Voronoi start's sharp fronts to the diffuse, growing interface of the single-large-domain run, and
the line reports that state (interface height, fraction of cells on general planes).  Two timed
regions of K steps each follow the warm-up: A, the steps as pf_step runs them (replayed
from the captured CUDA graph), gives `value` and `ms_per_step`; B, the next K steps with the
library's per-kernel CUDA-event timers (every kernel launched directly between its two events),
gives the per-kernel durations, their shares and the roofline of the dominant kernel, and its own
`ms_per_step_kernel_timers`.  The roofline's algorithmic bytes are the kernels' own tally of the
last step (pf_step_bytes): 16 B a cell on pure-liquid planes, 88 B on general planes.  The general
planes' sweeps are bound by the FP32 units, so a second roofline (`roofline_general`) sets their
FP32 operation rate against the FP32 peak derived from the SM count and the sampled clock.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--pre-steps P] [--impl gb300|reference]

With N > 1 (torchrun, one process per GPU) every rank runs its own replica of the
workload (the path has no exchange step on one domain per GPU: replicas only, weak
scaling); value = all ranks' cell updates / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX, NY, NZ = 256, 256, 1024
GRAINS = 64
TRIGGER = 512.0
SEED = 0
PRE_STEPS = 2000  # the single-large-domain configuration runs 2000 steps
WORKLOAD = "single domain 256x256x1024, 64 grains, window trigger z=512, symmetric parameter set"
METRIC = "phi+mu step MLUP/s (FP32 stencil; FP64 and compensated FP32 GPU paths and their errors reported beside it)"

# Algorithmic bytes per kernel and launch come from the library (pf_step_bytes): the mu-sweep
# reads phi^n, phi^{n+1} (16 B each) and mu^n (8 B) and writes mu^{n+1} (8 B); the phi-sweep
# reads phi^n and mu^n and writes phi^{n+1}.  The fused step's general planes move 48 B a cell
# (phi^n, mu^n in, phi^{n+1}, mu^{n+1} out); its pure-liquid planes (the lean kernel) 16 B (mu^n
# in, mu^{n+1} out; phi^{n+1} = e_l is stored only where the destination does not hold it
# already) -- tallied by the kernels themselves.
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) over the kernel's algorithmic
# bytes, from an ncu capture of the kernel as it is now on 256x256x512 (the same workload at half the
# depth, mu larger than L2; the capture and its command are in profiles/lean_step_traffic_fp32_256x256x512.md);
# traffic of a full launch = this ratio x the launch's algorithmic bytes (traffic grows with the lean
# cells).  Remove an entry when its kernel changes.
TRAFFIC_RATIO = {"lean_step": 0.93}

# kernels behind one per-kernel timer record of the library (pf_profile_read)
KERNELS_PER_RECORD = {"general_sweeps": 2}


# The general planes' two sweeps (the interface cells) are bound by the FP32 units, not HBM: per general
# cell, the FP32 operations (FADD, FMUL = 1, FFMA = 2) and the thread instructions of both sweeps, halo
# and prologue work included, from the SASS counters of an ncu capture of the kernels as they are now
# (summed over general_phi_kernel and general_mu_kernel, divided by the general cells the launch
# processed; the capture and its command are in profiles/general_sweeps_flops_fp32_256x256x512.md).
# None: not measured for the current kernels.  Remove the entries when the kernels change.
GENERAL_FLOPS_PER_CELL = 728.0
GENERAL_INSTS_PER_CELL = 1354.0


def alu_roofline(k, general_cells, clk):
    """Roofline of the general planes' sweeps against the FP32 units: FP32 operations per second over
    SMs x 128 FP32 lanes x 2 (a fused multiply-add) x the median SM clock sampled in the timed region,
    and thread instructions per second over SMs x 4 schedulers x 32 lanes x that clock."""
    import torch
    if not k or general_cells <= 0:
        return None
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = (clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz") or 2070.0
    secs = k["ms_avg"] / 1e3
    peak = sms * 128 * 2 * mhz * 1e6 / 1e12
    out = {"bound": "alu", "kernel": "general_sweeps", "unit": "TFLOP/s", "peak": peak,
           "peak_kind": f"derived: {sms} SMs x 128 FP32 lanes x 2 (FMA) x {mhz:.0f} MHz (median sampled)",
           "general_cells_per_launch": general_cells, "general_gcells_per_s": general_cells / secs / 1e9,
           "achieved": None, "frac": None}
    if GENERAL_FLOPS_PER_CELL:
        a = GENERAL_FLOPS_PER_CELL * general_cells / secs / 1e12
        out.update(achieved=a, frac=a / peak, flops_per_cell=GENERAL_FLOPS_PER_CELL)
    if GENERAL_INSTS_PER_CELL:
        issue_peak = sms * 4 * 32 * mhz * 1e6
        out.update(insts_per_cell=GENERAL_INSTS_PER_CELL,
                   issue_frac=GENERAL_INSTS_PER_CELL * general_cells / secs / issue_peak)
    return out


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int, path: str | None = None):
        import tempfile
        self.device = device
        self.proc = None
        self.path = path or os.path.join(tempfile.gettempdir(), f"pf_clocks_{os.getpid()}_{device}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(ms: float, dist=None, device: str = "cpu") -> float:
    """The slowest rank's time (the timed region of every rank ends at the same barrier)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world: int, cells_per_rank: int, steps: int, ms_max: float) -> float:
    """Cell updates of all ranks (one replica of the workload each) / the slowest rank's time."""
    return world * cells_per_rank * steps / (ms_max / 1e3) / 1e6


def cpu_baseline(min_seconds: float = 10.0, max_steps: int = 40):
    """The FP64 C oracle as it stands, on this host's cores, on a bounded sample of the
    workload: the full 256x256 x-y extent, the bottom 16 planes (the 8 seeded planes with
    their interface and liquid above), the same grains and seed; steps repeated until
    min_seconds of CPU work (at least 2)."""
    import oracle
    from paper_1506_01684_gb300 import workloads as W

    nzs = 16
    p = W.symmetric_params(n_grains=GRAINS)
    st = oracle.State(p, NX, NY, nzs).init(SEED)
    st.step(1)  # first-touch of the oracle's buffers
    t0 = time.perf_counter()
    n = 0
    while n < 2 or (time.perf_counter() - t0 < min_seconds and n < max_steps):
        st.step(1)
        n += 1
    dt = time.perf_counter() - t0
    cells = NX * NY * nzs
    return {"value": cells * n / dt / 1e6, "unit": "MLUP/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{NX}x{NY}x{nzs} bottom slab of the workload (64 grains, seed 0), {n} FP64 steps, "
                      f"{dt:.1f} s",
            "cpu_model": _cpu_model(), "samples": oracle_samples()}


def _cpu_model():
    try:
        impl = part = None
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.lower()
                if key.startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
                if key.startswith("cpu implementer") and impl is None:
                    impl = line.split(":", 1)[1].strip()
                if key.startswith("cpu part") and part is None:
                    part = line.split(":", 1)[1].strip()
        if impl and part:  # Arm: the implementer and part numbers (0x41 / 0xd4f: Arm Neoverse V2)
            return f"Arm CPU implementer {impl}, part {part}"
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


# the oracle's two further samples: the small configuration (32x32x64, 12 grains, seed 0) and the
# paper's interface block at 128^3 (columnar grains below z = 64, liquid above; 2 relaxation steps)
ORACLE_SAMPLES = {"small_32x32x64": (32, 32, 64, 20), "interface_128x128x128": (128, 128, 128, 3)}


def _sample_state(name):
    import oracle
    from paper_1506_01684_gb300 import workloads as W
    nx, ny, nz, _ = ORACLE_SAMPLES[name]
    if name.startswith("small"):
        p = W.symmetric_params(n_grains=12)
        return p, (nx, ny, nz), None
    phi, mu = W.region_fields("interface", nx, ny, nz, seed=0)
    return W.symmetric_params(), (nx, ny, nz), (phi, mu)


def oracle_samples(reps: int = 3):
    """The FP64 oracle on the host cores on the small configuration and a 128^3 interface block:
    MLUP/s, the median of `reps` timed runs of a few steps each."""
    import oracle
    out = {}
    for name, (nx, ny, nz, steps) in ORACLE_SAMPLES.items():
        p, shape, fields = _sample_state(name)
        st = oracle.State(p, *shape)
        if fields is None:
            st.init(SEED)
        else:
            st.phi, st.mu = fields[0].copy(), fields[1].copy()
        st.step(2)
        rates = []
        for _ in range(reps):
            t0 = time.perf_counter()
            st.step(steps)
            rates.append(nx * ny * nz * steps / (time.perf_counter() - t0) / 1e6)
        out[name] = {"mlups": statistics.median(rates), "runs_mlups": rates, "steps_per_run": steps}
    return out


def gpu_on_oracle_samples(stream, steps: int = 200):
    """The FP32 GPU step (the library's variant choice) on the oracle's two further samples."""
    import torch

    from paper_1506_01684_gb300 import pf
    out = {}
    for name in ORACLE_SAMPLES:
        p, shape, fields = _sample_state(name)
        sim = pf.Simulation(*shape, p, "fp32", stream=stream)
        if fields is None:
            sim.init(SEED)
        else:
            sim.set_fields(*fields)
        sim.step(5)
        sim.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        out[name] = shape[0] * shape[1] * shape[2] * steps / (e0.elapsed_time(e1) / 1e3) / 1e6
        sim.close()
    return out


def gpu_on_cpu_sample(stream, steps: int = 200):
    """The GPU path (FP32, the library's variant choice) on the CPU baseline's sample: the same
    256x256x16 bottom slab, grains and seed, so the oracle's rate has a like-for-like GPU figure."""
    import torch

    from paper_1506_01684_gb300 import pf
    from paper_1506_01684_gb300 import workloads as W

    nzs = 16
    sim = pf.Simulation(NX, NY, nzs, W.symmetric_params(n_grains=GRAINS), "fp32", stream=stream)
    sim.init(SEED)
    sim.step(5)
    sim.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    sim.close()
    return NX * NY * nzs * steps / (ms / 1e3) / 1e6


def run_reference(args, rank):
    """The reference arm: the oracle on the host cores, each step one bounded sample."""
    if rank != 0:
        return
    import oracle
    from paper_1506_01684_gb300 import workloads as W

    nzs = 16
    p = W.symmetric_params(n_grains=GRAINS)
    st = oracle.State(p, NX, NY, nzs).init(SEED)
    for _ in range(args.warmup):
        st.step(1)
    t0 = time.perf_counter()
    st.step(args.steps)
    dt = time.perf_counter() - t0
    cells = NX * NY * nzs
    v = cells * args.steps / dt / 1e6
    sample = f"{NX}x{NY}x{nzs} bottom slab of the workload per step (64 grains, seed 0), FP64"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": v, "unit": "MLUP/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "MLUP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batched_study(args):
    """64 independent domains of uneven size (x, y in {32, 64, 96, 128}, z in {128, 256, 512}),
    each with its own pulling velocity and gradient, FP32: the autotuned batched launch (one
    persistent kernel per step, graph-replayed) against the same domains stepped one by one."""
    import torch

    from paper_1506_01684_gb300 import pf
    from paper_1506_01684_gb300 import workloads as W

    doms = W.batched_domains(64, seed=0)
    shapes = [(d["nx"], d["ny"], d["nz"]) for d in doms]
    params = [W.symmetric_params(G=d["G"], v=d["v"], n_grains=12) for d in doms]
    seeds = [d["seed"] for d in doms]
    cells = sum(a * b * c for a, b, c in shapes)
    stream = torch.cuda.Stream()
    b = pf.Batch(shapes, params, "fp32", stream=stream)
    b.init(seeds)
    zc, tune_ms = pf.pf_batch_autotune(b.h, 5)
    tuned = pf.pf_batch_config(b.h)
    b.step(args.warmup)
    b.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    b.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_batch = e0.elapsed_time(e1) / args.steps
    b.sync()
    # algorithmic bytes of a step (the kernels' own tally of the last step): the whole batched step
    # against the HBM roofline, and the design bound its bytes set
    sb = pf.pf_batch_step_bytes(b.h)
    step_bytes = sb["general_and_fused"] + sb["lean_step"]
    hbm, peak_kind = _peaks()
    achieved = step_bytes / (ms_batch / 1e3) / 1e9
    design_bound = hbm * 1e9 / (step_bytes / cells) / 1e6 if step_bytes else None
    b.close()
    # one by one: each domain its own pf_sim (fused kernel, graph replay), run back to back
    sims = []
    for shp, p, sd in zip(shapes, params, seeds):
        sim = pf.Simulation(*shp, p, "fp32", stream=stream, variant="fused")
        sim.init(sd)
        sim.step(args.warmup)
        sims.append(sim)
    torch.cuda.synchronize()
    e0.record(stream)
    for sim in sims:
        sim.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_single = e0.elapsed_time(e1) / args.steps
    for sim in sims:
        sim.close()
    line = {"metric": "batched phi+mu step MLUP/s, 64 uneven domains (FP32)", "unit": "MLUP/s",
            "value": cells / (ms_batch / 1e3) / 1e6, "one_by_one": cells / (ms_single / 1e3) / 1e6,
            "speedup_vs_one_by_one": ms_single / ms_batch, "ms_per_step": ms_batch,
            "ms_per_step_one_by_one": ms_single, "cells": cells, "domains": len(shapes),
            "autotuned_zchunk": zc, "autotuned_general_ctas_per_sm": tuned["general_ctas_per_sm"],
            "autotuned_lean_split": tuned["lean_split"], "autotuned_lean_tile": [32, tuned["lean_tile_rows"]],
            "autotune_ms_per_step": tune_ms, "steps": args.steps, "warmup": args.warmup,
            "roofline": {"bound": "hbm", "kernel": "whole batched step", "achieved": achieved, "peak": hbm,
                         "unit": "GB/s", "frac": achieved / hbm, "peak_kind": peak_kind,
                         "bytes_per_cell": step_bytes / cells,
                         "lean_share_of_bytes": sb["lean_step"] / step_bytes if step_bytes else None,
                         "what": "algorithmic bytes of one step (the kernels' tally) / the step's time"},
            "frac_of_design_bound": (cells / (ms_batch / 1e3) / 1e6) / design_bound if design_bound else None,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "64 domains, x,y in {32,64,96,128}, z in {128,256,512}, v in [5e-3,2e-2], "
                                   "G in [5e-4,2e-3], 12 grains each (numpy PCG64 seed 0)"}}
    print(json.dumps(line), flush=True)


def run_serving_study(args):
    """Poisson stream of solidification requests (sizes as the batched study plus a fraction at
    256x256x512, steps uniform in a range, random v, G and seed) served with continuous batching;
    the arrival rate puts the offered load at `load` x the measured batched capacity.  Reports
    p50/p99 latency (submission to result) and the aggregate MLUP/s."""
    import time as _t

    import numpy as np
    import torch

    from paper_1506_01684_gb300 import pf
    from paper_1506_01684_gb300 import workloads as W

    reqs = W.serving_requests(args.requests, seed=0, big_fraction=0.1,
                              steps_range=(args.min_steps, args.max_steps))
    work = np.array([r["nx"] * r["ny"] * r["nz"] * r["steps"] for r in reqs], dtype=float)
    # capacity: the batched launch on a sample of the request mix
    sample = reqs[: min(16, len(reqs))]
    b = pf.Batch([(r["nx"], r["ny"], r["nz"]) for r in sample],
                 [W.symmetric_params(G=r["G"], v=r["v"]) for r in sample], "fp32")
    b.init([r["seed"] for r in sample])
    b.step(4)
    b.sync()
    t0 = _t.perf_counter()
    b.step(20)
    b.sync()
    cap = sum(r["nx"] * r["ny"] * r["nz"] for r in sample) * 20 / (_t.perf_counter() - t0)  # cells/s
    b.close()
    mean_gap = work.mean() / (args.load * cap)
    arrivals = np.array([r["arrival"] for r in reqs]) * mean_gap
    srv = pf.pf_server_create(0, 0, args.chunk)
    tickets = {}
    lat = {}
    t_start = _t.perf_counter()
    nxt = 0
    while len(lat) < len(reqs):
        now = _t.perf_counter() - t_start
        while nxt < len(reqs) and arrivals[nxt] <= now:
            r = reqs[nxt]
            tickets[nxt] = pf.pf_submit(srv, r["nx"], r["ny"], r["nz"],
                                        pf.params_from_dict(W.symmetric_params(G=r["G"], v=r["v"]), pf.PF_FP32),
                                        r["seed"], r["steps"])
            nxt += 1
        for i in [i for i in tickets if i not in lat]:
            res = pf.pf_poll(srv, tickets[i])
            if res is not None:
                lat[i] = res[2]
        _t.sleep(0.0005)
    makespan = _t.perf_counter() - t_start
    st = pf.pf_server_stats(srv)
    pf.pf_server_destroy(srv)
    L = np.array([lat[i] for i in range(len(reqs))])
    line = {"metric": "served solidification requests: p50/p99 latency and aggregate MLUP/s (FP32)",
            "unit": "s", "p50_latency_s": float(np.percentile(L, 50)), "p99_latency_s": float(np.percentile(L, 99)),
            "mean_latency_s": float(L.mean()), "aggregate_mlups": float(work.sum() / makespan / 1e6),
            "busy_mlups": st["mlups"], "makespan_s": makespan, "requests": len(reqs),
            "offered_load": args.load, "capacity_mlups_estimate": cap / 1e6, "chunk_steps": args.chunk,
            "higher_is_better": False, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{len(reqs)} Poisson arrivals, sizes x,y in {{32,64,96,128}}, z in {{128,256,512}} "
                                   f"plus 10% at 256x256x512, steps U[{args.min_steps},{args.max_steps}], random v, G, "
                                   "seed (numpy PCG64 seed 1)"}}
    print(json.dumps(line), flush=True)


def run_split_study(args):
    """The block decomposition on one GPU (pf_split: y-slabs with ghost rows, Algorithm 1's exchanges
    and Algorithm 2's overlap) against the undivided domain stepped with the same two sweeps
    (PF_VARIANT_UNFUSED) and with the library's default step, FP32, 64 grains, from the 200-step
    state: MLUP/s by CUDA events over the timed steps, and whether the fields agree bit for bit."""
    import numpy as np
    import torch

    from paper_1506_01684_gb300 import pf
    from paper_1506_01684_gb300 import workloads as W

    nx, ny, nz = (int(x) for x in args.split_shape.split("x"))
    p = W.symmetric_params(n_grains=GRAINS, window_trigger_z=nz / 2)
    cells = nx * ny * nz
    pre, k = 200, max(args.steps, 10)

    def timed(obj):
        obj.step(pre + args.warmup)
        obj.sync()
        torch.cuda.synchronize()
        # the split runs on several streams of its own: wall clock between two full synchronisations
        t0 = time.perf_counter()
        obj.step(k)
        obj.sync()
        wall = time.perf_counter() - t0
        return cells * k / wall / 1e6

    res = {}
    whole = pf.Simulation(nx, ny, nz, p, "fp32", variant="unfused").init(SEED)
    res["undivided_unfused"] = {"mlups": timed(whole)}
    ref_phi, ref_mu = whole.fields()
    whole.close()
    auto = pf.Simulation(nx, ny, nz, p, "fp32").init(SEED)
    res["undivided_default"] = {"mlups": timed(auto)}
    auto.close()
    for n in (1, 2, 4, 8, 16):
        sp = pf.Split(nx, ny, nz, p, n, "fp32").init(SEED)
        m = timed(sp)
        phi, mu = sp.fields()
        res[f"split_{n}"] = {"mlups": m, "bitwise_equal_to_unfused": bool(np.array_equal(phi, ref_phi)
                                                                           and np.array_equal(mu, ref_mu))}
        sp.close()
    print(json.dumps({"metric": "block decomposition on one GPU: MLUP/s (FP32)",
                      "config": {"workload": f"{nx}x{ny}x{nz}, {GRAINS} grains, seed {SEED}, timed {k} steps "
                                             f"after {pre + args.warmup}, wall clock between synchronisations"},
                      "results": res, "data": "synthetic"}), flush=True)


def run_precision_study(args):
    """128x128x512 cells, 20000 steps by default: compensated FP32 vs plain FP32 vs FP64 on the GPU.
    First each GPU path's agreement with the CPU oracle on the small case (32x32x64, 200 steps);
    then, on the study case, the error of phase fractions and lamella counts against the FP64 run."""
    import time as _t

    import numpy as np
    import torch

    import oracle
    from paper_1506_01684_gb300 import analysis, pf
    from paper_1506_01684_gb300 import workloads as W

    small = {}
    p0 = W.symmetric_params()
    ref = oracle.State(p0, 32, 32, 64).init(0)
    ref.step(200)
    for prec in ("fp64", "fp32", "fp32c"):
        sim = pf.Simulation(32, 32, 64, p0, prec)
        sim.init(0)
        sim.step(200)
        phi, mu = sim.fields()
        small[prec] = {"max_abs_dphi": float(np.abs(phi - ref.phi).max()),
                       "max_rel_dmu": float(np.abs(mu - ref.mu).max() / max(np.abs(ref.mu).max(), 1e-8))}
        sim.close()
    nx, ny, nz = (int(x) for x in args.study_shape.split("x"))
    p = W.symmetric_params(n_grains=20)
    res = {}
    for prec in ("fp64", "fp32c", "fp32"):
        sim = pf.Simulation(nx, ny, nz, p, prec)
        sim.init(0)
        sol0 = sim.stats()["solute"]
        torch.cuda.synchronize()
        t0 = _t.perf_counter()
        sim.step(args.study_steps)
        sim.sync()
        dt = _t.perf_counter() - t0
        st = sim.stats()
        phi, mu = sim.fields()
        res[prec] = {"mlups": nx * ny * nz * args.study_steps / dt / 1e6, "seconds": dt,
                     "fractions": [float(x) for x in sim.fractions()], "h_int": st["h_int"],
                     "lamellae": analysis.lamella_count(phi, st["h_int"]),
                     "solute_drift": [float((st["solute"][c] - sol0[c]) / sol0[c]) for c in range(2)],
                     "_phi": phi, "_mu": mu}
        sim.close()
    base = res["fp64"]
    for prec in ("fp32c", "fp32"):
        r = res[prec]
        r["max_abs_dphi_vs_fp64"] = float(np.abs(r["_phi"] - base["_phi"]).max())
        r["max_rel_dmu_vs_fp64"] = float(np.abs(r["_mu"] - base["_mu"]).max() / max(np.abs(base["_mu"]).max(), 1e-8))
        r["max_abs_dfraction_vs_fp64"] = float(np.abs(np.array(r["fractions"]) - np.array(base["fractions"])).max())
        r["lamella_diff_vs_fp64"] = [a - b for a, b in zip(r["lamellae"], base["lamellae"])]
    for r in res.values():
        r.pop("_phi")
        r.pop("_mu")
    line = {"metric": "precision study: FP32 / compensated FP32 vs FP64 on the GPU", "config": {
        "workload": f"{nx}x{ny}x{nz}, 20 grains, seed 0, {args.study_steps} steps, symmetric parameter set"},
        "small_case_vs_oracle": small, "results": res, "data": "synthetic"}
    print(json.dumps(line), flush=True)


def run_region_study(args):
    """The paper's block compositions (Section 4: liquid, solid and interface blocks) at one
    domain size: FP32 MLUP/s of the default step (PF_VARIANT_AUTO, which chooses its path from the
    block's state), of the lean path ("fused") and of the two whole-domain sweeps on each, after a
    warm-up that gives the initially sharp interfaces their diffuse profile."""
    import time as _t

    import numpy as np

    from paper_1506_01684_gb300 import pf
    from paper_1506_01684_gb300 import workloads as W

    nx, ny, nz = (int(x) for x in args.region_shape.split("x"))
    p = W.symmetric_params()
    out = {}
    for kind in W.REGION_KINDS:
        phi0, mu0 = W.region_fields(kind, nx, ny, nz, seed=0)
        row = {}
        for variant in ("auto", "fused", "unfused"):
            sim = pf.Simulation(nx, ny, nz, p, "fp32", variant=variant)
            sim.set_fields(phi0, mu0)
            sim.step(20)
            sim.sync()
            if variant == "fused":
                phi, _ = sim.fields()
                onehot = (phi == 1.0).any(axis=0)
                row["interface_cell_fraction"] = float(1.0 - onehot.mean())
                row["liquid_cell_fraction"] = float((phi[3] == 1.0).mean())
            sim.step(args.warmup)
            sim.sync()
            t0 = _t.perf_counter()
            sim.step(args.steps)
            sim.sync()
            dt = _t.perf_counter() - t0
            row[variant + "_mlups"] = nx * ny * nz * args.steps / dt / 1e6
            if variant == "auto":  # the path the default chose from the block's state
                # (the lean path tallies its lean kernel and its general planes, a block without
                # pure-liquid planes only the latter)
                row["auto_path"] = "lean path" if set(sim.step_bytes()) & {"lean_step", "general_sweeps"} else "two sweeps"
            sim.close()
        row["auto_vs_best"] = row["auto_mlups"] / max(row["fused_mlups"], row["unfused_mlups"])
        out[kind] = row
        del phi0, mu0
    line = {"metric": "FP32 step MLUP/s on the paper's block compositions (liquid, solid, interface)",
            "unit": "MLUP/s", "higher_is_better": True, "steps": args.steps, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{nx}x{ny}x{nz} blocks: liquid; 3D solid grains ~48 cells; columnar "
                                   "grains ~12 cells below z = nz/2 with liquid above; 20 relaxation steps",
                       "timing": "wall clock around pf_step(K) + pf_sync, graph replay"},
            "regions": out}
    print(json.dumps(line), flush=True)


def run_mesh_study(args):
    """Per-phase interface meshes (the paper's isosurface output, Section 3.2) of the benchmark
    domain after a growth phase: device time of the three mesh kernels (CUDA events around each
    launch) and the wall time of the whole pf_interface_mesh call (count, scan, totals to the host,
    emit, copy of the triangles to pageable host memory), for each phase at iso 0.5.  Roofline of the
    counting kernel (the one that reads the whole field): the layout's algorithmic bytes, every
    cell's phi (4 words: the AoS cell the phase value sits in) read once."""
    import time as _t

    from paper_1506_01684_gb300 import pf
    from paper_1506_01684_gb300 import workloads as W

    p = W.symmetric_params(n_grains=args.grains, window_trigger_z=TRIGGER)
    sim = pf.Simulation(NX, NY, NZ, p, "fp32")
    sim.init(SEED)
    sim.step(args.mesh_steps)
    sim.sync()
    peak, peak_kind = _peaks()
    ncell = NX * NY * NZ
    phases = {}
    for a in range(4):
        for _ in range(args.warmup):
            tris = sim.interface_mesh(a, 0.5)
        pf.pf_profile(sim.h, True)
        pf.pf_profile_read(sim.h)
        t0 = _t.perf_counter()
        for _ in range(args.steps):
            tris = sim.interface_mesh(a, 0.5)
        wall = (_t.perf_counter() - t0) / args.steps
        prof = pf.pf_profile_read(sim.h)
        pf.pf_profile(sim.h, False)
        ms = {k: prof[k][0] / prof[k][1] for k in ("mesh_count", "mesh_scan", "mesh_emit")}
        b_c = 16.0 * ncell
        phases[a] = {"triangles": len(tris), "count_ms": ms["mesh_count"], "scan_ms": ms["mesh_scan"],
                     "emit_ms": ms["mesh_emit"], "call_ms": wall * 1e3,
                     "count_gbs": b_c / ms["mesh_count"] / 1e6,
                     "count_frac_of_" + peak_kind: b_c / ms["mesh_count"] / 1e6 / peak,
                     "kernel_gcells_per_s": ncell / sum(ms.values()) / 1e6}
    sim.close()
    line = {"metric": "interface-mesh extraction (per phase, marching tetrahedra): cells/s of the mesh kernels",
            "unit": "Gcell/s", "higher_is_better": True, "steps": args.steps, "warmup": args.warmup,
            "dtype": "f32", "data": "synthetic",
            "value": min(ph["kernel_gcells_per_s"] for ph in phases.values()),
            "peak_hbm_gbs": peak, "peak_kind": peak_kind,
            "config": {"workload": f"{WORKLOAD}, after {args.mesh_steps} steps, iso 0.5",
                       "timing": "CUDA events around each mesh kernel; wall clock around each call"},
            "phases": phases}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=None, help="steps of the FP64 comparison run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--study", default=None, choices=["batched", "serving", "precision", "regions", "mesh", "split"],
                    help="run a secondary study instead of the headline line")
    ap.add_argument("--requests", type=int, default=100, help="serving study: number of requests")
    ap.add_argument("--min-steps", type=int, default=100, help="serving study: fewest steps per request")
    ap.add_argument("--max-steps", type=int, default=1000, help="serving study: most steps per request")
    ap.add_argument("--load", type=float, default=0.8, help="serving study: offered load / capacity")
    ap.add_argument("--chunk", type=int, default=64, help="serving study: steps per scheduling round")
    ap.add_argument("--study-shape", default="128x128x512", help="precision study: domain")
    ap.add_argument("--study-steps", type=int, default=20000, help="precision study: steps")
    ap.add_argument("--region-shape", default="256x256x256", help="region study: block size")
    ap.add_argument("--mesh-steps", type=int, default=3000, help="mesh study: growth steps before the meshes")
    ap.add_argument("--variant", default="auto", choices=["auto", "unfused", "fused"],
                    help="kernel variant of the FP32 step (auto: the library's choice)")
    ap.add_argument("--grains", type=int, default=GRAINS,
                    help="Voronoi grains (0: pure liquid, a bulk-only diagnostic)")
    ap.add_argument("--shape", default=None,
                    help="NXxNYxNZ: a smaller domain of the same workload (profiling captures)")
    ap.add_argument("--pre-steps", type=int, default=PRE_STEPS,
                    help="untimed steps before the warm-up: the timed steps start from the state the "
                         "single-large-domain configuration reaches after its 2000 steps (0: the sharp initial state)")
    ap.add_argument("--state-file", default=None,
                    help="checkpoint of the pre-stepped state: written after the pre-steps when the file does not "
                         "exist, restored instead of the pre-steps when it does (a profiling capture then starts "
                         "from the same state without thousands of launches before the captured one)")
    ap.add_argument("--split-shape", default="256x256x256", help="split study: domain")
    ap.add_argument("--clocks-csv", default=None,
                    help="file for the nvidia-smi clock samples of the timed region (default: a temporary file)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.shape:
        global NX, NY, NZ, WORKLOAD
        NX, NY, NZ = (int(x) for x in args.shape.lower().split("x"))
    if args.shape or args.grains != GRAINS:
        WORKLOAD = (f"single domain {NX}x{NY}x{NZ}, {args.grains} grains, window trigger z=512, "
                    "symmetric parameter set")

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)

    if args.impl == "reference":
        run_reference(args, rank)
        return

    import numpy as np
    import torch

    from paper_1506_01684_gb300 import pf
    from paper_1506_01684_gb300 import workloads as W

    torch.cuda.set_device(local)
    if args.study == "batched":
        run_batched_study(args)
        return
    if args.study == "serving":
        run_serving_study(args)
        return
    if args.study == "precision":
        run_precision_study(args)
        return
    if args.study == "mesh":
        run_mesh_study(args)
        return
    if args.study == "regions":
        run_region_study(args)
        return
    if args.study == "split":
        run_split_study(args)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    # CPU baseline first (rank 0 only, N = 1 only), before any GPU work starts
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()

    params = W.symmetric_params(n_grains=args.grains, window_trigger_z=TRIGGER)
    stream = torch.cuda.Stream()
    cells = NX * NY * NZ

    # ---------------- FP32: the timed run ----------------
    sim = pf.Simulation(NX, NY, NZ, params, "fp32", stream=stream, variant=args.variant)
    sim.init(SEED)
    sol0 = sim.stats()["solute"]
    # the configuration's state: pre-steps advance the front from its sharp Voronoi start to the
    # diffuse, growing interface the configuration's 2000 steps reach (untimed)
    if args.state_file and os.path.exists(args.state_file):
        sim.restore(args.state_file)  # FP32 values: the pre-stepped state itself, bit for bit
    else:
        if args.pre_steps > 0:
            sim.step(args.pre_steps)
        if args.state_file:
            sim.checkpoint(args.state_file)
    sim.step(args.warmup)
    sim.sync()
    st_pre = sim.stats()
    clocks = ClockSampler(torch.cuda.current_device(), args.clocks_csv)
    clocks.start()
    time.sleep(0.3)
    # timed region A (the value): K steps as pf_step runs them, replayed from the captured graph
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    # timed region B (the kernels): the next K steps with the library's per-kernel event timers,
    # which launch every kernel directly between its two events (no graph)
    pf.pf_profile(sim.h, True)
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    pf.pf_profile(sim.h, False)
    ms_prof = e0.elapsed_time(e1)
    clk = clocks.stop()
    prof = pf.pf_profile_read(sim.h)
    sim.sync()
    # algorithmic bytes per kernel of the last timed step as the kernels tallied them (the front
    # moves less than a plane over the timed steps, so every timed launch moves about the same bytes)
    kbytes = sim.step_bytes()
    step_bytes = sum(kbytes.values())
    bytes_per_cell = {k: v / cells for k, v in kbytes.items()}
    ms_max = max_over_ranks(ms, dist, "cuda")
    value = whole_job_mlups(world, cells, args.steps, ms_max)
    # kernels launched in the timed steps: a timer record of the general planes' sweeps brackets their
    # two kernels (phi-sweep, mu-sweep), every other record one kernel
    launches = sum(n * KERNELS_PER_RECORD.get(k, 1) for k, (_, n) in prof.items())

    # dominant kernel and its roofline
    hbm, peak_kind = _peaks()
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms = prof[dom][0] / max(prof[dom][1], 1)
    kern = {k: {"ms_avg": v[0] / max(v[1], 1), "launches": v[1], "share": v[0] / max(sum(x[0] for x in prof.values()), 1e-30)}
            for k, v in prof.items()}
    achieved = bytes_per_cell.get(dom, 0) * cells / (dom_ms / 1e3) / 1e9
    traffic = None
    if dom in TRAFFIC_RATIO and dom in kbytes:
        traffic = TRAFFIC_RATIO[dom] * kbytes[dom]
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "peak_kind": peak_kind, "traffic": traffic,
            "bytes_per_cell": bytes_per_cell.get(dom)}
    for k in kern:
        if k in bytes_per_cell:
            kern[k]["gbs"] = bytes_per_cell[k] * cells / (kern[k]["ms_avg"] / 1e3) / 1e9
    design_bytes = step_bytes / cells
    fused_bound = hbm * 1e9 / (48 * cells) * cells / 1e6  # MLUP/s at 48 B/cell (fused FP32 minimum)
    unfused_bound = hbm * 1e9 / (88 * cells) * cells / 1e6
    design_bound = hbm * 1e9 / design_bytes / 1e6 if design_bytes else None
    # cells of the general planes (88 algorithmic bytes each in FP32: both sweeps' words)
    general_cells = kbytes.get("general_sweeps", 0.0) / 88.0
    roof_alu = alu_roofline(kern.get("general_sweeps"), general_cells, clk)

    phi32, mu32 = sim.fields()
    st32 = sim.stats()
    steps_done = args.pre_steps + args.warmup + 2 * args.steps

    # ---------------- FP64 GPU path on the same workload ----------------
    n64 = args.fp64_steps if args.fp64_steps is not None else steps_done
    fp64 = None
    fp32c = None
    if n64 > 0:
        s64 = pf.Simulation(NX, NY, NZ, params, "fp64", stream=stream)
        s64.init(SEED)
        w64 = min(args.warmup, n64)
        s64.step(w64)
        s64.sync()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        s64.step(n64 - w64)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1)
        fp64 = {"mlups": cells * (n64 - w64) / (ms64 / 1e3) / 1e6 if n64 > w64 else None, "steps": n64}
        if n64 == steps_done:
            phi64, mu64 = s64.fields()
            st64 = s64.stats()
            fp64["max_abs_dphi"] = float(np.abs(phi32 - phi64).max())
            fp64["max_rel_dmu"] = float(np.abs(mu32 - mu64).max() / max(np.abs(mu64).max(), 1e-8))
            fp64["solute_drift_fp32"] = [float((st32["solute"][c] - sol0[c]) / sol0[c]) for c in range(2)]
            fp64["solute_drift_fp64"] = [float((st64["solute"][c] - sol0[c]) / sol0[c]) for c in range(2)]
            s64.close()
            # the compensated FP32 path on the same workload: timed from the same state, and its error
            # against the same FP64 run after the same steps
            sc = pf.Simulation(NX, NY, NZ, params, "fp32c", stream=stream)
            sc.init(SEED)
            sc.step(args.pre_steps + args.warmup)
            sc.sync()
            f0.record(stream)
            sc.step(args.steps)
            f1.record(stream)
            torch.cuda.synchronize()
            msc = f0.elapsed_time(f1)
            sc.step(steps_done - args.pre_steps - args.warmup - args.steps)
            phic, muc = sc.fields()
            stc = sc.stats()
            fp32c = {"mlups": cells * args.steps / (msc / 1e3) / 1e6, "ms_per_step": msc / args.steps,
                     "steps": steps_done, "max_abs_dphi": float(np.abs(phic - phi64).max()),
                     "max_rel_dmu": float(np.abs(muc - mu64).max() / max(np.abs(mu64).max(), 1e-8)),
                     "solute_drift": [float((stc["solute"][c] - sol0[c]) / sol0[c]) for c in range(2)],
                     "what": "compensated FP32 state (hi + lo words), timed over the same K steps from the "
                             "same 2000-step state; error against the FP64 run after the same steps"}
            sc.close()
            del phi64, mu64, phic, muc
        else:
            s64.close()

    # ---------------- end to end through the public API with host buffers ----------------
    e2e = None
    if not args.no_e2e:
        # pinned host copies of the state in FP32 SoA (the ABI's FP32 host layout: the FP32 state's
        # own values, half the bytes of the FP64 layout)
        hphi = torch.from_numpy(phi32.astype(np.float32)).pin_memory()
        hmu = torch.from_numpy(mu32.astype(np.float32)).pin_memory()
        ophi = torch.empty_like(hphi).pin_memory()
        omu = torch.empty_like(hmu).pin_memory()
        del phi32, mu32
        import ctypes
        L = pf.lib()
        dp = ctypes.POINTER(ctypes.c_float)
        # one untimed run (first-use costs of the staging buffers and the pinned pages), then three
        # timed runs (host-memory bandwidth varies with other tenants of the machine): the median
        walls = []
        for it in range(4):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc = L.pf_write_fields_f32(sim.h, ctypes.cast(hphi.data_ptr(), dp), ctypes.cast(hmu.data_ptr(), dp))
            rc |= L.pf_step(sim.h, args.steps)
            rc |= L.pf_read_fields_f32(sim.h, ctypes.cast(ophi.data_ptr(), dp), ctypes.cast(omu.data_ptr(), dp),
                                       cells)
            torch.cuda.synchronize()
            if it > 0:
                walls.append(time.perf_counter() - t0)
            assert rc == 0, rc
        wall = statistics.median(walls)
        nbytes = cells * 6 * 4
        e2e = {"value": cells * args.steps / wall / 1e6, "unit": "MLUP/s",
               "h2d_bytes_per_step": nbytes / args.steps, "d2h_bytes_per_step": nbytes / args.steps,
               "runs_mlups": [cells * args.steps / w / 1e6 for w in walls],
               "what": "pf_write_fields_f32 (pinned FP32 host state) + pf_step(K) + pf_read_fields_f32, wall "
                       "clock, median of three runs after an untimed one"}
    sim.close()
    if cpu is not None:
        cpu["gpu_same_sample_mlups"] = gpu_on_cpu_sample(stream)
        cpu["gpu_same_sample_what"] = "the FP32 GPU step on the same 256x256x16 slab, 200 steps, CUDA events"
        g = gpu_on_oracle_samples(stream)
        for name, v in g.items():
            cpu["samples"][name]["gpu_fp32_mlups"] = v

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "MLUP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "ms_per_step_kernel_timers": ms_prof / args.steps,
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "nz": NZ, "cells": cells, "precision": "fp32",
                   "parallelism": f"replicas x{world}", "l2": "inputs (1.6 GB of fields) larger than L2"},
        "roofline": roof,
        "kernels": kern,
        "roofline_general": roof_alu,
        "bounds_mlups": {"fused_48B": fused_bound, "unfused_88B": unfused_bound,
                         "this_design_bytes_per_cell": design_bytes, "this_design": design_bound},
        "frac_of_design_bound": value / design_bound if design_bound else None,
        "state": {"steps_before_timing": args.pre_steps + args.warmup, "h_int": st_pre["h_int"],
                  "general_cell_fraction": general_cells / cells,
                  "what": "the timed steps start after the configuration's 2000 steps (pre-steps) and the warm-up"},
        "variant": ("lean kernel + general sweeps" if "lean_step" in prof
                    else ("fused" if "fused_step" in prof else "unfused")),
        "frac_of_unfused_bound": value / unfused_bound, "frac_of_fused_bound": value / fused_bound,
        "fp64": fp64, "fp32c": fp32c, "e2e": e2e, "cpu_baseline": cpu, "clocks": clk, "gpu_launches": launches,
        "window": {"h_int": st32["h_int"], "offset": st32["window_offset"]},
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
