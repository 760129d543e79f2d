#!/usr/bin/env python3
"""Throughput of the coupled D3Q15 + D3Q7 MRT multiphase update on GB300.

One benchmark step is one full time step of the solver over the whole grid (order
parameter pass, chemical-potential pass, fused stream-collide pass).  The workload is
the Rayleigh-Taylor instability at Re = 4000, At = 0.5 on a 256 x 256 x 1024 grid
(67M cells, FP32 storage), initial condition of Eqs. 42-43.

Printed JSON line (rank 0):
  value      MLUPS (million cell updates per second) over all ranks, device-timed with
             CUDA events around exactly --steps steps; inputs resident in HBM.
  e2e        the same metric through the public C ABI with host buffers: pinned-host
             phi0 uploaded by lbm_init_phi, every step taken by lbm_step_reduce_async
             (the step plus the FP64 mass, momentum and non-finite count of its result,
             copied to pinned host memory and checked there, two steps in flight),
             lbm_read_fields (phi, u, p) at the end.
  roofline   the fused stream-collide kernel: algorithmic bytes per launch / its mean
             CUDA-event duration, against the measured HBM copy bandwidth.
  cpu_baseline  the FP64 oracle on a bounded sample, one single-threaded replica per host
             core (rank 0, N = 1).
  storage_variants / pattern_variants / model_variants  the same measurement with FP16
             and BF16 storage, the in-place pattern, the single-pass step, the SRT flow
             lattice, the D3Q7-weighted stencils, and interface tracking with the
             prescribed deformation field (periodic 256^3).
  serving    the request loop: a seeded Poisson stream of Rayleigh-Taylor runs of
             mixed grids served by continuous batching and one at a time; p50/p99
             time to solution and aggregate MLUPS of each (step counts scaled by
             --serve-scale, 0.1 by default, to keep the leg near a minute).
With --impl reference the oracle alone is timed on the host cores (the reference arm).
Under torchrun each rank runs an independent replica (weak scaling, no collective on
the data path).
"""
from __future__ import annotations

import argparse
import copy
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "coupled D3Q15+D3Q7 MLUPS"
UNIT = "MLUPS"

# Algorithmic bytes per cell of the fused stream-collide kernel, FP32: read f (7) and
# g (15) populations, phi u of the previous step (3), phi and mu at the cell (2); write
# f, g and phi u (25).  The neighbour values of phi and mu are re-reads of the same two
# planes, which the kernel is meant to serve from cache.
COLLIDE_BYTES_PER_CELL = (22 + 3 + 2) * 4 + (22 + 3) * 4
STEP_BYTES_PER_CELL = COLLIDE_BYTES_PER_CELL + (7 + 1) * 4 + (1 + 1) * 4  # + k_phi + k_mu

# The same with 16-bit populations: 22 x 2 B populations + 12 B phi u, read and written,
# plus phi and mu (k_collide); 7 x 2 B of f, the previous phi and the new phi (k_phi).
COLLIDE_BYTES_PER_CELL_16 = 2 * (22 * 2 + 12) + 8
STEP_BYTES_PER_CELL_16 = COLLIDE_BYTES_PER_CELL_16 + (7 * 2 + 4 + 4) + 8

# Interface tracking with a prescribed velocity (k_che): read f, phi and mu at the cell
# and phi u of the previous step (48 B), write f and phi u (40 B); the step adds k_phi
# and k_mu.
CHE_BYTES_PER_CELL = (7 + 1 + 1 + 3) * 4 + (7 + 3) * 4
CHE_STEP_BYTES_PER_CELL = CHE_BYTES_PER_CELL + (7 + 1) * 4 + (1 + 1) * 4

# The one-kernel step (k_fused): the state read and written once (200 B in FP32); with
# 16-bit populations 2 x (44 + 12) plus phi of the previous step read and the new phi
# written (the slot-0 shift).
FUSED_BYTES_PER_CELL = 2 * (22 + 3) * 4
FUSED_BYTES_PER_CELL_16 = 2 * (22 * 2 + 12) + 8

# DRAM traffic per cell of the dominant kernel from an ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum divided by the cells of the captured launch), valid only for the
# kernel source it was taken on (hash of csrc/lbm_device.cuh, lbm_cells.cuh,
# lbm_kernels.cu and lbm_fused.cu).  Captures of one launch on the 128 x 128 x 512 case
# (8,388,608 cells), scaled by cells to the benchmark: the traffic of these kernels grows
# in proportion to the cells.
NCU_TRAFFIC = {
    # 955.4 MB read + 793.1 MB written (stencil rows staged in shared memory)
    "k_collide2t": {"bytes_per_cell": 208.43, "kernel_sha": "162676c4fdc99dd4"},
    # 536.9 MB + 432.6 MB
    "k_collide2_fp16": {"bytes_per_cell": 115.58, "kernel_sha": "162676c4fdc99dd4"},
    # 856.6 MB + 797.7 MB with segments of 64 planes and no L2 prefetch (the traffic of
    # the single pass depends on both: 266.3 B per cell with 18 planes and 2 planes of
    # prefetch)
    "k_fused": {"bytes_per_cell": 197.20, "kernel_sha": "162676c4fdc99dd4", "segment": 64,
                "prefetch": 0},
}

WORKLOADS = {
    "rt256": dict(W=256, Re=4000.0, desc="Rayleigh-Taylor 256x256x1024, Re=4000, At=0.5, "
                                        "sqrt(gW)=0.04, D=4, sigma=1e-4, Pe=50, FP32 storage"),
    "rt128": dict(W=128, Re=1024.0, desc="Rayleigh-Taylor 128x128x512, Re=1024, At=0.5"),
    "rt64": dict(W=64, Re=256.0, desc="Rayleigh-Taylor 64x64x256, Re=256, At=0.5"),
}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in ("lbm_device.cuh", "lbm_cells.cuh", "lbm_kernels.cu", "lbm_fused.cu"):
        with open(os.path.join(ROOT, "paper_1507_07294_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks ------
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.device_index = device_index
        self.proc = None
        self.lines = []
        self._thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.device_index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self._thread = threading.Thread(target=self._read, daemon=True)
        self._thread.start()

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
        if self._thread:
            self._thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------- CPU oracle ------
ORACLE_CHILD = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
from oracle import lbm_oracle as O
from paper_1507_07294_gb300 import inputs as I
W, Re, nz, warm, steps_max, budget = {W}, {Re}, {nz}, {warm}, {steps_max}, {budget}
start_at = {start_at}
w = I.rayleigh_taylor(W=W, Re=Re, nz=nz)
o = O.Oracle(O.Params.from_workload(w))
o.init(w.phi0)
o.step(max(1, warm))
while time.time() < start_at:  # replicas start their timed loops together
    time.sleep(0.01)
t0 = time.perf_counter(); n = 0
while n < steps_max and (n < 1 or time.perf_counter() - t0 < budget):
    o.step(1); n += 1
dt = time.perf_counter() - t0
print(json.dumps({{"cells": w.cells, "steps": n, "seconds": dt, "grid": [w.nx, w.ny, w.nz]}}))
"""


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_oracle_sample(W: int, Re: float, nz: int, steps_max: int, budget_s: float,
                      warm: int = 1, replicas: int = 1) -> dict:
    """Time the FP64 oracle as independent single-threaded replicas, one per host core,
    each in a fresh interpreter (spawned, so no CUDA state is inherited), all starting
    their timed loops at the same moment.  Returns the summed cell updates over the
    slowest replica's time."""
    env = dict(os.environ)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[var] = "1"
    start_at = time.time() + 5.0 + 0.2 * replicas
    code = ORACLE_CHILD.format(root=ROOT, W=W, Re=Re, nz=nz, warm=warm, steps_max=steps_max,
                               budget=budget_s, start_at=start_at)
    procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True, env=env)
             for _ in range(replicas)]
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=1800)
        if p.returncode != 0:
            raise RuntimeError("oracle sample failed: " + err[-2000:])
        outs.append(json.loads(out.strip().splitlines()[-1]))
    d = dict(outs[0])
    d["replicas"] = replicas
    d["seconds"] = max(o["seconds"] for o in outs)
    d["steps_each"] = [o["steps"] for o in outs]
    d["steps"] = min(o["steps"] for o in outs)
    d["mlups"] = sum(o["cells"] * o["steps"] for o in outs) / d["seconds"] / 1e6
    return d


def oracle_baseline(budget_s: float = 15.0) -> dict:
    cores = host_cores()
    d = run_oracle_sample(64, 4000.0, 64, 200, budget_s, replicas=cores)
    return {"value": round(d["mlups"], 4), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 numpy oracle as it stands, {cores} independent single-threaded "
                      f"replicas (one per host core), each the Rayleigh-Taylor setup at Re=4000 "
                      f"on a 64x64x64 slab, {min(d['steps_each'])}-{max(d['steps_each'])} steps "
                      f"after 1 untimed step, {d['seconds']:.1f} s; summed cell updates over "
                      f"the slowest replica's time"}


# ------------------------------------------------------------------ helpers ------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class RankGroup:
    """The host-side collectives of the benchmark: a barrier and a max over ranks.

    Each rank runs an independent replica, so these are the only collectives; they
    are used for timing, never on the data path.  backend "nccl" reduces a CUDA tensor,
    "gloo" a CPU one; with one rank both are no-ops.
    """

    def __init__(self, world: int, rank: int, backend: str = "nccl"):
        self.world, self.rank, self.backend = world, rank, backend

    def _device(self):
        return "cuda" if self.backend == "nccl" else "cpu"

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max(self, x: float) -> float:
        if self.world == 1:
            return float(x)
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(x)], dtype=torch.float64, device=self._device())
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())


def aggregate_mlups(cells: int, steps: int, world: int, elapsed_s: float) -> float:
    """Whole-job MLUPS: the cell updates of all replicas over the slowest rank's time."""
    return cells * steps * world / elapsed_s / 1e6


def config_dict(args, w, world):
    spec = WORKLOADS[args.workload]
    return {"workload": f"{args.workload}: {spec['desc']}",
            "grid": [w.nx, w.ny, w.nz], "cells": w.cells, "walls_z": bool(w.walls_z),
            "storage": getattr(args, "storage", "fp32"), "pattern": getattr(args, "pattern", "ab"),
            "l2": f"state {w.cells * 100 / 1e9:.1f} GB (f, g, phi u) > 129 MB L2: no flush needed",
            "parallelism": f"replicas x{world} (independent runs per GPU)"}


# ------------------------------------------------------------ serving leg -------
def run_serving(args, rank: int) -> dict:
    """The continuous-batching request loop against one-at-a-time service, on the same
    seeded Poisson request stream: grids 32^3, 64^3, 64x64x256, 128x128x512; Re, At,
    sigma uniform; step counts uniform in [2000, 20000] x --serve-scale; arrivals
    rescaled so the offered load is --serve-load x the one-at-a-time capacity measured
    on this GPU; admission by a --serve-budget-gb device-memory budget."""
    import torch
    from paper_1507_07294_gb300 import serve as S

    lo, hi = max(1, round(2000 * args.serve_scale)), max(1, round(20000 * args.serve_scale))
    reqs = S.request_stream(args.serve_requests, seed=1000 + rank, steps=(lo, hi))
    eng = S.GpuEngine()
    # untimed: batch grid autotuning on one run per grid, per-grid service times alone
    tuned = S.tune_batch(eng, S.GRIDS, quantum=args.serve_quantum)
    model = S.service_time_model(eng, S.GRIDS, steps=200)
    loaded = S.with_load(reqs, lambda r: model[r.grid][0] * r.steps + model[r.grid][1],
                         args.serve_load)
    budget = int(args.serve_budget_gb * 1e9)
    res = {}
    # runs that take their own launches (the tuned size split) count as large
    large_cells = tuned.get("split_cells") or max(g[0] * g[1] * g[2] for g in S.GRIDS)
    max_large = args.serve_max_large or None
    for name, batched in (("batched", True), ("one_at_a_time", False)):
        srv = S.Server(eng, budget, max_runs=args.serve_slots, quantum=args.serve_quantum,
                       batched=batched, max_large=max_large if batched else None,
                       large_cells=large_cells)
        outs = srv.serve(loaded)
        summ = S.summarize(outs)
        by_rid = {r.rid: r for r in loaded}
        bad = [by_rid[o.rid] for o in outs if not o.stable]
        summ["unstable_by_grid"] = {"x".join(map(str, g)): sum(r.grid == g for r in bad)
                                    for g in S.GRIDS}
        summ["unstable_min_nu"] = (round(min(0.04 * r.grid[0] / r.re for r in bad), 6)
                                   if bad else None)
        summ.update(peak_runs=srv.peak_runs, peak_gb=round(srv.peak_bytes / 1e9, 3),
                    quanta=srv.quanta)
        res[name] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in summ.items()}
    eng.close()
    return {
        "requests": len(reqs), "grids": [list(g) for g in S.GRIDS],
        "steps_range": [lo, hi], "re": [100, 4000], "atwood": [0.1, 0.9],
        "sigma": [1e-3, 1e-2], "offered_load_x_one_at_a_time": args.serve_load,
        "arrival_span_s": round(loaded[-1].arrival, 3), "budget_gb": args.serve_budget_gb,
        "max_runs": args.serve_slots, "quantum_steps": args.serve_quantum,
        "max_large_runs": max_large, "large_cells": large_cells,
        "alone_ms_per_step": {"x".join(map(str, g)): round(v[0] * 1e3, 4)
                              for g, v in model.items()},
        "batch_tuning": {k: v for k, v in tuned.items() if not k.endswith("_ms")},
        "time_to_solution": "arrival to phi and the FP64 sums on the host",
        **res,
        "mlups_ratio": round(res["batched"]["mlups"] / res["one_at_a_time"]["mlups"], 3),
    }


# ------------------------------------------------------------ reference arm -----
def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1507_07294_gb300 import inputs as I
    spec = WORKLOADS[args.workload]
    w = I.rayleigh_taylor(W=spec["W"], Re=spec["Re"])
    # Each reference step is one oracle step on a bounded sample of the workload: the
    # 64-wide crop of the same setup, depth shrunk so W + K steps fit ~150 s.
    total = args.warmup + args.steps
    cores = host_cores()
    probe = run_oracle_sample(64, spec["Re"], 64, 1, 0.0)  # calibration
    per_cell = probe["seconds"] / probe["cells"]
    nz = int(max(16, min(256, 150.0 / max(total, 1) / per_cell / (64 * 64))))
    d = run_oracle_sample(64, spec["Re"], nz, args.steps, 1e9, warm=args.warmup,
                          replicas=cores)
    value = d["mlups"]
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * d["seconds"] / d["steps"], 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic: Rayleigh-Taylor initial condition (Eqs. 42-43)",
            "config": config_dict(args, w, world),
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": cores,
                             "kind": "oracle",
                             "sample": f"FP64 numpy oracle as it stands, {cores} independent "
                                       f"single-threaded replicas (one per host core); one bench "
                                       f"step is one oracle step of every replica on a "
                                       f"64x64x{nz} slab of the same setup"},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm ------
def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    device = torch.cuda.current_device()

    from paper_1507_07294_gb300 import inputs as I
    from paper_1507_07294_gb300 import lbm as L

    spec = WORKLOADS[args.workload]
    w = I.rayleigh_taylor(W=spec["W"], Re=spec["Re"])
    stream = torch.cuda.current_stream()
    solver = L.Solver(w, stream=stream.cuda_stream, pattern=args.pattern, storage=args.storage)
    ctx = solver.ctx
    if not getattr(args, "cell_pairs", 1):
        L.lbm_set_tuning(ctx, L.LBM_TUNE_CELL_PAIRS, 0)
    single_pass = bool(getattr(args, "single_pass", False))
    if single_pass:
        L.lbm_set_tuning(ctx, L.LBM_TUNE_FUSED, 1)
        if getattr(args, "fused_segment", None) is not None:
            L.lbm_set_tuning(ctx, L.LBM_TUNE_FUSED_SEGMENT, args.fused_segment)
        if getattr(args, "fused_prefetch", None) is not None:
            L.lbm_set_tuning(ctx, L.LBM_TUNE_FUSED_PREFETCH, args.fused_prefetch)

    group = RankGroup(world, rank, "nccl")

    def barrier():
        torch.cuda.synchronize()
        group.barrier()
        torch.cuda.synchronize()

    max_over_ranks = group.max

    # ---- warm-up and autotuning (untimed) ------------------------------------
    from paper_1507_07294_gb300 import tune
    solver.step(args.warmup)
    tuning = None
    if not args.no_tune:
        tuning = (tune.autotune_fused if single_pass else tune.autotune)(ctx)
        torch.cuda.synchronize()

    # ---- device-timed region -------------------------------------------------
    L.lbm_profile(ctx, True)
    clocks = ClockSampler(device)
    clocks.start()
    time.sleep(0.3)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    solver.step(args.steps)
    e1.record(stream)
    barrier()
    clock = clocks.stop()
    elapsed_ms = max_over_ranks(e0.elapsed_time(e1))
    kernels = {}
    for k, name in enumerate(L.KERNEL_NAMES):
        ms, n = L.lbm_profile_read(ctx, k)
        kernels[name] = {"launches": n, "total_ms": round(ms, 4),
                         "mean_ms": round(ms / max(n, 1), 5)}
    L.lbm_profile(ctx, False)
    sum_phi, _ = solver.reduce()  # the run stayed finite
    pairs = L.lbm_get_tuning(ctx, L.LBM_TUNE_CELL_PAIRS) == 1
    staged = L.lbm_get_tuning(ctx, L.LBM_TUNE_STENCIL_STAGE) == 1
    coll_name = ("k_fused" if L.lbm_get_tuning(ctx, L.LBM_TUNE_FUSED) == 1
                 else "k_collide2t" if staged else "k_collide2" if pairs else "k_collide")

    cells = w.cells
    value = aggregate_mlups(cells, args.steps, world, elapsed_ms * 1e-3)
    coll_ms = kernels["k_collide"]["mean_ms"]
    peak, peak_kind = measured_peaks()
    wide = args.storage == "fp32"
    coll_bytes = COLLIDE_BYTES_PER_CELL if wide else COLLIDE_BYTES_PER_CELL_16
    step_bytes = STEP_BYTES_PER_CELL if wide else STEP_BYTES_PER_CELL_16
    if coll_name == "k_fused":  # the whole step: the state read and written once
        coll_bytes = step_bytes = FUSED_BYTES_PER_CELL if wide else FUSED_BYTES_PER_CELL_16
    achieved = coll_bytes * cells / (coll_ms * 1e-3) / 1e9
    src_hash = kernel_source_hash()
    tr = NCU_TRAFFIC.get(coll_name if wide else f"{coll_name}_{args.storage}")
    if tr and coll_name == "k_fused":  # the single pass's traffic depends on its settings
        if (tr.get("segment"), tr.get("prefetch")) != (
                L.lbm_get_tuning(ctx, L.LBM_TUNE_FUSED_SEGMENT),
                L.lbm_get_tuning(ctx, L.LBM_TUNE_FUSED_PREFETCH)):
            tr = None
    traffic = round(tr["bytes_per_cell"] * cells) if tr and tr.get("kernel_sha") == src_hash else None

    # ---- end-to-end region through the C ABI with host buffers ---------------
    def e2e_run(nsteps):
        phi_host = torch.empty(cells, dtype=torch.float64, pin_memory=True).numpy()
        phi_host[:] = w.phi0.reshape(-1)
        # page-locked result buffers, allocated once like a server's I/O buffers
        outs = {k: torch.empty(c * cells, dtype=torch.float64, pin_memory=True).numpy()
                for k, c in (("phi", 1), ("u", 3), ("p", 1))}
        # every step's FP64 sums (sum phi, momentum, count of non-finite cells) go to the
        # host through two pinned slots, which the library's reduction writes directly
        # (the out_dev of lbm_step_reduce_async may be host memory the device can write):
        # step k is enqueued once the sums of step k - 2 have arrived and been checked, so
        # the GPU never waits for the host
        sums_host = torch.zeros((2, 8), dtype=torch.float64, pin_memory=True)
        arrived = [torch.cuda.Event(), torch.cuda.Event()]

        def check_sums(slot):
            arrived[slot].synchronize()
            v = sums_host[slot].numpy()
            if v[4] != 0 or not np.isfinite(v[:4]).all():
                raise RuntimeError(f"e2e run diverged: sums {v[:5]}")

        def run(n):
            """Upload, n steps with their sums, read-out; the host times of each part."""
            t0 = time.perf_counter()
            L.lbm_init_phi(ctx, phi_host)
            t1 = time.perf_counter()
            for k in range(n):
                slot = k & 1
                if k >= 2:
                    check_sums(slot)
                L.lbm_step_reduce_async(ctx, 1, sums_host[slot].data_ptr())  # step + its sums
                arrived[slot].record(stream)
            for k in range(max(0, n - 2), n):
                check_sums(k & 1)
            t2 = time.perf_counter()
            out = L.lbm_read_fields(ctx, L.LBM_FIELD_PHI | L.LBM_FIELD_U | L.LBM_FIELD_P,
                                    out=outs)
            t3 = time.perf_counter()
            assert np.isfinite(out["phi"]).all()
            return t3 - t0, (t1 - t0, t2 - t1, t3 - t2)

        run(4)  # untimed: the library's device staging buffers come from the allocator's cache
        barrier()
        t_e2e, parts = run(nsteps)
        barrier()
        t_e2e = max_over_ranks(t_e2e)
        return {"value": round(aggregate_mlups(cells, nsteps, world, t_e2e), 3), "unit": UNIT,
                "h2d_bytes_per_step": round(8 * cells / nsteps),
                "d2h_bytes_per_step": round(5 * 8 + 5 * 8 * cells / nsteps),
                "steps": nsteps, "seconds": round(t_e2e, 4),
                "upload_ms": round(1e3 * parts[0], 2), "steps_ms": round(1e3 * parts[1], 2),
                "readout_ms": round(1e3 * parts[2], 2)}

    e2e = None
    e2e_sustained = None
    if not args.no_e2e:
        e2e = e2e_run(args.steps)
        # the same over 1000 steps or more: the one upload and the one read-out amortised
        e2e_sustained = e2e if args.steps >= 1000 else e2e_run(1000)

    # ---- reduced-precision storage variants (same workload and step count) ------
    variants = None
    pattern_variants = None
    model_variants = None
    if not args.no_variants and args.storage == "fp32":
        solver.close()
        variants = {}
        pattern_variants = {}
        runs = [("fp16", "ab", "fp16"), ("bf16", "ab", "bf16")]
        if args.pattern == "ab":
            runs.append(("aa", "aa", "fp32"))  # in place: half the state memory
            runs.append(("aa_fp16", "aa", "fp16"))  # in place with 16-bit populations
            runs.append(("single_pass", "ab", "fp32"))  # one kernel per step (LBM_TUNE_FUSED)
        for name, pattern, storage in runs:
            wide_v = storage == "fp32"
            cb = COLLIDE_BYTES_PER_CELL if wide_v else COLLIDE_BYTES_PER_CELL_16
            sb = STEP_BYTES_PER_CELL if wide_v else STEP_BYTES_PER_CELL_16
            vs = L.Solver(w, stream=stream.cuda_stream, pattern=pattern, storage=storage)
            if name == "single_pass":
                L.lbm_set_tuning(vs.ctx, L.LBM_TUNE_FUSED, 1)
            vs.step(args.warmup)
            if not args.no_tune:
                vt = (tune.autotune_fused if name == "single_pass" else tune.autotune)(vs.ctx)
            L.lbm_profile(vs.ctx, True)
            barrier()
            v0 = torch.cuda.Event(enable_timing=True)
            v1 = torch.cuda.Event(enable_timing=True)
            v0.record(stream)
            vs.step(args.steps)
            v1.record(stream)
            barrier()
            vms = max_over_ranks(v0.elapsed_time(v1))
            cms, cn = L.lbm_profile_read(vs.ctx, L.KERNEL_COLLIDE)
            cmean = cms / max(cn, 1)
            entry = {
                "value": round(aggregate_mlups(cells, args.steps, world, vms * 1e-3), 3),
                "unit": UNIT, "ms_per_step": round(vms / args.steps, 5),
                "speedup_vs_fp32": round(elapsed_ms / vms, 3),
                "k_collide_ms": round(cmean, 5),
                "k_collide_bytes_per_cell": cb,
                "k_collide_frac": round(cb * cells / (cmean * 1e-3) / 1e9 / peak, 4),
                "step_bytes_per_cell": sb}
            if not args.no_tune:
                entry["tuning"] = {k: v["value"] for k, v in vt.items()}
            if name == "single_pass":
                entry["kernel"] = "k_fused"
                entry["k_fused_ms"] = entry.pop("k_collide_ms")
                entry["algorithmic_bytes_per_cell"] = 200
                entry["hbm_frac_at_200_bytes"] = round(
                    200 * cells / (cmean * 1e-3) / 1e9 / peak, 4)
                for key in ("k_collide_bytes_per_cell", "k_collide_frac", "step_bytes_per_cell"):
                    entry.pop(key)
                entry["segment_planes"] = L.lbm_get_tuning(vs.ctx, L.LBM_TUNE_FUSED_SEGMENT)
                pattern_variants[name] = entry
            elif pattern == "aa":
                for key, pat, sto in (("context_gb", pattern, storage), ("context_gb_ab", "ab", "fp32")):
                    grid_p, params_p = L.params_from_workload(w, pat, sto)
                    entry[key] = round(L.lbm_memory_bytes(grid_p, params_p) / 1e9, 2)
                pattern_variants[name] = entry
            else:
                variants[name] = entry
            vs.close()

        # ---- model variants: the SRT flow lattice and the D3Q7-weighted stencils on the
        # same workload, and interface tracking with the prescribed deformation field of
        # Eq. 41 on a periodic 256^3 box (the paper's Sec. III B test at twice the size)
        if args.pattern == "ab":
            model_variants = {}
            srt = copy.copy(w)
            srt.srt_flow = True
            d7 = copy.copy(w)
            d7.stencil = "d3q7"
            mruns = [("srt_flow", srt, "k_collide", COLLIDE_BYTES_PER_CELL, STEP_BYTES_PER_CELL),
                     ("d3q7_stencil", d7, "k_collide", COLLIDE_BYTES_PER_CELL,
                      STEP_BYTES_PER_CELL),
                     ("interface_tracking", I.deformation(n=256), "k_che", CHE_BYTES_PER_CELL,
                      CHE_STEP_BYTES_PER_CELL)]
            for name, wv, kname, cb, sb in mruns:
                vs = L.Solver(wv, stream=stream.cuda_stream)
                vs.step(args.warmup)
                vt = tune.autotune(vs.ctx) if not args.no_tune else None
                L.lbm_profile(vs.ctx, True)
                barrier()
                v0 = torch.cuda.Event(enable_timing=True)
                v1 = torch.cuda.Event(enable_timing=True)
                v0.record(stream)
                vs.step(args.steps)
                v1.record(stream)
                barrier()
                vms = max_over_ranks(v0.elapsed_time(v1))
                cms, cn = L.lbm_profile_read(vs.ctx, L.KERNEL_COLLIDE)
                cmean = cms / max(cn, 1)
                entry = {
                    "workload": wv.name if name == "interface_tracking" else "as the main line",
                    "cells": wv.cells,
                    "value": round(aggregate_mlups(wv.cells, args.steps, world, vms * 1e-3), 3),
                    "unit": UNIT, "ms_per_step": round(vms / args.steps, 5),
                    "kernel": kname, "kernel_ms": round(cmean, 5),
                    "kernel_bytes_per_cell": cb,
                    "kernel_frac": round(cb * wv.cells / (cmean * 1e-3) / 1e9 / peak, 4),
                    "step_bytes_per_cell": sb,
                    "step_hbm_frac": round(sb * wv.cells * args.steps / (vms * 1e-3) / 1e9 / peak,
                                           4)}
                if vt:
                    entry["tuning"] = {k: v["value"] for k, v in vt.items()}
                model_variants[name] = entry
                vs.close()

    if variants is None:
        solver.close()

    serving = None
    if not args.no_serving:
        barrier()
        serving = run_serving(args, rank)
        barrier()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_baseline()

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(elapsed_ms / args.steps, 5), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic: Rayleigh-Taylor initial condition (Eqs. 42-43), no dataset",
                "config": config_dict(args, w, world),
                "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                             "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                             "kernel": coll_name,
                             "bytes_per_cell": coll_bytes,
                             "peak_source": f"{peak_kind} HBM copy bandwidth"},
                "step_bytes_per_cell": step_bytes,
                "step_hbm_frac": round(step_bytes * cells * args.steps /
                                       (elapsed_ms * 1e-3) / 1e9 / peak, 4),
                "kernels": kernels,
                "tuning": {k: v["value"] for k, v in tuning.items()} if tuning else None,
                "storage_variants": variants, "pattern_variants": pattern_variants,
                "model_variants": model_variants,
                "serving": serving,
                "cpu_baseline": cpu, "e2e": e2e, "e2e_sustained": e2e_sustained, "clocks": clock,
                "gpu_launches": (1 if coll_name == "k_fused" else 3) * args.steps,
                "sum_phi": sum_phi}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="rt256")
    ap.add_argument("--pattern", choices=("ab", "aa"), default="ab",
                    help="population storage: two arrays (ab) or in place (aa)")
    ap.add_argument("--storage", choices=("fp32", "fp16", "bf16"), default="fp32",
                    help="population storage of the main run (arithmetic is FP32 in all)")
    ap.add_argument("--single-pass", action="store_true",
                    help="run the main leg with the one-kernel step (LBM_TUNE_FUSED)")
    ap.add_argument("--fused-segment", type=int, default=None,
                    help="with --single-pass: planes per block segment (0: by grid size)")
    ap.add_argument("--fused-prefetch", type=int, default=None,
                    help="with --single-pass: L2 prefetch distance in planes")
    ap.add_argument("--cell-pairs", type=int, choices=(0, 1), default=1,
                    help="two cells per thread in the stream-collide pass where it applies")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip timing the FP16/BF16 population-storage variants")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the untimed autotuning of prefetch distances")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the request-loop leg (batched vs one at a time)")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-scale", type=float, default=0.1,
                    help="step counts are uniform in [2000, 20000] times this")
    ap.add_argument("--serve-load", type=float, default=1.5,
                    help="offered load in units of the one-at-a-time capacity")
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    ap.add_argument("--serve-slots", type=int, default=16)
    ap.add_argument("--serve-quantum", type=int, default=64)
    ap.add_argument("--serve-max-large", type=int, default=2,
                    help="at most this many large runs (those that take their own "
                         "launches) at once in the batched server (0: no cap)")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
