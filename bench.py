#!/usr/bin/env python
"""Benchmark of the plane-strain LBM time loop on GB300.

One benchmark step is one time step of the whole method (Fig. 3): boundary
accelerations and reset, interior accelerations, Newmark, and the LBE for both
population sets, over the full lattice.  Default workload: the 8192 x 8192
lattice with lambda/mu = 3, a clamped bottom edge, traction-free other edges
and 32 seeded Gaussian dilatation/rotation pulses, FP32 populations, FP64
displacement (its state, 9.7 GB, is far larger than L2).

Prints one JSON line (rank 0).  Metric: two-field lattice updates per second
(GLUPS = lattice points x time steps / s / 1e9), whole job.
  --impl reference  times the FP64 CPU oracle on the host cores instead
                    (bounded sample of the same workload).
  --storage bf16|f16|bfp13  populations in the 16-bit formats (FP32 moments,
                    16-bit non-equilibrium sums); dtype stays the arithmetic type.
  --precision       adds the relative L2 error of FP32, BF16, FP16 and BFP13 storage
                    against the FP64 oracle on a 1024^2 crop rerun (5000
                    steps; about a minute of oracle time on the host cores).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))

METRIC = "two-field GLUPS"
UNIT = "GLUPS"
# algorithmic bytes per interior update: read + write of the populations and
# of u, du/dt (FP64); the 16-bit formats hold per set f^0, Jx, Jy in FP32 and
# two 16-bit non-equilibrium sums
BYTES_PER_UPDATE = {"f32": 2 * (10 * 4 + 4 * 8), "f64": 2 * (10 * 8 + 4 * 8),
                    "bf16": 2 * (6 * 4 + 4 * 2 + 4 * 8), "f16": 2 * (6 * 4 + 4 * 2 + 4 * 8),
                    "bfp13": 2 * (6 * 4 + 4 * 2 + 4 * 8)}


# ----------------------------------------------------------------- helpers

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate(local_seconds, local_units, world, reduce_max, reduce_sum):
    """Whole-job throughput: units summed over ranks / slowest rank's time."""
    t = reduce_max(local_seconds)
    u = reduce_sum(local_units)
    return u / t, t, u


def reducers(dist, device):
    """(max, sum) over the ranks of a process group of one Python float each,
    through a tensor on ``device`` ("cuda" under NCCL, "cpu" under gloo);
    plain float() when there is no process group."""
    if dist is None:
        return float, float
    import torch

    def red(x, op):
        t = torch.tensor([float(x)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=op)
        return float(t.item())

    return (lambda x: red(x, dist.ReduceOp.MAX)), (lambda x: red(x, dist.ReduceOp.SUM))


def workload(name, size=None):
    """(config name, Domain) of a workload recipe."""
    from paper_2301_00228_gb300 import workloads as W

    if name == "pulses":
        size = size or 8192
        return f"pulses_{size}", W.many_pulses(size=size)
    if name == "waves":
        size = size or 1024
        return f"waves_{size}", W.periodic_waves(size=size)
    if name == "square":
        return "square_64", W.square_64()
    if name == "hole":
        size = size or 8192
        return f"hole_{size}", W.hole_square(size)
    if name == "slab":
        size = size or 16384
        return f"slab_pulses_{size}", W.many_pulses(size=size)
    raise SystemExit(f"unknown workload {name}")


def describe(d):
    bc = {1: "N", 2: "D"}
    edges = "periodic" if d.periodic_x and d.periodic_y else "".join(bc[e] for e in d.edge_type)
    if d.hole is not None:
        out = {"nx": d.nx, "ny": d.ny, "lambda_over_mu": d.lam / d.mu, "a0_phi": d.a0_phi,
               "edges_bottom_right_top_left": edges, "hole": "centred, diameter 0.266 L, traction-free",
               "loads": "tension ramp to 0.005 mu at L/c_s", "sync_every": d.sync_every}
        nt = getattr(d, "node_type", None)
        if nt is not None:
            out.update(void_points=int((nt == 3).sum()), boundary_points=int(((nt == 1) | (nt == 2)).sum()))
        return out
    return {"nx": d.nx, "ny": d.ny, "lambda_over_mu": d.lam / d.mu, "a0_phi": d.a0_phi,
            "edges_bottom_right_top_left": edges, "pulses": len(d.pulses), "wave": d.wave}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm_sorted = sorted(sm)
        return {"sm_mhz": sm_sorted[len(sm) // 2], "sm_max_mhz": max(smax), "power_w_max": max(power),
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash():
    """sha256 (first 16 hex digits) of the code the normal build compiles
    from the kernel sources: the two files without // comments, blank lines
    and the branches only the range-checked build compiles (#ifdef
    LBPS_CHECKED), so editing a comment or the checked build keeps the
    recorded ncu traffic valid and editing the normal build's code does not."""
    code = []
    for name in ("lbps_kernels.cu", "lbps_device.cuh"):
        text = (ROOT / "paper_2301_00228_gb300" / "csrc" / name).read_text()
        stack = []  # per open #if: True while its lines belong to the checked build only
        for line in text.splitlines():
            line = re.sub(r"//.*", "", line).rstrip()
            d = line.strip()
            if d.startswith("#if"):
                stack.append(d == "#ifdef LBPS_CHECKED")
                if stack[-1]:
                    continue
            elif d.startswith("#else") and stack:
                was = stack[-1]
                stack[-1] = False
                if was:
                    continue
            elif d.startswith("#endif") and stack:
                if stack.pop():
                    continue
            if d and not any(stack):
                code.append(line)
    return hashlib.sha256("\n".join(code).encode()).hexdigest()[:16]


def ncu_traffic(workload_name, storage, kernel="bulk_kernel"):
    """DRAM bytes per launch of the kernel from the committed ncu summary, if it
    was taken on the current kernel source (else None)."""
    f = ROOT / "profiles" / f"{kernel}_{workload_name}_{storage}.md"
    if not f.exists():
        return None
    text = f.read_text()
    h = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", text)
    b = re.search(r"dram_bytes_per_full_launch:\s*([0-9.eE+]+)", text)
    if not h or not b or h.group(1) != kernel_source_hash():
        return None
    return float(b.group(1))


# ------------------------------------------------------------ CPU oracle

def oracle_lattice(d, side=1024):
    """The FP64 oracle on a side x side crop of the workload (bottom-left
    corner, same edge types; a plate with a hole is rebuilt at that size),
    initialised.  Returns (lattice, points, description of the sample)."""
    import numpy as np
    import oracle as O
    from paper_2301_00228_gb300 import workloads as W

    O.set_threads(os.cpu_count() or 1)
    if d.hole is not None:
        # the same plate with a hole at side x side, loads and synchronisation
        # (the oracle builds the plate's cells itself)
        n = min(side, d.nx)
        dd = W.hole_square(n, a0_phi=d.a0_phi, sync_every=d.sync_every)
        nt, bv, cell = O.disk_cells(n, n, *dd.hole, dd.edge_type, np.asarray(dd.edge_value, float).ravel())
        lat = O.OracleLattice(n, n, dd.lam, dd.mu, dd.rho, a0_phi=dd.a0_phi, node_type=nt, bc_value=bv,
                              cell=cell, sync_every=dd.sync_every)
        for kind, t_ramp, t_hold in dd.loads:
            lat.set_load(kind, t_ramp, t_hold)
        lat.init(np.zeros((n, n)), np.zeros((n, n)))
        return lat, n * n, f"{n}x{n} plate with the same hole, loads and synchronisation"
    side_x, side_y = min(side, d.nx), min(side, d.ny)
    if d.periodic_x and d.periodic_y:
        c = W.Domain(side_x, side_y, d.lam, d.mu, d.rho, d.a0_phi, periodic_x=True, periodic_y=True)
        m, n, ad, as_ = d.wave
        ux, uy = W.plane_wave_displacement(side_x, side_y, max(1, round(m * side_x / d.nx)),
                                           round(n * side_y / d.ny), ad, as_)
        nt = bv = None
    else:
        c = W.crop(d, 0, 0, side_x, side_y)
        ux, uy = d.displacement(window=(0, 0, side_x, side_y))
        et = [d.edge_type[0], 1, 1, d.edge_type[3]]
        nt, bv = O.rect_bc(side_x, side_y, et, np.asarray(d.edge_value, float).ravel())
    lat = O.OracleLattice(side_x, side_y, c.lam, c.mu, c.rho, a0_phi=c.a0_phi, periodic_x=c.periodic_x,
                          periodic_y=c.periodic_y, node_type=nt, bc_value=bv)
    lat.init(ux, uy)
    return lat, side_x * side_y, f"{side_x}x{side_y} corner crop of the workload (same material, edges of the corner kept)"


def time_oracle(lat, target_seconds, per=None):
    """Steps of the oracle lattice filling about target_seconds (the time per
    step measured on two steps unless given): (seconds, steps, seconds per step)."""
    if per is None:
        t0 = time.perf_counter()
        lat.step(2)
        per = (time.perf_counter() - t0) / 2
    steps = max(1, int(target_seconds / max(per, 1e-9)))
    t0 = time.perf_counter()
    lat.step(steps)
    dt = time.perf_counter() - t0
    return dt, steps, dt / steps


def oracle_sample(d, target_seconds=15.0, side=1024):
    """Time the FP64 oracle on the crop of oracle_lattice for as many steps as
    fill about target_seconds."""
    lat, points, what = oracle_lattice(d, side)
    dt, steps, _ = time_oracle(lat, target_seconds)
    return {"value": points * steps / dt / 1e9, "unit": UNIT, "cores": os.cpu_count() or 1, "kind": "oracle",
            "sample": f"{what}, {steps} FP64 steps in {dt:.1f} s"}, dt, steps


def precision_report(d, side, steps):
    """Relative L2 per field of every storage format against the FP64 oracle
    on a side x side stand-alone crop of the workload (the window with the
    most pulse centres; the workload's edge types on its edges; the pulses
    centred inside), run for the given number of steps."""
    import numpy as np
    import oracle as O
    from paper_2301_00228_gb300 import lbps
    from paper_2301_00228_gb300 import workloads as W

    x0, y0 = W.busiest_crop(d, side)
    c = W.crop(d, x0, y0, side, side)
    ux, uy = c.displacement()
    ev = np.asarray(c.edge_value, float).ravel()
    fields = ("ux", "uy", "phi", "psi")
    got = {}
    for st in ("f32", "bf16", "f16", "bfp13"):
        lat = lbps.Lattice.rectangle(side, side, c.lam, c.mu, c.edge_type, ev, a0_phi=c.a0_phi, storage=st)
        lat.init(ux, uy).step(steps)
        got[st] = ({k: lat.read(k) for k in fields}, lat.scale_exp)
        lat.close()
    O.set_threads(os.cpu_count() or 1)
    nt, bv = O.rect_bc(side, side, c.edge_type, ev)
    t0 = time.perf_counter()
    ref = O.OracleLattice(side, side, c.lam, c.mu, c.rho, a0_phi=c.a0_phi, node_type=nt, bc_value=bv)
    ref.init(ux, uy).step(steps)
    secs = time.perf_counter() - t0
    rf = ref.fields()
    out = {}
    for st, (g, e) in got.items():
        errs = {}
        for grp in (("ux", "uy"), ("phi", "psi")):
            gn = np.sqrt(sum(np.linalg.norm(rf[k]) ** 2 for k in grp))
            for k in grp:
                den = max(np.linalg.norm(rf[k]), 1e-2 * gn, 1e-300)
                errs[k] = float(np.linalg.norm(g[k] - rf[k]) / den)
        out[st] = {"rel_l2": errs, "max": max(errs.values()), "scale_exp": e,
                   "bytes_per_update": BYTES_PER_UPDATE[st]}
    return {"crop": f"{side}x{side} at ({x0}, {y0})", "pulses": len(c.pulses), "steps": steps,
            "a0_phi": c.a0_phi, "oracle_seconds": secs, "oracle_threads": os.cpu_count() or 1, "formats": out}


def run_reference(args):
    """The FP64 oracle on the host cores, one bounded sample per timed step
    (a crop of the workload, built once): each step runs as many oracle steps
    as fill min(--ref-seconds, 150 s / steps), so the whole run stays within a
    few minutes for any --steps."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    wname, d = workload(args.workload, args.size)
    lat, points, what = oracle_lattice(d)
    target = min(args.ref_seconds, 150.0 / max(1, args.steps))
    _, _, per = time_oracle(lat, 0.5)
    for _ in range(args.warmup):
        time_oracle(lat, target, per)
    secs, n_steps = [], []
    for _ in range(args.steps):
        dt, steps, per = time_oracle(lat, target, per)
        secs.append(dt)
        n_steps.append(steps)
    value = points * sum(n_steps) / sum(secs) / 1e9
    cb = {"value": value, "unit": UNIT, "cores": os.cpu_count() or 1, "kind": "oracle",
          "sample": f"{what}; {args.steps} timed samples of {min(n_steps)}-{max(n_steps)} FP64 steps, "
                    f"{sum(secs):.1f} s in all"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(secs) / len(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wname, **describe(d)},
            "cpu_baseline": cb, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm

def run_batch(args):
    """256 seeded rectangles (sides U{64..512}, random edges and lambda/mu), all
    advanced as one batch; compared with stepping the same lattices one at a time."""
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:  # each rank advances its own copy of the batch (weak scaling)
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2301_00228_gb300 import lbps
    from paper_2301_00228_gb300 import workloads as W

    ds = W.mixed_batch(count=args.batch_count)
    lats = []
    for d in ds:
        lat = lbps.Lattice.rectangle(d.nx, d.ny, d.lam, d.mu, d.edge_type, np.asarray(d.edge_value, float).ravel(),
                                     a0_phi=d.a0_phi, storage=args.storage)
        lat.init(*d.displacement())
        lats.append(lat)
    points = sum(d.nx * d.ny for d in ds)
    interior = sum((d.nx - 2) * (d.ny - 2) for d in ds)
    b = lbps.Batch(lats)
    if args.batch_tuning:  # a fixed launch shape (profiling), no tuner
        shape = [int(x) for x in args.batch_tuning.split(",")]
        variant, rows = shape[:2]
        b.set_tuning(variant, rows)
        if len(shape) > 2:
            b.set_graph_steps(shape[2])
        tuned_ms = None
    else:
        variant, rows, tuned_ms = b.tune(repeats=5)
    pairs = args.batch_pairs == "on"
    if pairs:  # two steps per sweep for every lattice
        b.set_step_pairs(True)
    stream = torch.cuda.current_stream()
    b.step(args.warmup)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    if dist is not None:
        dist.barrier()
    clock = clocks.stop()
    if b.check() != 0:
        raise SystemExit("state became non-finite")
    rmax, rsum = reducers(dist, "cuda")
    seconds = rmax(e0.elapsed_time(e1) / 1000.0)          # slowest rank
    value = rsum(points * args.steps) / seconds / 1e9      # points of all ranks
    # the same lattices stepped one at a time (same kernels, one lattice per
    # launch), each with single steps, its faster mode at these sizes
    if pairs:
        for lat in lats:
            lbps.lbps_set_step_pairs(lat._h, 0)
    loop_steps = max(2, args.steps // 10)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for lat in lats:
        lbps.lbps_step_async(lat._h, loop_steps)
    torch.cuda.synchronize()
    loop_s = time.perf_counter() - t0
    loop_value = points * loop_steps / loop_s / 1e9
    peak, peak_kind = measured_peaks()
    step_s = seconds / args.steps
    per_update = BYTES_PER_UPDATE[args.storage]
    if pairs:
        # per pair of steps: the points at least 3 from every edge read and
        # written once, the first step on the points 1..3 from the edges and
        # the second on those 1..2 from them read and written once each
        deep = sum(max(d.nx - 6, 0) * max(d.ny - 6, 0) for d in ds)
        band = lambda w: sum((d.nx - 2) * (d.ny - 2) - max(d.nx - 2 - 2 * w, 0) * max(d.ny - 2 - 2 * w, 0) for d in ds)
        alg_pair = (deep + band(3) + band(2)) * per_update
        achieved = alg_pair / (2 * step_s) / 1e9
    else:
        achieved = interior * per_update / step_s / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * step_s, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.storage == "f64" else "f32", "data": "synthetic",
            "config": {"workload": f"mixed_batch_{len(ds)}", "domains": len(ds), "sides": "U{64..512}",
                       "points": points, "storage": args.storage, "l2": "state larger than L2",
                       "steps_per_sweep": 2 if pairs else 1,
                       "tuned": {"variant": variant, "rows_per_warp": rows, "graph_steps": b.graph_steps,
                                 "ms_per_step": tuned_ms}},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "whole batched step",
                         "peak_source": peak_kind},
            "one_at_a_time": {"value": loop_value, "unit": UNIT, "steps": loop_steps,
                              "speedup_of_batch": value / loop_value},
            # per step: the persistent kernel (strips and Newmark tasks) and the reset
            # (two steps per sweep: two persistent kernels and two resets a pair)
            "gpu_launches": (3 if args.storage == "bfp13" else 2) * args.steps, "clocks": clock}
    if rank == 0:
        print(json.dumps(line), flush=True)
    b.close()
    for lat in lats:
        lat.close()
    return 0


def serve_measure(requests=64, rate_factor=1.2, burst=32, budget_gb=64.0, small_budget=None, max_chunk=500,
                  sample=6, pairs=True):
    """Serving measurements on one GPU: a Poisson stream of solves (sides
    log-uniform 128..2048, steps U{500..20000}, edges and lambda/mu as in the
    mixed batch) at rate_factor x the capacity of the one-solve-at-a-time
    loop (measured first on a sample of the same recipe), served by
    continuous batching and by that loop; a second batched run under a small
    device-memory budget (default 1.2 x the largest request's footprint, so
    admission binds: requests wait for memory, memory_waits > 0); and a burst of the first requests arriving at once
    (capacity).  With pairs the batched server takes two time steps per sweep
    (each solve charged its scratch copy).  Latency = completion - arrival."""
    from paper_2301_00228_gb300 import serve as S
    from paper_2301_00228_gb300 import workloads as W

    smp = [S.Request(i, 0.0, d, d.steps)
           for i, (_, d) in enumerate(W.poisson_requests(count=sample, seed=55, rate_hz=1.0))]
    prep = {r.rid: r.domain.displacement() for r in smp}
    S.serve_one_at_a_time(smp[:1], prepared=prep)  # warm-up
    t0 = time.perf_counter()
    S.serve_one_at_a_time(smp, prepared=prep)
    service = (time.perf_counter() - t0) / len(smp)
    rate = rate_factor / service
    reqs = [S.Request(i, t, d, d.steps)
            for i, (t, d) in enumerate(W.poisson_requests(count=requests, seed=5, rate_hz=rate))]
    prepared = {r.rid: r.domain.displacement() for r in reqs}
    work = sum(r.domain.nx * r.domain.ny * r.steps for r in reqs)
    budget = int(budget_gb * (1 << 30))
    biggest = max(S.footprint(r.domain, pairs=pairs) for r in reqs)
    small_bytes = int(small_budget * (1 << 30)) if small_budget else int(1.2 * biggest)
    served = S.serve_batched(reqs, budget, prepared=prepared, max_chunk=max_chunk, pairs=pairs)
    small = S.serve_batched(reqs, small_bytes, prepared=prepared, max_chunk=max_chunk, pairs=pairs)
    loop = S.serve_one_at_a_time(reqs, prepared=prepared)
    sv, lp = served.summary(), loop.summary()
    out = {"config": {"requests": len(reqs), "sides": "log-U 128..2048", "steps": "U{500..20000}",
                      "rate_hz": rate, "rate_factor": rate_factor, "loop_service_s_mean": service,
                      "budget_gb": budget_gb, "lattice_updates": work, "batch_steps_per_sweep": 2 if pairs else 1},
           "served": {**sv, "glups": work / served.makespan / 1e9},
           "one_at_a_time": {**lp, "glups": work / loop.makespan / 1e9},
           "speedup_solves_per_s": sv["solves_per_s"] / lp["solves_per_s"],
           "p99_latency_ratio": lp["p99_latency_s"] / sv["p99_latency_s"],
           "served_small_budget": {**small.summary(), "budget_gb": small_bytes / (1 << 30),
                                   "largest_request_gb": biggest / (1 << 30)}}
    bst = [S.Request(r.rid, 0.0, r.domain, r.steps) for r in reqs[:burst]]
    bwork = sum(r.domain.nx * r.domain.ny * r.steps for r in bst)
    bs = S.serve_batched(bst, budget, prepared=prepared, max_chunk=max_chunk, pairs=pairs)
    bl = S.serve_one_at_a_time(bst, prepared=prepared)
    out["capacity_burst"] = {"requests": len(bst), "served_solves_per_s": bs.summary()["solves_per_s"],
                             "loop_solves_per_s": bl.summary()["solves_per_s"],
                             "served_glups": bwork / bs.makespan / 1e9, "loop_glups": bwork / bl.makespan / 1e9,
                             "speedup": bl.makespan / bs.makespan, "served_max_active": bs.max_active}
    return out, served


def run_serve(args):
    """Serving as its own JSON line (metric: served solves/s); see serve_measure."""
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:  # each rank serves its own copy of the stream (replicas)
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    m, served = serve_measure(args.requests, args.rate_factor, args.burst, args.budget_gb,
                              args.small_budget_gb or None, args.max_chunk, args.serve_sample)
    sv = m["served"]
    rmax, rsum = reducers(dist, "cuda")
    total = rsum(sv["solves_per_s"])               # solves/s of all replicas
    sv["p99_latency_s_max_over_ranks"] = rmax(sv["p99_latency_s"])
    line = {"metric": "served solves/s", "value": total, "unit": "solves/s", "n_gpus": world,
            "steps": m["config"]["requests"], "warmup": 1,
            "ms_per_step": 1000.0 * served.makespan / m["config"]["requests"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"serve_poisson_{m['config']['requests']}", **m["config"]},
            **{k: v for k, v in m.items() if k != "config"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_slab(args):
    """One lattice split into slabs of rows, one per rank (strong scaling:
    the lattice is the same for every N), ghost rows exchanged through NCCL
    after every step (paper_2301_00228_gb300.slab).  Default: the 16384^2
    many-pulse lattice (same recipe as the pulses workload).  At N = 1 the one
    slab is the whole lattice and nothing is exchanged."""
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2301_00228_gb300 import lbps
    from paper_2301_00228_gb300 import slab as S
    from paper_2301_00228_gb300 import workloads as W

    size = args.size or 16384
    d = W.many_pulses(size=size)
    ev = np.asarray(d.edge_value, float).ravel()
    nt, bv = lbps.lbps_rect_bc(d.nx, d.ny, 0, 0, 1.0, d.edge_type, ev)
    p = S.plan(d.ny, world, rank)
    eng = S.CudaSlab(p, d.nx, d.lam, d.mu, d.rho, node_type=nt, bc_value=bv, a0_phi=d.a0_phi, storage=args.storage)
    run = S.SlabRun(eng, p, dist)
    ux, uy = d.displacement_torch("cuda", rows=(p.first, p.rows))
    run.init_rows(ux, uy)
    del ux, uy
    stream = torch.cuda.current_stream()
    run.step(args.warmup)
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    lbps.lbps_profile(eng.lat._h, 1)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    barrier()
    clock = clocks.stop()
    if eng.lat.check() != 0:
        raise SystemExit("state became non-finite")
    prof = lbps.lbps_profile_read(eng.lat._h)
    lbps.lbps_profile(eng.lat._h, 0)
    seconds = e0.elapsed_time(e1) / 1000.0
    owned = (p.y1 - p.y0) * d.nx
    rmax, rsum = reducers(dist, "cuda")
    value_ups, t_max, units_all = aggregate(seconds, owned * args.steps, world, rmax, rsum)
    bulk_ms, bulk_n = float(prof[0]), float(prof[1])
    interior = (d.nx - 2) * (p.rows - 2)
    alg = interior * BYTES_PER_UPDATE[args.storage]
    peak, peak_kind = measured_peaks()
    achieved = alg / (bulk_ms / max(bulk_n, 1) / 1000.0) / 1e9
    halo = lbps.lbps_halo_bytes(eng.lat._h, S.HALO)
    line = {"metric": METRIC, "value": value_ups / 1e9, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * t_max / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f64" if args.storage == "f64" else "f32",
            "data": "synthetic",
            "config": {"workload": f"slab_pulses_{size}", **describe(d), "storage": args.storage,
                       "displacement": "f64", "parallelism": f"slab{world}", "halo_rows": S.HALO,
                       "rows_per_rank": [p.y1 - p.y0], "halo_bytes_per_message": halo if world > 1 else 0,
                       "l2": "state larger than L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "kernel": "bulk_kernel (rank 0's slab)", "peak_source": peak_kind},
            # per step: boundary Newmark, interior, reset; per neighbour one pack and
            # one unpack (copy, boundary mirror, boundary stresses)
            "gpu_launches": int(bulk_n) * (4 if args.storage == "bfp13" else 3) +
            args.steps * 4 * ((p.down is not None) + (p.up is not None)),
            "clocks": clock}
    if rank == 0:
        print(json.dumps(line), flush=True)
    eng.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def bulk_roofline(prof, d, args, seconds, geometry, peak, peak_kind, wname):
    """The interior kernel of single steps: the state read and written once per
    step at every interior point (events around every launch)."""
    bulk_ms, bulk_n, bnd_ms, bnd_n = (float(x) for x in prof)
    if geometry is not None:  # interior points only; the kernel also reads one node-type byte per point
        interior = int((geometry[0] == 0).sum())
        alg_bytes = interior * (BYTES_PER_UPDATE[args.storage] + 1)
    else:
        interior = (d.nx - (0 if d.periodic_x else 2)) * (d.ny - (0 if d.periodic_y else 2))
        alg_bytes = interior * BYTES_PER_UPDATE[args.storage]
    bulk_avg_s = bulk_ms / max(bulk_n, 1) / 1000.0
    achieved = alg_bytes / bulk_avg_s / 1e9
    # timed on the lattice's stream: the interior kernel and the boundary
    # reset; the boundary Newmark pass runs beside the interior kernel on a
    # second stream and is not timed (lbps_profile)
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": ncu_traffic(wname, args.storage), "kernel": "bulk_kernel", "peak_source": peak_kind,
            "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": bulk_avg_s * 1000.0,
            "share_of_step_time": bulk_ms / (1000.0 * seconds),
            "kernel_timing": "a window after the timed steps (--graphs)" if args.graphs
            else "CUDA events around every launch of the timed steps",
            "timed_boundary_passes_ms_per_step": bnd_ms / args.steps,
            "boundary_newmark_pass": "beside the interior kernel on a second stream, not timed"}


def pair_roofline(prof, d, args, seconds, peak, peak_kind, wname):
    """The two-step kernel: it reads the state of the points at least 3 from
    every edge once and writes it once per launch, for two steps of updates
    (events around every launch), with u, du/dt integrated over both steps
    in one composed Newmark update."""
    pair_ms, pair_n = float(prof[0]), float(prof[1])
    deep = (d.nx - 6) * (d.ny - 6)
    alg_bytes = deep * BYTES_PER_UPDATE[args.storage]
    avg_s = pair_ms / max(pair_n, 1) / 1000.0
    achieved = alg_bytes / avg_s / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": ncu_traffic(wname, args.storage, kernel="pair_kernel"), "kernel": "pair_kernel",
            "peak_source": peak_kind, "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_s * 1000.0,
            "steps_per_launch": 2, "updates_per_launch": 2 * deep,
            "bytes_per_update": alg_bytes / (2 * deep),
            "limiter": "latency at 20 warps/SM with the FP64 pipe about 2/3 busy (one composed Newmark update of u, du/dt per point per launch)",
            "share_of_step_time": pair_ms / (1000.0 * seconds),
            "kernel_timing": "CUDA events around every two-step launch of the timed steps",
            "frame_and_boundary_passes": "beside the two-step kernel on a second stream of greatest priority, "
                                          "not timed; they run on SM slots the kernel's retiring blocks free, so "
                                          "the kernel's launch time includes them"}


def single_step_window(lbps, lat, d, args, points, peak, stream):
    """The same lattice with single steps, timed over a shorter window (for
    comparison with two steps per sweep); the lattice keeps its state."""
    import torch

    lbps.lbps_set_step_pairs(lat._h, 0)
    n = min(args.steps, 300)
    lat.step(4)
    lbps.lbps_profile(lat._h, 1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rc = lbps.lbps_step_async(lat._h, n)
    e1.record(stream)
    e1.synchronize()
    prof = lbps.lbps_profile_read(lat._h)
    lbps.lbps_profile(lat._h, 0)
    lbps.lbps_set_step_pairs(lat._h, 1)
    if rc != 0:
        raise SystemExit(f"step failed: {lbps.lbps_strerror(rc)}")
    s = e0.elapsed_time(e1) / 1000.0
    bulk_avg_s = float(prof[0]) / max(float(prof[1]), 1) / 1000.0
    alg = (d.nx - 2) * (d.ny - 2) * BYTES_PER_UPDATE[args.storage]
    return {"value": points * n / s / 1e9, "unit": UNIT, "steps": n, "ms_per_step": 1000.0 * s / n,
            "bulk_kernel_frac": alg / bulk_avg_s / 1e9 / peak, "bulk_kernel_avg_ms": bulk_avg_s * 1000.0}


def run_gpu(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU for the default arm")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2301_00228_gb300 import lbps

    wname, d = workload(args.workload, args.size)
    et = d.edge_type
    ev = np.asarray(d.edge_value, float).ravel()
    stream = torch.cuda.current_stream()
    geometry = None
    if d.hole is not None:  # the plate's node types and cells, built by the library
        geometry = lbps.lbps_disk_cells(d.nx, d.ny, 1.0, *d.hole, et, ev)
        d.node_type = geometry[0]
    sync_every = args.sync_every if args.sync_every or geometry is None else d.sync_every
    mk = dict(a0_phi=d.a0_phi, storage=args.storage, sync_every=sync_every,
              step_pairs={"auto": "auto", "on": True, "off": False}[args.pairs])
    if geometry is not None:
        nt, bv, cell = geometry
        lat = lbps.Lattice(d.nx, d.ny, d.lam, d.mu, d.rho, node_type=nt, bc_value=bv, cell=cell, **mk)
        for kind, t_ramp, t_hold in d.loads:
            lat.set_load(kind, t_ramp, t_hold)
    elif d.periodic_x and d.periodic_y:
        lat = lbps.Lattice(d.nx, d.ny, d.lam, d.mu, d.rho, periodic_x=True, periodic_y=True, **mk)
    else:
        lat = lbps.Lattice.rectangle(d.nx, d.ny, d.lam, d.mu, et, ev, **mk)
    if args.tuning:  # a fixed launch shape of the interior kernel (profiling a smaller lattice like a larger)
        variant, rows = (int(x) for x in args.tuning.split(","))
        lbps.lbps_set_tuning(lat._h, variant, rows)
    pairs = bool(lbps.lbps_step_pairs(lat._h))  # two steps per sweep (large rectangles)
    ux, uy = d.displacement_torch("cuda")
    lat.init(ux, uy)
    torch.cuda.synchronize()

    # warm-up
    lat.step(args.warmup)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    # per-kernel CUDA events around every launch of the timed steps; with
    # --graphs the timed steps replay captured step pairs instead (no events
    # inside), and the kernel timings come from a window of steps after them
    lbps.lbps_profile(lat._h, 0 if args.graphs else 1)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rc = lbps.lbps_step_async(lat._h, args.steps)
    e1.record(stream)
    e1.synchronize()
    barrier()
    clock = clocks.stop()
    if rc != 0:
        raise SystemExit(f"step failed: {lbps.lbps_strerror(rc)}")
    if lat.check() != 0:
        raise SystemExit("state became non-finite")
    if args.graphs:
        lbps.lbps_profile(lat._h, 1)
        lat.step(min(args.steps, 200))
    prof = lbps.lbps_profile_read(lat._h)
    lbps.lbps_profile(lat._h, 0)
    seconds = e0.elapsed_time(e1) / 1000.0
    # lattice updates: body points (void points of a general geometry hold no state)
    points = int((geometry[0] != 3).sum()) if geometry is not None else d.nx * d.ny
    units = points * args.steps

    rmax, rsum = reducers(dist, "cuda")
    value_ups, t_max, units_all = aggregate(seconds, units, world, rmax, rsum)
    value = value_ups / 1e9

    # roofline of the dominant kernel
    peak, peak_kind = measured_peaks()
    if pairs:
        roofline = pair_roofline(prof, d, args, seconds, peak, peak_kind, wname)
        # per pair of steps: the two-step kernel; beside it the boundary
        # Newmark and reset of each step and two frame passes of four launches
        # (BFP13 storage: one more launch per reset, its y streams)
        split = 1 if args.storage == "bfp13" else 0
        gpu_launches = (args.steps // 2) * (13 + 2 * split) + (args.steps % 2) * (3 + split)
        single = single_step_window(lbps, lat, d, args, points, peak, stream)
    else:
        roofline = bulk_roofline(prof, d, args, seconds, geometry, peak, peak_kind, wname)
        bounded = not (d.periodic_x and d.periodic_y)
        # per step: boundary Newmark, interior, boundary reset (a periodic lattice
        # has no boundary); per synchronisation: the sync kernel and the refresh
        # of the boundary mirror
        split = 1 if args.storage == "bfp13" else 0
        gpu_launches = args.steps * ((3 + split) if bounded else 1) + (
            (args.steps // sync_every) * (2 if bounded else 1) if sync_every else 0)
        single = None

    # end to end through the C ABI with host buffers
    e2e = None
    if args.e2e_steps > 0:
        pin_ux = torch.empty((d.ny, d.nx), dtype=torch.float64, pin_memory=True)
        pin_uy = torch.empty((d.ny, d.nx), dtype=torch.float64, pin_memory=True)
        pin_ux.copy_(ux.cpu())
        pin_uy.copy_(uy.cpu())
        out_x = torch.empty((d.ny, d.nx), dtype=torch.float64, pin_memory=True)
        out_y = torch.empty((d.ny, d.nx), dtype=torch.float64, pin_memory=True)
        # untimed warm-up of the same calls: each init swaps the state copies,
        # so two passes capture the step graphs of both starting copies; both
        # reads, so that the copy engine has touched both host buffers
        for _ in range(2):
            lbps.lbps_init(lat._h, pin_ux.numpy(), pin_uy.numpy())
            lbps.lbps_step(lat._h, 64)
            lbps.lbps_read(lat._h, lbps.LBPS_UX, out_x.numpy())
            lbps.lbps_read(lat._h, lbps.LBPS_UY, out_y.numpy())
        barrier()
        t0 = time.perf_counter()
        lbps.lbps_init(lat._h, pin_ux.numpy(), pin_uy.numpy())
        ti = time.perf_counter()
        rc = lbps.lbps_step(lat._h, args.e2e_steps)
        ts = time.perf_counter()
        lbps.lbps_read(lat._h, lbps.LBPS_UX, out_x.numpy())
        lbps.lbps_read(lat._h, lbps.LBPS_UY, out_y.numpy())
        t1 = time.perf_counter()
        barrier()
        if rc != 0:
            raise SystemExit(f"e2e step failed: {lbps.lbps_strerror(rc)}")
        e2e_ups, _, _ = aggregate(t1 - t0, points * args.e2e_steps, world, rmax, rsum)
        e2e = {"value": e2e_ups / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": 2 * d.nx * d.ny * 8, "d2h_bytes_per_step": 2 * d.nx * d.ny * 8,
               "seconds": {"init": ti - t0, "steps": ts - ti, "read": t1 - ts},
               "step": f"one solve: lbps_init from pinned host u0, lbps_step({args.e2e_steps}), "
                       f"lbps_read of u_x and u_y into pinned host memory (after two untimed solves of 64 steps)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, _, _ = oracle_sample(d, target_seconds=args.ref_seconds)
    serving = None
    if rank == 0 and world == 1 and args.serve_requests > 0:
        lat.close()  # its device memory back before the serving runs
        serving, _ = serve_measure(args.serve_requests, args.rate_factor, args.serve_burst, args.budget_gb, None,
                                   args.max_chunk, args.serve_sample)
    precision = None
    if rank == 0 and args.precision and not (d.periodic_x and d.periodic_y):
        precision = precision_report(d, args.precision_side, args.precision_steps)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1000.0 * t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.storage == "f64" else "f32",
                "data": "synthetic",
                "config": {"workload": wname, **describe(d), "storage": args.storage,
                           "displacement": "f64", "sync_every": sync_every,
                           "l2": "state larger than L2" if roofline["alg_bytes_per_launch"] > 1.3e8 else "state fits L2",
                           "replicas_per_gpu": 1, **({"tuning": args.tuning} if args.tuning else {})},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches,
                "clocks": clock}
        line["config"]["steps_per_sweep"] = 2 if pairs else 1
        if single is not None:
            line["single_step"] = single
        if precision is not None:
            line["precision"] = precision
        if serving is not None:
            line["serving"] = serving
        print(json.dumps(line), flush=True)
    lat.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="pulses",
                    choices=["pulses", "waves", "square", "hole", "batch", "serve", "slab"])
    ap.add_argument("--requests", type=int, default=64, help="serve: requests in the Poisson stream")
    ap.add_argument("--serve-sample", type=int, default=6, help="serve: solves timed to set the arrival rate")
    ap.add_argument("--rate-factor", type=float, default=1.2, help="serve: arrival rate / loop capacity")
    ap.add_argument("--budget-gb", type=float, default=64.0, help="serve: device-memory admission budget")
    ap.add_argument("--small-budget-gb", type=float, default=0.0,
                    help="serve: budget of the second run (0: 1.2 x the largest request's footprint)")
    ap.add_argument("--max-chunk", type=int, default=500, help="serve: most steps between completions checks")
    ap.add_argument("--burst", type=int, default=32, help="serve: requests arriving at once for the capacity run")
    ap.add_argument("--serve-requests", type=int, default=48,
                    help="serving section of the lattice workloads' line: requests (0: none)")
    ap.add_argument("--serve-burst", type=int, default=24, help="serving section: burst requests")
    ap.add_argument("--batch-count", type=int, default=256, help="domains of the batch workload")
    ap.add_argument("--batch-pairs", default="on", choices=["on", "off"],
                    help="batch: two time steps per sweep for every lattice")
    ap.add_argument("--batch-tuning", default=None,
                    help="batch: launch shape 'variant,rows[,steps per graph]' instead of running the autotuner")
    ap.add_argument("--pairs", default="auto", choices=["auto", "on", "off"],
                    help="lattice workloads: two time steps per sweep (auto: on from 3M points where they apply)")
    ap.add_argument("--tuning", default=None,
                    help="lattice workloads: interior-kernel launch shape 'variant,rows' instead of the default")
    ap.add_argument("--size", type=int, default=None, help="lattice side (pulses: 8192, waves: 1024)")
    ap.add_argument("--storage", default="f32", choices=["f32", "f64", "bf16", "f16", "bfp13"])
    ap.add_argument("--precision", action="store_true",
                    help="pulses: add rel-L2 of every storage format against the FP64 oracle on a crop rerun")
    ap.add_argument("--precision-side", type=int, default=1024)
    ap.add_argument("--precision-steps", type=int, default=5000)
    ap.add_argument("--sync-every", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=1000)
    ap.add_argument("--graphs", action="store_true",
                    help="time the steps as lbps_step runs them for a caller (pairs replayed from CUDA graphs) "
                         "and take the per-kernel timings from a window after them")
    ap.add_argument("--ref-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "slab":
        return run_slab(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
