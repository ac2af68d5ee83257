"""Continuous-batching serving of plane-strain LBM solves on one GPU.

A request is one solve: a rectangle (sizes, material, edges, initial
displacement) and a step count.  ``Server.run`` takes requests with arrival
times and serves them as they arrive:

* admission: a waiting request is admitted when the device memory its
  lattice needs (``lbps_state_bytes``) fits in what the budget has left; its
  populations then stay resident until it completes;
* batching: all admitted solves advance together as one ``Batch`` (one launch
  of each kernel per time step for all of them, CUDA graphs for step pairs),
  in chunks no longer than the shortest remaining solve, so every solve stops
  exactly at its step count; a solve that is alone on the device is stepped
  directly (lbps_step, the single-lattice kernels and their launch shape);
* completion: finished solves leave the batch at the chunk boundary; they
  are read out (their u fields) and freed while the next chunk runs, and
  requests that arrive meanwhile are created and initialised then too (on
  streams of their own, beside the batch's), joining at the next boundary;
* cancellation: a request withdrawn by its client (``cancel_at``) leaves the
  queue, or the batch at the next chunk boundary, and its memory is freed.

``serve_one_at_a_time`` is the plain baseline: the same kernels, one solve at
a time in arrival order.  Both report per-request latency (completion minus
arrival) and throughput.  A solve gets the same bits alone, in the batch, or
in the baseline loop, because the batched kernels run the per-point
arithmetic of the single-lattice ones.  With ``pairs`` the batch takes two
time steps per sweep (lbps_batch_set_step_pairs) when every member allows
it: the populations are the same bits, u and du/dt the same up to the
rounding of the composed two-step update, and each admitted solve is
charged one more state copy (its scratch copy).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import lbps


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    domain: object          # workloads.Domain
    steps: int
    cancel_at: float | None = None  # the client withdraws the request at this time (None: never)

    def cancelled_by(self, now):
        return self.cancel_at is not None and self.cancel_at <= now


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    completed: float
    ux: np.ndarray | None = None
    uy: np.ndarray | None = None

    @property
    def latency(self):
        return self.completed - self.arrival


@dataclass
class Report:
    results: list = field(default_factory=list)
    makespan: float = 0.0
    chunks: int = 0
    rebuilds: int = 0
    max_active: int = 0
    peak_bytes: int = 0
    cancelled: list = field(default_factory=list)   # rids withdrawn before completion
    memory_waits: int = 0          # chunk boundaries at which an arrived request did not fit the budget
    memory_wait_s: float = 0.0     # summed time requests waited for memory after they arrived

    def summary(self):
        lat = np.array([r.latency for r in self.results])
        return {"solves": len(self.results), "solves_per_s": len(self.results) / self.makespan,
                "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
                "mean_latency_s": float(lat.mean()), "makespan_s": self.makespan, "chunks": self.chunks,
                "batch_rebuilds": self.rebuilds, "max_active": self.max_active, "peak_state_bytes": self.peak_bytes,
                "cancelled": len(self.cancelled), "memory_waits": self.memory_waits,
                "memory_wait_s": self.memory_wait_s}


def _params(d, storage):
    return lbps.lbps_params(d.nx, d.ny, d.lam, d.mu, d.rho, 1.0, d.a0_phi, int(d.periodic_x), int(d.periodic_y),
                            0, 0, lbps.STORAGES[storage], 0, None)


def pairs_apply(d):
    """Two steps per sweep apply to the domain: a rectangle without periodic
    axes, at least 16 points a side."""
    return not d.periodic_x and not d.periodic_y and min(d.nx, d.ny) >= 16


def footprint(d, storage="f32", pairs=False):
    """Device bytes one solve holds while admitted; with two steps per sweep
    also the scratch state copy, counted as half the lattice's block (which
    holds two copies and more: an upper bound)."""
    b = lbps.lbps_state_bytes(_params(d, storage))
    return b + b // 2 if pairs and pairs_apply(d) else b


def _lattice(d, storage, u0=None, stream=None):
    lat = lbps.Lattice.rectangle(d.nx, d.ny, d.lam, d.mu, d.edge_type, np.asarray(d.edge_value, float).ravel(),
                                 periodic_x=d.periodic_x, periodic_y=d.periodic_y, a0_phi=d.a0_phi,
                                 storage=storage, stream=stream)
    ux, uy = u0 if u0 is not None else d.displacement()
    return lat.init(ux, uy)


class _Clock:
    def __init__(self, clock):
        self.clock = clock
        self.t0 = clock()

    def now(self):
        return self.clock() - self.t0

    def wait_until(self, t):
        while True:
            dt = t - self.now()
            if dt <= 0:
                return
            time.sleep(min(dt, 0.01))


def _streams():
    """(a function giving each new lattice a stream, the batch stream):
    non-blocking CUDA streams from torch's pool, so that new solves are
    created, initialised and read out, and a lone solve is stepped, while a
    chunk of the batch runs (the legacy default stream would wait for it);
    no streams without a GPU."""
    try:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.Stream, torch.cuda.Stream()
    except ImportError:
        pass
    return (lambda: None), None


def serve_batched(requests, budget_bytes, storage="f32", max_chunk=500, keep_fields=True, tuning=None,
                  clock=time.perf_counter, prepared=None, pairs=False):
    """Continuous batching.  ``prepared[rid]`` may hold (ux, uy) host arrays
    computed beforehand (input generation kept out of the timed run).

    While a chunk runs on the device the host admits the requests that have
    arrived and fit (creating and initialising their lattices on a stream of
    their own; they join the batch at the next chunk boundary) and reads out
    the solves that finished in the chunk before."""
    reqs = sorted(requests, key=lambda r: r.arrival)
    foot = (lambda d: footprint(d, storage, pairs=True)) if pairs else (lambda d: footprint(d, storage))
    for r in reqs:
        if foot(r.domain) > budget_bytes:
            raise ValueError(f"request {r.rid} needs more device memory than the whole budget")
    new_stream, batch_stream = _streams()
    clk = _Clock(clock)
    rep = Report()
    waiting = []                 # arrived, not admitted
    ready = []                   # admitted and initialised: [request, lattice, remaining, admitted]
    active = []                  # advancing together (the batch, or one lattice alone)
    finished = []                # stepped to the end, not read out yet
    state = {"next": 0, "used": 0}
    batch = None
    batch_members = ()

    def arrivals():
        now = clk.now()
        while state["next"] < len(reqs) and reqs[state["next"]].arrival <= now:
            waiting.append(reqs[state["next"]])
            state["next"] += 1
        # withdrawn requests leave the queue, or the device (at a chunk
        # boundary), and give their memory back
        for r in [r for r in waiting if r.cancelled_by(now)]:
            waiting.remove(r)
            rep.cancelled.append(r.rid)

    refused_at = {}              # rid -> when it first did not fit the budget

    def admit():
        while waiting:
            need = foot(waiting[0].domain)
            if state["used"] + need > budget_bytes:
                rep.memory_waits += 1
                refused_at.setdefault(waiting[0].rid, clk.now())
                break
            r = waiting.pop(0)
            if r.rid in refused_at:
                rep.memory_wait_s += clk.now() - refused_at.pop(r.rid)
            u0 = prepared.get(r.rid) if prepared else None
            ready.append([r, _lattice(r.domain, storage, u0, stream=new_stream()), r.steps, clk.now()])
            state["used"] += need
            rep.peak_bytes = max(rep.peak_bytes, state["used"])

    def read_out():
        for r, lat, _, admitted in finished:
            res = Result(r.rid, r.arrival, admitted, 0.0)
            if keep_fields:
                res.ux, res.uy = lat.read("ux"), lat.read("uy")
            else:
                lat.norms("ux")
            res.completed = clk.now()
            rep.results.append(res)
            state["used"] -= foot(r.domain)
            lat.close()
        finished.clear()

    while state["next"] < len(reqs) or waiting or ready or active or finished:
        arrivals()
        now = clk.now()
        for group in (ready, active):
            for a in [a for a in group if a[0].cancelled_by(now)]:
                group.remove(a)
                a[1].close()
                state["used"] -= foot(a[0].domain)
                rep.cancelled.append(a[0].rid)
        admit()
        active.extend(ready)
        ready.clear()
        rep.max_active = max(rep.max_active, len(active))
        if not active:
            read_out()
            if batch is not None:  # the last members were withdrawn
                batch.close()
                batch, batch_members = None, ()
            if state["next"] < len(reqs) and not waiting:
                clk.wait_until(reqs[state["next"]].arrival)
            continue
        members = tuple(id(a[1]) for a in active)
        if members != batch_members:
            if batch is not None:
                batch.close()
                batch = None
            if len(active) > 1:
                batch = lbps.Batch([a[1] for a in active], stream=batch_stream)
                if tuning is not None:
                    batch.set_tuning(*tuning)
                if pairs and all(pairs_apply(a[0].domain) for a in active):
                    batch.set_step_pairs(True)
                rep.rebuilds += 1
            elif pairs:
                # alone: two steps per sweep only where they pay on one lattice
                d = active[0][0].domain
                lbps.lbps_set_step_pairs(active[0][1]._h,
                                         int(pairs_apply(d) and d.nx * d.ny >= lbps.PAIRS_AUTO_POINTS))
            batch_members = members
        k = min(max_chunk, min(a[2] for a in active))
        if batch is not None:
            batch.step(k)
        else:  # alone on the device: the single-lattice path
            rc = lbps.lbps_step_async(active[0][1]._h, k)
            if rc != lbps.LBPS_OK:
                raise lbps.LbpsError(rc, "serve: lone step")
        # host work while the chunk runs: results of the previous chunk, new arrivals
        read_out()
        arrivals()
        admit()
        rc = batch.check() if batch is not None else lbps.lbps_check(active[0][1]._h)  # waits for the chunk
        if rc != lbps.LBPS_OK:
            raise lbps.LbpsError(rc, "serve: chunk check")
        rep.chunks += 1
        for a in active:
            a[2] -= k
        done = [a for a in active if a[2] == 0]
        if done:
            finished.extend(done)
            active = [a for a in active if a[2] > 0]
            if not active and not ready and not waiting:
                read_out()       # nothing to overlap with
    if batch is not None:
        batch.close()
    rep.makespan = clk.now()
    rep.results.sort(key=lambda r: r.rid)
    return rep


def serve_one_at_a_time(requests, storage="f32", keep_fields=True, clock=time.perf_counter, prepared=None):
    """Baseline: one solve at a time, in arrival order, with lbps_step.  A
    request withdrawn before its turn is skipped; one running is not
    interrupted (lbps_step runs it to the end)."""
    reqs = sorted(requests, key=lambda r: r.arrival)
    clk = _Clock(clock)
    rep = Report()
    for r in reqs:
        clk.wait_until(r.arrival)
        if r.cancelled_by(clk.now()):
            rep.cancelled.append(r.rid)
            continue
        admitted = clk.now()
        u0 = prepared.get(r.rid) if prepared else None
        lat = _lattice(r.domain, storage, u0)
        lat.step(r.steps)
        res = Result(r.rid, r.arrival, admitted, 0.0)
        if keep_fields:
            res.ux, res.uy = lat.read("ux"), lat.read("uy")
        else:
            lat.norms("ux")
        res.completed = clk.now()
        rep.results.append(res)
        rep.chunks += 1
        lat.close()
    rep.makespan = clk.now()
    rep.max_active = 1
    rep.results.sort(key=lambda r: r.rid)
    return rep
