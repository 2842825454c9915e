"""Continuous-batching server for advance-k-steps requests.

Each request is an independent block set (its own mesh, size, block edge,
precision and initial state) that must be advanced k steps.  The server keeps
every admitted request's state resident on the device and steps all of them
together through one ``fx_batch`` (one replayed CUDA graph per step).  It
admits waiting requests, in arrival order, whenever a batch slot and enough
of the device-memory budget are free, so requests that arrive while others
are on the GPU join at the next step boundary and their work overlaps.
Latency of a request = completion time - arrival time.

``serve_per_request`` is the plain baseline: one request at a time, in
arrival order, each stepped alone in FP64 with ``fx_step``.

The request stream follows the serving configuration: Poisson arrivals,
log-uniform block counts, block edges 8/16/32, k in 1..20, setups drawn from
the Sod/KH/Sedov/advection initial states, half FP64 and half FP32-bulk.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import fx, inputs

SETUPS = ("sod", "kh", "sedov", "advection")


@dataclass
class Request:
    rid: int
    setup: str
    nblocks: int
    nxb: int
    precision: int
    k: int
    arrival: float
    admitted: float | None = None
    done: float | None = None
    zones: int = 0
    status: int = 0
    extra: dict = field(default_factory=dict)


def _factor(nb: int, parts: int):
    """``parts`` integers whose product is ``nb``, as balanced as possible."""
    dims = [1] * parts
    rest = nb
    p = 2
    primes = []
    while p * p <= rest:
        while rest % p == 0:
            primes.append(p)
            rest //= p
        p += 1
    if rest > 1:
        primes.append(rest)
    for q in sorted(primes, reverse=True):
        i = int(np.argmin(dims))
        dims[i] *= q
    return tuple(sorted(dims, reverse=True))


def make_stream(n: int, rate: float, seed: int = 11630, blocks=(8, 4096), nxbs=(8, 16, 32),
                ksteps=(1, 20), setups=SETUPS, f32_frac: float = 0.5):
    """Poisson arrivals at ``rate`` requests/s (``rate`` = inf: all at t = 0)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        if math.isfinite(rate):
            t += rng.exponential(1.0 / rate)
        nb = int(round(math.exp(rng.uniform(math.log(blocks[0]), math.log(blocks[1])))))
        nxb = int(rng.choice(nxbs))
        k = int(rng.integers(ksteps[0], ksteps[1] + 1))
        setup = str(rng.choice(setups))
        prec = fx.FX_F32BULK if rng.random() < f32_frac else fx.FX_F64
        out.append(Request(i, setup, nb, nxb, prec, k, t if math.isfinite(rate) else 0.0))
    return out


def with_arrivals(reqs, rate: float, seed: int = 11630):
    """The same requests with new Poisson arrival times at ``rate``."""
    rng = np.random.default_rng(seed + 1)
    t = 0.0
    out = []
    for r in reqs:
        if math.isfinite(rate):
            t += rng.exponential(1.0 / rate)
        out.append(Request(r.rid, r.setup, r.nblocks, r.nxb, r.precision, r.k,
                           t if math.isfinite(rate) else 0.0))
    return out


def request_problem(req: Request):
    """Mesh and primitive initial state of a request (seeded, synthetic)."""
    n = req.nxb
    ng = 4
    if req.setup == "sod":
        dims = _factor(req.nblocks, 2)
        mesh = inputs.uniform_mesh(2, dims, n, ng, inputs.OUTFLOW)
        return mesh, inputs.sod_state(mesh)
    if req.setup == "kh":
        mesh = inputs.uniform_mesh(3, _factor(req.nblocks, 3), n, ng, inputs.PERIODIC)
        return mesh, inputs.kh_state(mesh)
    if req.setup == "advection":
        mesh = inputs.uniform_mesh(3, _factor(req.nblocks, 3), n, ng, inputs.PERIODIC)
        return mesh, inputs.advection_state(mesh)
    # sedov: coarse c^3 blocks with the central (c/2)^3 refined (~2 c^3 blocks)
    c = max(2, 2 * int(round(0.5 * (req.nblocks / 2.0) ** (1.0 / 3.0))))
    base = inputs.uniform_mesh(3, (c, c, c), n, ng, inputs.OUTFLOW)
    lo = c // 4
    flags = []
    for b in range(base.nb):
        bc = base.origin[b] // n
        flags.append(all(lo <= bc[d] < lo + c // 2 for d in range(3)))
    mesh = inputs.refine(base, np.array(flags))
    return mesh, inputs.sedov_state(mesh)


def state_bytes(mesh, precision: int) -> int:
    el = 8 if precision == fx.FX_F64 else 4
    return 2 * mesh.nb * mesh.nvar * mesh.PZ * mesh.P * mesh.P * el


def prepare(reqs, pinned: bool = True):
    """Build every request's mesh and initial state on the host (the client's
    side of the protocol), before the clock starts.  With ``pinned`` the
    states are held in page-locked host memory, so that admitting a request
    is an asynchronous copy rather than a staged one."""
    out = {}
    for r in reqs:
        mesh, W = request_problem(r)
        if pinned:
            import torch
            W = torch.from_numpy(np.ascontiguousarray(W, dtype=np.float64)).pin_memory()
        out[r.rid] = (mesh, W)
    return out


def _percentiles(reqs):
    lat = np.array([r.done - r.arrival for r in reqs])
    return float(np.percentile(lat, 50)), float(np.percentile(lat, 99)), float(lat.max())


def serve(reqs, problems, budget_bytes: float = 120e9, max_slots: int = 256, cfl: float = 0.8,
          tune: bool = True, realtime: bool = True, keep=(), f64_arith: int = 0):
    """Continuous batching.  Returns a stats dict; fills admitted/done/zones.
    Requests whose rid is in ``keep`` get their final state (host copy) in
    ``req.extra["state"]``.  ``f64_arith`` = 1 updates the FP64 requests in
    double-word arithmetic (fx_set_option "f64_arith")."""
    import torch
    ctx = fx.fx_init(1.4, 16, 4)
    if f64_arith:
        fx.fx_set_option(ctx, "f64_arith", f64_arith)
    batch = fx.Batch(ctx, max_slots)
    pending = deque(sorted(reqs, key=lambda r: r.arrival))
    active = {}
    rem = {}          # slot -> steps the request still needs (host view)
    step_s = 0.0      # running estimate of one batched step's wall time
    syncs = 0
    used = 0
    max_used = 0
    max_active = 0
    steps = 0
    tuned = not tune
    t0 = time.perf_counter()
    try:
        while pending or active:
            now = time.perf_counter() - t0
            added = False
            while pending and pending[0].arrival <= now and len(active) < max_slots:
                req = pending[0]
                mesh, W = problems[req.rid]
                need = state_bytes(mesh, req.precision)
                if used + need > budget_bytes:
                    if not active and need > budget_bytes:
                        raise ValueError(f"request {req.rid} needs more than the budget")
                    break                       # wait for memory to free up
                pending.popleft()
                bs = fx.BlockSet(mesh, 1.4, precision=req.precision, ctx=ctx)
                bs.set_primitive(W)
                slot = batch.add(bs, cfl, req.k)
                rem[slot] = req.k
                req.admitted = time.perf_counter() - t0
                req.zones = mesh.leaf_zones() * req.k
                active[slot] = (req, bs, need)
                used += need
                max_used = max(max_used, used)
                max_active = max(max_active, len(active))
                added = True
            if not active:
                if pending and realtime:
                    time.sleep(max(0.0, min(0.001, pending[0].arrival - now)))
                continue
            if added and not tuned:
                batch.tune()
                tuned = True
            # Steps to run before the host looks again: up to the first
            # completion (the host knows every request's remaining steps), or
            # fewer if a waiting request arrives sooner and could be admitted;
            # one host synchronisation per such run, not per step.
            nrun = min(rem.values())
            if pending and len(active) < max_slots:
                head = pending[0]
                fits = used + state_bytes(problems[head.rid][0], head.precision) <= budget_bytes
                if fits:
                    wait = head.arrival - (time.perf_counter() - t0)
                    nrun = max(1, min(nrun, int(wait / step_s))) if step_s > 0 else 1
            tr = time.perf_counter()
            batch.run(nrun)
            steps += nrun
            left = batch.poll()
            syncs += 1
            dt_run = (time.perf_counter() - tr) / nrun
            step_s = dt_run if step_s == 0.0 else 0.8 * step_s + 0.2 * dt_run
            for sl in rem:
                rem[sl] -= nrun
            for slot in [s for s in active if left[s] == 0]:
                rem.pop(slot)
                req, bs, need = active.pop(slot)
                batch.remove(slot)
                req.status = bs.status()
                req.done = time.perf_counter() - t0
                if req.rid in keep:
                    req.extra["state"] = bs.state()
                bs.close()
                used -= need
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        choices = {f"{nd}d_{name}": batch.choice(nd, pr) for nd in (2, 3)
                   for pr, name in ((0, "f64"), (1, "f32bulk"), (2, "f64_double_word"))}
    finally:
        batch.close()
        fx.fx_finalize(ctx)
    zones = sum(r.zones for r in reqs)
    p50, p99, pmax = _percentiles(reqs)
    return {"requests": len(reqs), "wall_s": wall, "batched_steps": steps, "host_syncs": syncs,
            "zone_updates_per_s": zones / wall, "requests_per_s": len(reqs) / wall,
            "p50_s": p50, "p99_s": p99, "max_s": pmax, "max_used_bytes": max_used,
            "max_concurrent": max_active, "launch_choices": choices,
            "failed": int(sum(1 for r in reqs if r.status != 0))}


def serve_per_request(reqs, problems, cfl: float = 0.8, precision: int | None = fx.FX_F64,
                      realtime: bool = True):
    """Baseline: one request at a time in arrival order, each stepped alone
    (fx_step per step) in ``precision`` (None: the request's own)."""
    import torch
    ctx = fx.fx_init(1.4, 16, 4)
    t0 = time.perf_counter()
    try:
        for req in sorted(reqs, key=lambda r: r.arrival):
            now = time.perf_counter() - t0
            if realtime and req.arrival > now:
                time.sleep(req.arrival - now)
            mesh, W = problems[req.rid]
            prec = req.precision if precision is None else precision
            bs = fx.BlockSet(mesh, 1.4, precision=prec, ctx=ctx)
            bs.set_primitive(W)
            req.admitted = time.perf_counter() - t0
            bs.run(req.k, cfl)
            req.status = bs.status()          # synchronises
            req.done = time.perf_counter() - t0
            req.zones = mesh.leaf_zones() * req.k
            bs.close()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    finally:
        fx.fx_finalize(ctx)
    zones = sum(r.zones for r in reqs)
    p50, p99, pmax = _percentiles(reqs)
    return {"requests": len(reqs), "wall_s": wall, "zone_updates_per_s": zones / wall,
            "requests_per_s": len(reqs) / wall, "p50_s": p50, "p99_s": p99, "max_s": pmax,
            "failed": int(sum(1 for r in reqs if r.status != 0))}
