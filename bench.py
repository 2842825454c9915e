"""Benchmark of the block-AMR Euler hot path on GB300.

One step = dt max-reduction + coarse-fine guard fill + fused MUSCL-Hancock/
HLLC update that reads same-level neighbours directly (+ flux correction and
restriction on AMR meshes) of the whole block set, through the C ABI (libfx),
i.e. exactly fx_step.  Default workload: the 3D Kelvin-Helmholtz
shear layer, 256^3 cells as 4096 blocks of 16^3 (+4 guard cells), periodic,
FP64 -- the configuration the zone-updates/s metric is quoted on.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload instead.

Multi-GPU (torchrun, one rank per GPU): every rank advances its own
independent replica of the workload (no data-path collective); value is the
sum of zones over ranks divided by the slowest rank's time (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "zone-updates/s"
UNIT = "zone-updates/s"
HBM_BYTES_PER_ZONE = {"f64": 80.0, "f32bulk": 40.0}
# FP64 arithmetic per zone update (each +, -, *, / and sqrt = 1): one
# primitive conversion, one cell's slopes/predictor/face states, ndim HLLC
# face fluxes, one conservative update and one CFL signal speed, counted on
# the oracle's op-counting build ("python -m oracle.opcount <workload> 4 10",
# one full step after 10).  The HLLC branch mix,
# and with it the count, depends a little on the flow.
ALGO_FLOPS_PER_ZONE = {"kh3d": 619.9, "sedov_amr": 597.2, "advection3d": 602.3,
                       "sod2d": 411.8}
# FP64 peak: 152 SMs x 2 DFMA/clk/SM x 2 flop x 2.07 GHz.
FP64_PEAK_FLOPS = 152 * 2 * 2 * 2.07e9
# DRAM bytes (read + written) per zone of the update kernel, from one ncu
# capture of the 128^3 KH case (dram__bytes_read.sum + dram__bytes_write.sum
# over 2,097,152 zones); the full launch's traffic scales with its zones.
# Valid for the kernel build those counters were taken on.
TRAFFIC_BYTES_PER_ZONE = {"f64": 101.3, "f32bulk": 66.6}


def measure_fma_peak(fx, stream, precision, reps: int = 3):
    """FMA-pipe throughput (flop/s) of this GPU now: the library's probe
    kernel (independent FMA chains on every SM), best of `reps` launches timed
    with CUDA events on `stream`."""
    import torch
    nsm = torch.cuda.get_device_properties(stream.device).multi_processor_count
    ctas = nsm * 8
    dtype = torch.float64 if precision == fx.FX_F64 else torch.float32
    out = torch.empty(ctas, dtype=dtype, device=stream.device)
    iters = 4000 if precision == fx.FX_F64 else 100000
    best = 0.0
    with torch.cuda.stream(stream):
        fx.fx_fma_probe(precision, ctas, 64, out.data_ptr(), stream)   # warm-up
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            flops = fx.fx_fma_probe(precision, ctas, iters, out.data_ptr(), stream)
            b.record(stream)
            stream.synchronize()
            best = max(best, flops / (a.elapsed_time(b) / 1e3))
    return best


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------------------
# distributed helpers (also exercised by the gloo CPU tests)
# ---------------------------------------------------------------------------

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(zones_local: float, seconds_local: float, device=None):
    """Whole-job throughput: sum of zones over ranks / max time over ranks."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return zones_local, seconds_local
    z = torch.tensor([zones_local], dtype=torch.float64, device=device)
    t = torch.tensor([seconds_local], dtype=torch.float64, device=device)
    dist.all_reduce(z, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(z.item()), float(t.item())


def link_bandwidth(host_in, host_out, stream, reps: int = 3):
    """Host->device and device->host GB/s of one copy of a pinned buffer
    (CUDA events on `stream`, median of `reps` after one warm-up copy)."""
    import torch
    dbuf = torch.empty(host_in.shape, dtype=host_in.dtype, device=stream.device)
    nbytes = host_in.numel() * host_in.element_size()
    out = []
    for copy in (lambda: dbuf.copy_(host_in, non_blocking=True),
                 lambda: host_out.copy_(dbuf, non_blocking=True)):
        ts = []
        with torch.cuda.stream(stream):
            for _ in range(reps + 1):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                copy()
                b.record(stream)
                stream.synchronize()
                ts.append(a.elapsed_time(b) / 1e3)
        out.append(nbytes / float(np.median(ts[1:])) / 1e9)
    del dbuf
    return out[0], out[1]


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-i", str(self.index), "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle baseline
# ---------------------------------------------------------------------------

def oracle_sample(workload: str, target_s: float = 12.0, max_steps: int = 50,
                  single_s: float = 4.0):
    """Time the FP64 oracle, as it is, on a bounded sample of the workload
    (REFERENCE_SAMPLE_SCALE: the same block size, physics and boundaries on
    fewer blocks), full steps (dt, guard fill, update) on all host cores, then
    for about ``single_s`` seconds on one thread."""
    import oracle
    from paper_2208_11630_gb300 import inputs
    mesh, W, _, _ = inputs.workload(workload, scale=REFERENCE_SAMPLE_SCALE.get(workload))
    desc = (f"FP64 CPU oracle on {workload_name(workload, mesh)} ({mesh.nb} blocks of "
            f"{mesh.nxb}^{mesh.ndim} + {mesh.ng} guard), the same workload at a bounded size")
    om = oracle.OracleMesh(mesh, 1.4)
    U = om.prim_to_cons(W)
    zones = mesh.leaf_zones()

    def timed(budget_s, cap):
        nonlocal U
        t0 = time.perf_counter()
        steps = 0
        while steps < cap:
            U, _ = om.step(U, cfl=0.8)
            steps += 1
            if time.perf_counter() - t0 > budget_s:
                break
        return steps, time.perf_counter() - t0

    cores = oracle.get_threads()
    steps, dt = timed(target_s, max_steps)
    out = {"value": zones * steps / dt, "unit": UNIT, "cores": cores,
           "kind": "oracle", "sample": f"{desc}; {steps} full steps in {dt:.1f} s"}
    oracle.set_threads(1)
    try:
        s1, t1 = timed(single_s, max_steps)
    finally:
        oracle.set_threads(cores)
    out["single_thread"] = {"value": zones * s1 / t1, "unit": UNIT, "cores": 1,
                            "sample": f"the same sample; {s1} full steps in {t1:.1f} s"}
    return out


def measure_variants(args, fx, inputs, mesh, dev, cfl, zones, bs, ws, hbm_peak):
    """The same workload (i) as one request of a batch -- coarse-fine fill,
    update and flux correction replayed as one CUDA graph per step (the
    persistent update, autotuned, or the per-block-set kernels for a request
    that fills the GPU) -- (ii) in the other precision, per call and as a
    batch, (v) as an FP64
    state updated in double-word arithmetic, each timed the same way (CUDA
    events on the launching stream, warm-up first), then (iv) with two
    species and (iii) with regridding."""
    import torch
    out = {}
    stream = torch.cuda.Stream(device=dev)
    sptr = stream.cuda_stream
    # (i) batched + graph
    ctx = fx.fx_init(1.4, mesh.nxb, mesh.ng)
    batch = fx.Batch(ctx, 1)
    slot = batch.add(bs, cfl, args.warmup + args.steps, stream=sptr)
    tuning = batch.tune(stream=sptr)
    batch.run(args.warmup, stream=sptr)
    stream.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    batch.run(args.steps, stream=sptr)
    b.record(stream)
    torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 1e3
    path = batch.path(slot)
    batch.remove(slot, stream=sptr)
    ok = bs.status() == 0
    tile, ctas = batch.choice(mesh.ndim, bs.precision)
    batch.close()
    fx.fx_finalize(ctx)
    z, t = aggregate(zones * args.steps, sec, dev)
    out["batched_graph"] = {"value": z / t, "unit": UNIT, "ms_per_step": 1e3 * t / args.steps,
                            "path": BATCH_PATHS[path], "tile": tile, "ctas_per_sm": ctas,
                            "tuning_us": tuning, "ok": ok}
    # (ii) the other precision, plain per-call path
    other = "f32bulk" if args.precision == "f64" else "f64"
    prec = fx.FX_F32BULK if other == "f32bulk" else fx.FX_F64
    mesh2, W, gamma, _ = inputs.workload(args.workload, scale=args.scale)
    bs2 = fx.BlockSet(mesh2, gamma, precision=prec, device=dev)
    bs2.set_primitive(W)
    del W
    dtp = bs2.dt.data_ptr()
    for _ in range(args.warmup):
        fx.fx_step(bs2.ctx, bs2.bs, cfl, dtp, sptr)
    stream.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    a.record(stream)
    for k in range(args.steps):
        fx.fx_compute_dt(bs2.ctx, bs2.bs, cfl, dtp, sptr)
        fx.fx_guardcell_fill_amr(bs2.ctx, bs2.bs, sptr)
        ev[k][0].record(stream)
        fx.fx_hydro_advance(bs2.ctx, bs2.bs, dtp, sptr)
        ev[k][1].record(stream)
    b.record(stream)
    torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 1e3
    hyd = float(np.mean([x.elapsed_time(y) for x, y in ev])) / 1e3
    z, t = aggregate(zones * args.steps, sec, dev)
    bpz = HBM_BYTES_PER_ZONE[other]
    ok2 = bs2.status() == 0
    # the same as one request of a batch (continuing from this state)
    gsec, gtile, gctas, gpath = timed_batch(fx, bs2, cfl, stream, args.warmup, args.steps,
                                            mesh2.nxb, mesh2.ng)
    gz, gt = aggregate(zones * args.steps, gsec, dev)
    out[other] = {"value": z / t, "unit": UNIT, "ms_per_step": 1e3 * t / args.steps,
                  "dtype": "f32" if other == "f32bulk" else "f64", "hydro_ms": hyd * 1e3,
                  "hydro_hbm_frac": bpz * zones / hyd / (hbm_peak * 1e9),
                  "step_hbm_frac": bpz * (z / t) / ws / (hbm_peak * 1e9),
                  "batched_graph": {"value": gz / gt, "ms_per_step": 1e3 * gt / args.steps,
                                    "path": BATCH_PATHS[gpath], "tile": gtile,
                                    "ctas_per_sm": gctas},
                  "ok": ok2 and bs2.status() == 0}
    bs2.close()
    # (v) FP64 state updated in double-word arithmetic (option f64_arith = 1):
    # timed like (ii); its deviation from the FP64 update after one step from
    # the same state, per cell relative to the variable's largest magnitude
    # (the momentum components share the largest |m|)
    mesh5, W5s, gamma5, _ = inputs.workload(args.workload, scale=args.scale)
    bs5 = fx.BlockSet(mesh5, gamma5, precision=fx.FX_F64, device=dev, options={"f64_arith": 1})
    bs5.set_primitive(W5s)
    ref5 = fx.BlockSet(mesh5, gamma5, precision=fx.FX_F64, device=dev)
    ref5.set_primitive(W5s)
    del W5s
    fx.fx_step(bs5.ctx, bs5.bs, cfl, bs5.dt.data_ptr(), sptr)
    fx.fx_step(ref5.ctx, ref5.bs, cfl, ref5.dt.data_ptr(), sptr)
    torch.cuda.synchronize()
    g5 = mesh5.ng
    sl = (slice(None), slice(None)) + ((slice(g5, g5 + mesh5.nxb),) if mesh5.ndim == 3 else
                                       (slice(None),)) + (slice(g5, g5 + mesh5.nxb),) * 2
    leaf5 = torch.as_tensor(mesh5.is_leaf().astype(bool), device=bs5.current.device)
    a5, r5 = bs5.current[sl][leaf5], ref5.current[sl][leaf5]
    scale5 = r5.abs().amax(dim=(0, 2, 3, 4), keepdim=True)
    scale5[:, 1:4] = r5[:, 1:4].square().sum(dim=1).sqrt().amax()
    scale5 = scale5.clamp_min(1e-300)
    dev5 = float(((a5 - r5).abs() / torch.maximum(r5.abs(), scale5)).max())
    del a5, r5
    ref5.close()
    dtp5 = bs5.dt.data_ptr()
    for _ in range(args.warmup):
        fx.fx_step(bs5.ctx, bs5.bs, cfl, dtp5, sptr)
    stream.synchronize()
    ev5 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    a.record(stream)
    for k in range(args.steps):
        fx.fx_compute_dt(bs5.ctx, bs5.bs, cfl, dtp5, sptr)
        fx.fx_guardcell_fill_amr(bs5.ctx, bs5.bs, sptr)
        ev5[k][0].record(stream)
        fx.fx_hydro_advance(bs5.ctx, bs5.bs, dtp5, sptr)
        ev5[k][1].record(stream)
    b.record(stream)
    torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 1e3
    hyd5 = float(np.mean([x.elapsed_time(y) for x, y in ev5])) / 1e3
    z, t = aggregate(zones * args.steps, sec, dev)
    eq5 = ALGO_FLOPS_PER_ZONE[args.workload] * zones / hyd5
    out["f64_double_word"] = {
        "value": z / t, "unit": UNIT, "ms_per_step": 1e3 * t / args.steps, "dtype": "f64 state, "
        "double-word (2 x f32) arithmetic", "hydro_ms": hyd5 * 1e3,
        "fp64_equivalent_tflops": eq5 / 1e12,
        "fp64_equivalent_frac_of_fp64_peak": eq5 / FP64_PEAK_FLOPS,
        "note": f"the scheme's {ALGO_FLOPS_PER_ZONE[args.workload]} FP64 flops per zone update, "
                "computed on the FP32 pipe",
        "max_rel_dev_from_f64_after_one_step": dev5, "ok": bs5.status() == 0}
    bs5.close()
    # (vi) the other FP32 reading: FP64 state (80 B/zone), FP32 arithmetic,
    # FP64 accumulation of the update (option f64_arith = 2); timed like (ii),
    # with its deviation from the FP64 update after one step
    mesh6, W6, gamma6, _ = inputs.workload(args.workload, scale=args.scale)
    bs6 = fx.BlockSet(mesh6, gamma6, precision=fx.FX_F64, device=dev, options={"f64_arith": 2})
    bs6.set_primitive(W6)
    ref6 = fx.BlockSet(mesh6, gamma6, precision=fx.FX_F64, device=dev)
    ref6.set_primitive(W6)
    del W6
    fx.fx_step(bs6.ctx, bs6.bs, cfl, bs6.dt.data_ptr(), sptr)
    fx.fx_step(ref6.ctx, ref6.bs, cfl, ref6.dt.data_ptr(), sptr)
    torch.cuda.synchronize()
    a6, r6 = bs6.current[sl][leaf5], ref6.current[sl][leaf5]
    scale6 = r6.abs().amax(dim=(0, 2, 3, 4), keepdim=True)
    scale6[:, 1:4] = r6[:, 1:4].square().sum(dim=1).sqrt().amax()
    dev6 = float(((a6 - r6).abs() / torch.maximum(r6.abs(), scale6.clamp_min(1e-300))).max())
    del a6, r6
    ref6.close()
    dtp6 = bs6.dt.data_ptr()
    for _ in range(args.warmup):
        fx.fx_step(bs6.ctx, bs6.bs, cfl, dtp6, sptr)
    stream.synchronize()
    ev6 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    a.record(stream)
    for k in range(args.steps):
        fx.fx_compute_dt(bs6.ctx, bs6.bs, cfl, dtp6, sptr)
        fx.fx_guardcell_fill_amr(bs6.ctx, bs6.bs, sptr)
        ev6[k][0].record(stream)
        fx.fx_hydro_advance(bs6.ctx, bs6.bs, dtp6, sptr)
        ev6[k][1].record(stream)
    b.record(stream)
    torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 1e3
    hyd6 = float(np.mean([x.elapsed_time(y) for x, y in ev6])) / 1e3
    z, t = aggregate(zones * args.steps, sec, dev)
    out["f64_state_f32_arith"] = {
        "value": z / t, "unit": UNIT, "ms_per_step": 1e3 * t / args.steps,
        "dtype": "f64 state, f32 arithmetic, f64 update accumulation", "hydro_ms": hyd6 * 1e3,
        "hydro_hbm_frac": HBM_BYTES_PER_ZONE["f64"] * zones / hyd6 / (hbm_peak * 1e9),
        "algorithmic_bytes_per_zone": HBM_BYTES_PER_ZONE["f64"],
        "max_rel_dev_from_f64_after_one_step": dev6, "ok": bs6.status() == 0}
    bs6.close()
    # (iv) multispecies perfect gas: the same workload carrying two species
    # (gamma 1.4 / A 28.96 inside the shear band, 5/3 / 4 outside)
    import dataclasses
    mesh4 = dataclasses.replace(mesh2, species=((1.4, 28.96), (5.0 / 3.0, 4.0)))
    W4 = np.zeros(mesh4.shape)
    _, W5, _, _ = inputs.workload(args.workload, scale=args.scale)
    W4[:, :5] = W5[:, :5]
    del W5
    g4, n4 = mesh4.ng, mesh4.nxb
    for b4 in range(mesh4.nb):
        _, y4, _ = mesh4.cell_centers(b4)
        inner = (np.abs(y4 - 0.5) < 0.25).astype(np.float64) * np.ones(
            (n4 if mesh4.ndim == 3 else 1, n4, n4))
        if mesh4.ndim == 3:
            W4[b4, 5, g4:g4 + n4, g4:g4 + n4, g4:g4 + n4] = inner
            W4[b4, 6, g4:g4 + n4, g4:g4 + n4, g4:g4 + n4] = 1.0 - inner
        else:
            W4[b4, 5, 0, g4:g4 + n4, g4:g4 + n4] = inner[0]
            W4[b4, 6, 0, g4:g4 + n4, g4:g4 + n4] = 1.0 - inner[0]
    # FP64 arithmetic, then the same in double-word arithmetic (f64_arith = 1)
    for key4, opts4 in (("multispecies_2", None), ("multispecies_2_double_word", {"f64_arith": 1})):
        bs4 = fx.BlockSet(mesh4, gamma, precision=fx.FX_F64, device=dev, options=opts4)
        bs4.set_primitive(W4)
        dtp4 = bs4.dt.data_ptr()
        for _ in range(args.warmup):
            fx.fx_step(bs4.ctx, bs4.bs, cfl, dtp4, sptr)
        stream.synchronize()
        ev4 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        a.record(stream)
        for k in range(args.steps):
            fx.fx_compute_dt(bs4.ctx, bs4.bs, cfl, dtp4, sptr)
            fx.fx_guardcell_fill_amr(bs4.ctx, bs4.bs, sptr)
            ev4[k][0].record(stream)
            fx.fx_hydro_advance(bs4.ctx, bs4.bs, dtp4, sptr)
            ev4[k][1].record(stream)
        b.record(stream)
        torch.cuda.synchronize()
        sec = a.elapsed_time(b) / 1e3
        hyd4 = float(np.mean([x.elapsed_time(y) for x, y in ev4])) / 1e3
        z, t = aggregate(zones * args.steps, sec, dev)
        out[key4] = {"value": z / t, "unit": UNIT, "ms_per_step": 1e3 * t / args.steps,
                     "dtype": "f64" if opts4 is None else "f64 state, double-word (2 x f32) arithmetic",
                     "nspec": 2, "hydro_ms": hyd4 * 1e3, "ok": bs4.status() == 0}
        bs4.close()
    del W4
    # (iii) dynamic AMR: the Sedov blast on its 2-level mesh, regridded every
    # 4 steps (Loehner indicator on density and pressure, up to level 2);
    # wall-clock time between synchronisations, since the plan runs on the host
    meshs, Ws, gammas, _ = inputs.workload("sedov_amr", scale=None)
    bs3 = fx.BlockSet(meshs, gammas, precision=fx.FX_F64, device=dev)
    bs3.set_primitive(Ws)
    del Ws
    nsteps = max(8, args.steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    zones_done, regrid_s, nregrid = 0, 0.0, 0
    for k in range(nsteps):
        if k % 4 == 0:
            torch.cuda.synchronize()
            r0 = time.perf_counter()
            bs3.regrid(refine_cutoff=0.8, derefine_cutoff=0.2, filt=0.01, max_level=2,
                       stream=sptr)
            regrid_s += time.perf_counter() - r0
            nregrid += 1
        fx.fx_step(bs3.ctx, bs3.bs, cfl, bs3.dt.data_ptr(), sptr)
        zones_done += bs3.mesh.leaf_zones()
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    z, t = aggregate(zones_done, sec, dev)
    out["dynamic_amr_sedov"] = {
        "value": z / t, "unit": UNIT, "steps": nsteps, "regrid_every": 4,
        "regrid_ms": 1e3 * regrid_s / nregrid, "blocks": int(bs3.mesh.nb),
        "levels": np.bincount(bs3.mesh.level).tolist(), "timing": "wall clock",
        "ok": bs3.status() == 0}
    bs3.close()
    return out


def timed_steps(fx, bs, cfl, stream, warmup, steps):
    """Device time of `steps` full steps of block set `bs` on `stream` (dt,
    coarse-fine fill, update = fx_step), after `warmup` untimed ones; returns
    (seconds of the steps, mean seconds of one update launch), CUDA events."""
    import torch
    sptr = stream.cuda_stream
    dtp = bs.dt.data_ptr()
    for _ in range(warmup):
        fx.fx_step(bs.ctx, bs.bs, cfl, dtp, sptr)
    stream.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for k in range(steps):
        fx.fx_compute_dt(bs.ctx, bs.bs, cfl, dtp, sptr)
        fx.fx_guardcell_fill_amr(bs.ctx, bs.bs, sptr)
        ev[k][0].record(stream)
        fx.fx_hydro_advance(bs.ctx, bs.bs, dtp, sptr)
        ev[k][1].record(stream)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3, float(np.mean([x.elapsed_time(y) for x, y in ev])) / 1e3


BATCH_PATHS = {0: "batched phases and the persistent update kernel (autotuned), one CUDA graph per step",
               1: "the per-block-set kernels on a branch of one CUDA graph per step (the request fills the GPU)"}


def timed_batch(fx, bs, cfl, stream, warmup, steps, nxb, ng):
    """The same as one request of a batch: coarse-fine fill, update and flux
    correction replayed as one CUDA graph per step (the persistent update with
    its launch choice autotuned, or the per-block-set kernels for a request
    that fills the GPU); returns (seconds of the `steps` timed steps, tile,
    CTAs/SM, path)."""
    import torch
    sptr = stream.cuda_stream
    ctx = fx.fx_init(1.4, nxb, ng)
    batch = fx.Batch(ctx, 1)
    try:
        slot = batch.add(bs, cfl, warmup + steps, stream=sptr)
        batch.tune(stream=sptr)
        batch.run(warmup, stream=sptr)
        stream.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        batch.run(steps, stream=sptr)
        b.record(stream)
        torch.cuda.synchronize()
        path = batch.path(slot)
        batch.remove(slot, stream=sptr)
        tile, ctas = batch.choice(bs.mesh.ndim, bs.precision)
    finally:
        batch.close()
        fx.fx_finalize(ctx)
    return a.elapsed_time(b) / 1e3, tile, ctas, path


def measure_configs(args, fx, inputs, dev, hbm_peak):
    """The other workloads of the benchmark plan, each timed on the device:
    the 2D Sod tube (50 steps, FP64 and FP32-bulk, per call and as a
    graph-replayed batch), the 3D Sedov blast on its two-level octree as a
    graph-replayed batch of one request (20 warm-up + 100 timed steps; FP64
    and FP32-bulk, and the per-call path beside it), and
    smooth advection at 512^3 (FP64 and FP32-bulk)."""
    import torch
    stream = torch.cuda.Stream(device=dev)
    out = {}
    for prec_name, prec in (("f64", fx.FX_F64), ("f32bulk", fx.FX_F32BULK)):
        bpz = HBM_BYTES_PER_ZONE[prec_name]
        # 2D Sod: 128^2 as 8 x 8 blocks of 16^2, 50 steps (state 1.3 MB: L2-resident)
        mesh, W, gamma, cfl = inputs.workload("sod2d")
        zones = mesh.leaf_zones()
        bs = fx.BlockSet(mesh, gamma, precision=prec, device=dev)
        bs.set_primitive(W)
        sec, hyd = timed_steps(fx, bs, cfl, stream, 5, 50)
        ok = bs.status() == 0
        bs.set_primitive(W)
        gsec, tile, ctas, path = timed_batch(fx, bs, cfl, stream, 5, 50, mesh.nxb, mesh.ng)
        out[f"sod2d_128^2_{prec_name}"] = {
            "value": zones * 50 / sec, "unit": UNIT, "ms_per_step": 1e3 * sec / 50,
            "hydro_ms": hyd * 1e3, "batched_graph": {"value": zones * 50 / gsec,
                                                     "ms_per_step": 1e3 * gsec / 50,
                                                     "tile": tile, "ctas_per_sm": ctas,
                                                     "path": BATCH_PATHS[path]},
            "steps": 50, "note": "1.3 MB state: L2-resident, launch-latency bound",
            "ok": ok and bs.status() == 0}
        bs.close()
        # 3D Sedov on the 2-level octree (1408 leaves of 16^3): batched graph,
        # 20 warm-up + 100 timed steps, and the per-call path
        mesh, W, gamma, cfl = inputs.workload("sedov_amr")
        zones = mesh.leaf_zones()
        bs = fx.BlockSet(mesh, gamma, precision=prec, device=dev)
        bs.set_primitive(W)
        gsec, tile, ctas, path = timed_batch(fx, bs, cfl, stream, 20, 100, mesh.nxb, mesh.ng)
        ok = bs.status() == 0
        bs.set_primitive(W)
        sec, hyd = timed_steps(fx, bs, cfl, stream, 20, 100)
        entry = {"value": zones * 100 / gsec, "unit": UNIT, "ms_per_step": 1e3 * gsec / 100,
                 "path": "batch of one request: " + BATCH_PATHS[path],
                 "tile": tile, "ctas_per_sm": ctas, "warmup": 20, "steps": 100,
                 "per_call": {"value": zones * 100 / sec, "ms_per_step": 1e3 * sec / 100,
                              "hydro_ms": hyd * 1e3},
                 "ok": ok and bs.status() == 0}
        if prec_name == "f64":
            entry["hydro_alu_frac_per_call"] = (ALGO_FLOPS_PER_ZONE["sedov_amr"] * zones / hyd
                                                / FP64_PEAK_FLOPS)
        else:
            entry["hydro_hbm_frac_per_call"] = bpz * zones / hyd / (hbm_peak * 1e9)
        out[f"sedov_amr_128^3_2level_{prec_name}"] = entry
        bs.close()
        del W
    # smooth advection 512^3 (32768 blocks of 16^3): 18 GB per FP64 buffer
    mesh, W, gamma, cfl = inputs.workload("advection3d")
    zones = mesh.leaf_zones()
    for prec_name, prec in (("f64", fx.FX_F64), ("f32bulk", fx.FX_F32BULK)):
        bs = fx.BlockSet(mesh, gamma, precision=prec, device=dev)
        bs.set_primitive(W)
        torch.cuda.empty_cache()
        sec, hyd = timed_steps(fx, bs, cfl, stream, 3, 10)
        bpz = HBM_BYTES_PER_ZONE[prec_name]
        entry = {"value": zones * 10 / sec, "unit": UNIT, "ms_per_step": 1e3 * sec / 10,
                 "hydro_ms": hyd * 1e3, "steps": 10,
                 "hydro_hbm_frac": bpz * zones / hyd / (hbm_peak * 1e9), "ok": bs.status() == 0}
        if prec_name == "f64":
            entry["hydro_alu_frac"] = ALGO_FLOPS_PER_ZONE["advection3d"] * zones / hyd / FP64_PEAK_FLOPS
        out[f"advection3d_512^3_{prec_name}"] = entry
        bs.close()
        torch.cuda.empty_cache()
    del W
    return out


def workload_name(name, mesh):
    edge = mesh.nroot[0] * mesh.nxb
    return {"kh3d": f"kh3d_{edge}^3", "advection3d": f"advection3d_{edge}^3",
            "sod2d": f"sod2d_{edge}^2", "sedov_amr": f"sedov_amr_{edge}^3_base_2level"}.get(name, name)


# bounded sample of each workload that the oracle steps on the host cores
# (blocks per axis of the sample; sod2d runs whole)
REFERENCE_SAMPLE_SCALE = {"kh3d": 4, "advection3d": 4, "sedov_amr": 4, "sod2d": None}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_2208_11630_gb300 import inputs
    oracle.build()
    # the line carries the GPU arm's configuration; the oracle steps a sample
    full = inputs.workload_mesh(args.workload, args.scale)
    mesh, W, gamma, _ = inputs.workload(args.workload, scale=REFERENCE_SAMPLE_SCALE[args.workload])
    om = oracle.OracleMesh(mesh, gamma)
    U = om.prim_to_cons(W)
    zones = mesh.leaf_zones()
    for _ in range(args.warmup):
        U, _ = om.step(U)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U, _ = om.step(U)
    sec = time.perf_counter() - t0
    v = zones * args.steps / sec
    sample = (f"FP64 CPU oracle on {workload_name(args.workload, mesh)} ({mesh.nb} blocks of "
              f"{mesh.nxb}^{mesh.ndim} + {mesh.ng} guard), the same workload at a bounded size; "
              f"each step one full step of that sample; {args.steps} steps")
    line = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, workload_name(args.workload, full), full)
            | {"replicas": 1,
               # what the oracle stepped: a bounded sample of that workload
               "ran": {"workload": workload_name(args.workload, mesh), "blocks": mesh.nb,
                       "cells": mesh.leaf_zones(), "nxb": mesh.nxb, "nguard": mesh.ng,
                       "sample_of": workload_name(args.workload, full)}},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.get_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(args, name, mesh):
    state_bytes = mesh.nb * mesh.nvar * mesh.PZ * mesh.P * mesh.P * (8 if args.precision == "f64" else 4)
    bc = "periodic" if mesh.bc[0][0] == 1 else "outflow"
    return {"workload": name, "blocks": mesh.nb, "leaf_blocks": int(mesh.is_leaf().sum()),
            "nxb": mesh.nxb, "nguard": mesh.ng, "cells": mesh.leaf_zones(), "bc": bc, "cfl": 0.8,
            "precision": args.precision,
            "l2": (f"inputs larger than L2 ({state_bytes / 1e9:.2f} GB per state buffer vs 129 MB L2)"
                   if state_bytes > 129e6 else
                   f"state ({state_bytes / 1e6:.1f} MB) fits in L2: launch-latency workload")}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2208_11630_gb300 import fx, inputs

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    fx.load()

    prec = fx.FX_F64 if args.precision == "f64" else fx.FX_F32BULK
    mesh, W, gamma, cfl = inputs.workload(args.workload, scale=args.scale)
    zones_per_step = mesh.leaf_zones()
    wname = workload_name(args.workload, mesh)
    kname = f"k_hydro<{mesh.ndim},{16 if mesh.nxb % 16 == 0 else 8},{'double' if prec == 0 else 'float'}>"
    bs = fx.BlockSet(mesh, gamma, precision=prec, device=dev)
    bs.set_primitive(W)
    U0 = bs.state()          # host copy of the initial state (for the e2e leg)
    del W
    stream = torch.cuda.Stream(device=dev)
    sptr = stream.cuda_stream
    dtp = bs.dt.data_ptr()

    def step():   # = fx_step: dt, coarse-fine fill, fused update
        fx.fx_compute_dt(bs.ctx, bs.bs, cfl, dtp, sptr)
        fx.fx_guardcell_fill_amr(bs.ctx, bs.bs, sptr)
        fx.fx_hydro_advance(bs.ctx, bs.bs, dtp, sptr)

    for _ in range(args.warmup):
        step()
    stream.synchronize()
    if bs.status() != 0:
        raise RuntimeError("non-physical state during warm-up")

    # ---- device-timed region
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(dev.index)
    clocks.start()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = fx.load().fx_kernel_launches()
    start.record(stream)
    for k in range(args.steps):
        fx.fx_compute_dt(bs.ctx, bs.bs, cfl, dtp, sptr)
        fx.fx_guardcell_fill_amr(bs.ctx, bs.bs, sptr)
        ev[k][0].record(stream)
        fx.fx_hydro_advance(bs.ctx, bs.bs, dtp, sptr)
        ev[k][1].record(stream)
    end.record(stream)
    torch.cuda.synchronize()
    launches = fx.load().fx_kernel_launches() - l0
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    sec = start.elapsed_time(end) / 1e3
    hydro_s = np.mean([a.elapsed_time(b) for a, b in ev]) / 1e3
    if bs.status() != 0:
        raise RuntimeError("non-physical state in the timed region")
    zones_all, sec_max = aggregate(zones_per_step * args.steps, sec, dev)
    value = zones_all / sec_max

    # ---- end-to-end through host buffers (pinned), one step per call: the
    # interior cells go up, one full step runs, the new interior comes back
    e2e = None
    if not args.no_e2e:
        host_in = torch.from_numpy(np.ascontiguousarray(mesh.interior(U0))).to(bs.dtype).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        e2e_steps = max(10, min(args.steps, 30))
        bs.run_host_interior(host_in.numpy(), host_out.numpy(), 1, cfl, stream=sptr)
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            bs.run_host_interior(host_in.numpy(), host_out.numpy(), 1, cfl, stream=sptr)
        e2e_sec = time.perf_counter() - t0
        ez, esec = aggregate(zones_per_step * e2e_steps, e2e_sec, dev)
        state_bytes = host_in.numel() * host_in.element_size()
        e2e = {"value": ez / esec, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
               "d2h_bytes_per_step": state_bytes, "call": "fx_run_host_interior"}
        # the host link alone (one copy of the same bytes each way): the
        # upload cannot overlap the update, whose dt needs the whole state
        h2d, d2h = link_bandwidth(host_in, host_out, stream)
        e2e.update({"link_gbs": {"h2d": h2d, "d2h": d2h},
                    "upload_ms": state_bytes / h2d / 1e6, "ms_per_step": esec / e2e_steps * 1e3})

    peaks, peak_kind = load_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    flops_per_zone = ALGO_FLOPS_PER_ZONE[args.workload]
    achieved_flops = flops_per_zone * zones_per_step / hydro_s
    bpz = HBM_BYTES_PER_ZONE[args.precision]
    if args.precision == "f64":
        pclk = ClockSampler(dev.index)
        pclk.start()
        fp64_meas = measure_fma_peak(fx, stream, fx.FX_F64, reps=10)
        pclk = pclk.stop()
        roof = {"bound": "alu", "kernel": kname,
                "achieved": achieved_flops / 1e12, "peak": FP64_PEAK_FLOPS / 1e12,
                "unit": "TFLOP/s", "frac": achieved_flops / FP64_PEAK_FLOPS,
                "traffic": TRAFFIC_BYTES_PER_ZONE["f64"] * zones_per_step
                if args.workload == "kh3d" else None,
                "peak_kind": "derived FP64 DFMA rate (152 SMs x 2 DFMA/clk x 2.07 GHz)",
                "peak_measured": fp64_meas / 1e12,
                "frac_of_measured": achieved_flops / fp64_meas,
                "peak_measured_kind": "FP64 FMA probe (fx_fma_probe) timed in this run",
                "peak_measured_clocks": pclk,
                "traffic_note": "bytes per launch: ncu DRAM read+write of the 128^3 case scaled by zones",
                "algorithmic_flops_per_zone": flops_per_zone,
                "algorithmic_flops_source": "oracle op-counting build (oracle/opcount.py)"}
    else:
        gbs = bpz * zones_per_step / hydro_s / 1e9
        roof = {"bound": "hbm", "kernel": kname, "achieved": gbs,
                "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                "traffic": TRAFFIC_BYTES_PER_ZONE["f32bulk"] * zones_per_step
                if args.workload == "kh3d" else None,
                "peak_kind": peak_kind, "algorithmic_bytes_per_zone": bpz}
    roof.update({"hydro_ms": hydro_s * 1e3,
                 "hbm_frac_of_step": (bpz * value / ws) / (hbm_peak * 1e9),
                 "hbm_peak_gbs": hbm_peak, "hbm_peak_kind": peak_kind})
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sec_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "f64" else "f32",
        "data": "synthetic",
        "config": workload_config(args, wname, mesh) | {"replicas": ws},
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if not args.no_variants:
        line["variants"] = measure_variants(args, fx, inputs, mesh, dev, cfl, zones_per_step, bs,
                                            ws, hbm_peak)
    if not args.no_configs:
        line["configs"] = measure_configs(args, fx, inputs, dev, hbm_peak)
    if not args.no_serving and ws == 1:
        # a bounded sample of the serving configuration (all block counts up
        # to 4096, fewer requests; `bench.py --serve` runs more)
        line["serving"] = serving_runs(24, 4096, args.serve_budget_gb, double_word=False)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:   # the CPU oracle at N = 1 only
        try:
            line["cpu_baseline"] = oracle_sample(args.workload)
        except Exception as e:  # report, never fake
            line["cpu_baseline"] = {"value": None, "error": str(e)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    bs.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def serving_runs(n_requests: int, max_blocks: int, budget_gb: float, double_word: bool = True):
    """The serving configuration: Poisson streams of advance-k-steps requests
    (seed 11630; 8..max_blocks blocks, log-uniform; nxb 8/16/32; k 1..20;
    Sod/KH/Sedov/advection states), served with continuous batching under a
    device-memory budget, against the plain per-request FP64 path on the same
    arrivals.  Two request mixes: half FP64 / half FP32-bulk, and all
    FP32-bulk (the served FP32-bulk path against per-request FP64 at a stated
    p99).  Each mix: capacity with every request present at t = 0, then
    Poisson arrivals at fractions of that capacity.  Wall clock on the host;
    the requests' initial states wait in page-locked host memory."""
    from paper_2208_11630_gb300 import fx, serve
    inf = float("inf")
    budget = budget_gb * 1e9
    out = {}
    t_prep = time.perf_counter()
    mixes = {"mixed": 0.5, "f32bulk": 1.0}
    streams = {name: serve.make_stream(n_requests, inf, seed=11630, blocks=(8, max_blocks),
                                       f32_frac=frac) for name, frac in mixes.items()}
    # the two mixes share sizes, setups and k (same seed); only precision differs
    probs = serve.prepare(streams["mixed"])
    out["prep_s"] = time.perf_counter() - t_prep
    for name, reqs in streams.items():
        runs = {}
        # warm-up pass: kernels loaded, launch choices tuned and cached
        serve.serve(serve.with_arrivals(reqs, inf), probs, budget, realtime=False)
        sat = serve.serve(serve.with_arrivals(reqs, inf), probs, budget, realtime=False)
        cap = sat["requests_per_s"]
        runs["saturated"] = sat
        fracs = (0.5, 0.8, 0.95) if name == "mixed" else (0.8,)
        for frac in fracs:
            runs[f"rate_{frac}"] = serve.serve(serve.with_arrivals(reqs, frac * cap), probs, budget)
        runs["per_request_fp64_at_0.8"] = serve.serve_per_request(
            serve.with_arrivals(reqs, 0.8 * cap), probs, precision=fx.FX_F64)
        if double_word and name == "mixed":
            serve.serve(serve.with_arrivals(reqs, inf), probs, budget, realtime=False, f64_arith=1)
            runs["saturated_f64_double_word"] = serve.serve(serve.with_arrivals(reqs, inf), probs,
                                                            budget, realtime=False, f64_arith=1)
            runs["rate_0.8_f64_double_word"] = serve.serve(serve.with_arrivals(reqs, 0.8 * cap),
                                                           probs, budget, f64_arith=1)
        out[name] = {"capacity_requests_per_s": cap, "runs": runs}
    blocks = [r.nblocks for r in streams["mixed"]]
    out["stream"] = {"requests": n_requests, "blocks": f"log-uniform 8..{max_blocks}",
                     "blocks_max_drawn": int(max(blocks)), "blocks_median": float(np.median(blocks)),
                     "nxb": "8/16/32", "k": "1..20", "setups": "sod/kh/sedov/advection",
                     "budget_gb": budget_gb, "arrivals": "Poisson, seed 11630, rate = fraction "
                     "of saturated capacity"}
    return out


def run_fma_probe(args):
    """FMA-pipe throughput of this GPU (FP64 and FP32), the library's probe
    kernel timed with CUDA events, with the SM clocks sampled meanwhile."""
    import torch
    from paper_2208_11630_gb300 import fx
    torch.cuda.set_device(0)
    fx.load()
    stream = torch.cuda.Stream()
    out = {"metric": "fma throughput", "unit": "TFLOP/s",
           "derived_fp64_peak": FP64_PEAK_FLOPS / 1e12,
           "derivation": "152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz"}
    for name, prec in (("fp64", fx.FX_F64), ("fp32", fx.FX_F32BULK)):
        clk = ClockSampler(0)
        clk.start()
        v = measure_fma_peak(fx, stream, prec, reps=50)
        out[name] = {"tflops": v / 1e12, "clocks": clk.stop()}
    print(json.dumps(out), flush=True)
    return 0


def run_precision_study(args):
    """Smooth advection at 512^3 (32768 blocks of 16^3, periodic) over one
    domain crossing, t = 1 (the last step shortened to land on it), in
    FP32-bulk and in FP64 on the GPU: the L1 error of the density of each
    against the exact translated profile rho(x - v t), and the largest
    per-cell deviation of FP32-bulk from FP64 (relative to the variable's
    largest magnitude; the momenta share the largest |m|)."""
    import torch
    from paper_2208_11630_gb300 import fx, inputs
    torch.cuda.set_device(0)
    fx.load()
    scale = args.scale or 32
    mesh, W, gamma, cfl = inputs.workload("advection3d", scale=scale)
    n, g = mesh.nxb, mesh.ng
    sl = (slice(None), 0, slice(g, g + n), slice(g, g + n), slice(g, g + n))
    x, y, z = mesh.cell_centers_all()
    exact = inputs.advection_density(x, y, z, 1.0)          # [nb, n, n, n], t = 1
    del x, y, z
    vol = 1.0 / mesh.leaf_zones()
    res = {}
    finals = {}
    for name, prec in (("f64", fx.FX_F64), ("f32bulk", fx.FX_F32BULK)):
        bs = fx.BlockSet(mesh, gamma, precision=prec)
        bs.set_primitive(W)
        t, steps = 0.0, 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while t < 1.0:
            fx.fx_compute_dt(bs.ctx, bs.bs, cfl, bs.dt.data_ptr(), None)
            dt = float(bs.dt.item())
            if t + dt > 1.0:
                dt = 1.0 - t
                bs.dt.fill_(dt)
            fx.fx_guardcell_fill_amr(bs.ctx, bs.bs, None)
            fx.fx_hydro_advance(bs.ctx, bs.bs, bs.dt.data_ptr(), None)
            t += dt
            steps += 1
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        rho = bs.current[sl].double().cpu().numpy()
        l1 = float(np.abs(rho - exact).sum() * vol)
        res[name] = {"steps": steps, "t": t, "wall_s": wall, "l1_rho_vs_exact": l1,
                     "status": bs.status(), "zone_updates_per_s": mesh.leaf_zones() * steps / wall}
        finals[name] = bs
    a = finals["f32bulk"].current
    r = finals["f64"].current
    g2 = (slice(None), slice(None), slice(g, g + n), slice(g, g + n), slice(g, g + n))
    dev = 0.0
    for v in range(5):
        rv = r[g2][:, v]
        sc = rv.abs().amax() if v in (0, 4) else r[g2][:, 1:4].square().sum(dim=1).sqrt().amax()
        dev = max(dev, float(((a[g2][:, v].double() - rv).abs() / torch.maximum(
            rv.abs(), sc.clamp_min(1e-300))).max()))
    res["max_rel_dev_f32bulk_from_f64"] = dev
    res["l1_relative_difference"] = abs(res["f32bulk"]["l1_rho_vs_exact"] -
                                        res["f64"]["l1_rho_vs_exact"]) / res["f64"]["l1_rho_vs_exact"]
    line = {"metric": "precision study", "workload": f"advection3d_{scale * n}^3", "crossing_t": 1.0,
            "blocks": mesh.nb, "zones": mesh.leaf_zones(), "cfl": cfl, "results": res,
            "data": "synthetic (seed 2208)"}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Serving stream at the configuration's sizes (blocks up to 4096)."""
    import torch
    from paper_2208_11630_gb300 import fx
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(0)
    fx.load()
    clocks = ClockSampler(0)
    clocks.start()
    res = serving_runs(args.serve_requests, args.serve_max_blocks, args.serve_budget_gb)
    clk = clocks.stop()
    line = {"metric": "served zone-updates/s",
            "value": res["mixed"]["runs"]["rate_0.8"]["zone_updates_per_s"],
            "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "dtype": "mixed f64/f32bulk", "config": {"workload": "serving stream"} | res["stream"],
            "serving": res, "clocks": clk,
            "timing": "wall clock on the host, requests' initial states in page-locked memory"}
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="kh3d")
    ap.add_argument("--precision", default="f64", choices=["f64", "f32bulk"])
    ap.add_argument("--scale", type=int, default=None,
                    help="blocks per axis (default: the full workload, 16 for kh3d)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the batched-graph and other-precision measurements")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workloads (Sod 2D, Sedov AMR batched, advection 512^3)")
    ap.add_argument("--serve", action="store_true", help="run the serving stream instead")
    ap.add_argument("--fma-probe", action="store_true",
                    help="measure the FP64 and FP32 FMA throughput instead")
    ap.add_argument("--precision-study", action="store_true",
                    help="run the 512^3 advection crossing in FP32-bulk and FP64 instead")
    ap.add_argument("--serve-requests", type=int, default=64)
    ap.add_argument("--serve-max-blocks", type=int, default=4096)
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the serving sample in the default line")
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    args = ap.parse_args(argv)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.serve:
        return run_serve(args)
    if args.precision_study:
        return run_precision_study(args)
    if args.fma_probe:
        return run_fma_probe(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
