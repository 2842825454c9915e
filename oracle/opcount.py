"""Arithmetic per zone update, counted on the oracle (op-counting build).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.  Runs the counting
build of the oracle (``opcount.cpp``) for whole steps of a workload and
reports, per step of the scheme, the FP64 operations per unit of work (+, -,
*, / and sqrt; min/max, absolute value and comparisons kept apart), and from
them the operations per zone update:

* algorithmic -- each unit as often as the scheme needs it once per zone: one
  primitive conversion, one cell's slopes/predictor/face states, ``ndim``
  face fluxes, one conservative update and one signal speed (for the next
  step's CFL reduction) per zone; the positivity check is a diagnostic and is
  listed separately;
* as executed by the oracle's block loops (primitives on every padded cell,
  the predictor on the interior grown by one, ...), for reference.

Usage: ``python -m oracle.opcount [workload] [blocks-per-axis] [warm-up steps]``
prints a Markdown summary (default: the 3D Kelvin-Helmholtz shear layer, 4^3
blocks of 16^3, after 10 steps; blocks-per-axis 0 = the workload's full size).  The counted step's state is also checked
against the normal oracle build, bit for bit.
"""
from __future__ import annotations

import ctypes
import sys

import numpy as np

STEPS = ["primitives (per cell)", "slopes + predictor + face states (per cell)",
         "HLLC flux (per face)", "conservative update (per cell)",
         "positivity check (per new cell)", "CFL signal speed (per cell)", "outside units"]
KINDS = ["add", "sub", "mul", "div", "sqrt", "minmax", "abs", "cmp"]
FLOP_KINDS = ("add", "sub", "mul", "div", "sqrt")


def _read(L):
    ops = np.zeros((7, 8), dtype=np.uint64)
    units = np.zeros(7, dtype=np.uint64)
    L.or_opcount_get(ops.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                     units.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    return ops.astype(np.float64), units.astype(np.float64)


def count_step(name: str = "kh3d", scale: int = 4, warm: int = 10, cfl: float = 0.8):
    """Count one full step (dt, guard fill, update) of workload ``name`` after
    ``warm`` uncounted steps.  Returns a dict with the per-unit and per-zone
    figures."""
    import oracle
    from paper_2208_11630_gb300 import inputs
    L = oracle.opcount_lib()
    mesh, W, gamma, _ = inputs.workload(name, scale=scale or None)
    om = oracle.OracleMesh(mesh, gamma)              # the normal build
    oc = oracle.OracleMesh(mesh, gamma, library=L)   # the counting build
    U = om.prim_to_cons(W)
    U, _, _ = om.run(U, nsteps=warm, cfl=cfl)
    L.or_opcount_reset()
    Uc, dtc = oc.step(U, cfl=cfl)
    L.or_opcount_close()
    ops, units = _read(L)
    Un, dtn = om.step(U, cfl=cfl)
    same = bool(np.array_equal(Uc, Un)) and dtc == dtn
    zones = float(mesh.leaf_zones())
    per_unit = {}
    for s in range(6):
        if units[s] > 0:
            per_unit[STEPS[s]] = {k: ops[s, i] / units[s] for i, k in enumerate(KINDS)}
            per_unit[STEPS[s]]["units"] = units[s]
    flops = {st: sum(d[k] for k in FLOP_KINDS) for st, d in per_unit.items()}
    nd = mesh.ndim
    mult = {STEPS[0]: 1.0, STEPS[1]: 1.0, STEPS[2]: float(nd), STEPS[3]: 1.0, STEPS[5]: 1.0}
    algo = sum(flops[k] * m for k, m in mult.items())
    executed = sum(ops[s, i] for s in range(7) for i, k in enumerate(KINDS)
                   if k in FLOP_KINDS and s != 4) / zones
    by_kind = {k: sum(per_unit[st][k] * m for st, m in mult.items()) for k in KINDS}
    return {"workload": name, "scale": scale, "warm": warm, "zones": zones, "ndim": nd,
            "per_unit": per_unit, "flops_per_unit": flops, "algorithmic_per_zone": algo,
            "algorithmic_by_kind": by_kind, "oracle_executed_per_zone": executed,
            "check_per_cell": flops.get(STEPS[4], 0.0), "same_as_oracle": same}


def summary(r) -> str:
    lines = [f"## {r['workload']} ({int(r['zones'] / 16 ** r['ndim'])} blocks of 16^{r['ndim']}, one full "
             f"step after {r['warm']} steps; {int(r['zones'])} zones)", "",
             "| step | units | add | sub | mul | div | sqrt | flops/unit | min/max | abs | cmp |",
             "|---|---|---|---|---|---|---|---|---|---|---|"]
    for st, d in r["per_unit"].items():
        lines.append(f"| {st} | {int(d['units'])} | " + " | ".join(
            f"{d[k]:.3f}" for k in FLOP_KINDS) + f" | {r['flops_per_unit'][st]:.3f} | "
            + " | ".join(f"{d[k]:.3f}" for k in ("minmax", "abs", "cmp")) + " |")
    bk = r["algorithmic_by_kind"]
    lines += ["", f"Algorithmic FP64 flops per zone update (1 primitive conversion, 1 predictor, "
              f"{r['ndim']} faces, 1 update, 1 signal speed): **{r['algorithmic_per_zone']:.1f}** "
              f"(add {bk['add']:.1f}, sub {bk['sub']:.1f}, mul {bk['mul']:.1f}, div {bk['div']:.1f}, "
              f"sqrt {bk['sqrt']:.1f}; besides: min/max {bk['minmax']:.1f}, abs {bk['abs']:.1f}, "
              f"compare {bk['cmp']:.1f}).",
              f"As executed by the oracle's block loops: {r['oracle_executed_per_zone']:.1f} "
              f"flops per zone (halo work included; positivity check excluded).",
              f"Positivity check (diagnostic, not counted): {r['check_per_cell']:.1f} flops per "
              f"cell.  Counted step identical to the normal oracle build: {r['same_as_oracle']}."]
    return "\n".join(lines)


def main(argv):
    name = argv[1] if len(argv) > 1 else "kh3d"
    scale = int(argv[2]) if len(argv) > 2 else 4
    warm = int(argv[3]) if len(argv) > 3 else 10
    print(summary(count_step(name, scale, warm)))


if __name__ == "__main__":
    main(sys.argv)
