"""Plain FP64 CPU oracle of the block-AMR unsplit Euler step (ctypes binding).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(``paper_2208_11630_gb300``) never imports it, and the two share no code; the
only common module is the seeded input generator, which holds no method
arithmetic.

The C sources (``oracle.c``, ``riemann_exact.c``) restate the scheme from its
textbook definitions; see ``fx_oracle.h`` for what each routine computes and
how it is pinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = [os.path.join(_HERE, f) for f in ("oracle.c", "riemann_exact.c")]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (-O2, OpenMP, no FP contraction)."""
    newest = max(os.path.getmtime(f) for f in _SRC + [os.path.join(_HERE, "fx_oracle.h")])
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-Wno-unknown-pragmas", "-o", tmp] + _SRC + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _bind(L):
    """Argument and result types of the oracle's C entry points on library L."""
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    i64p = ctypes.POINTER(ctypes.c_int64)
    L.or_mesh_create.restype = ctypes.c_void_p
    L.or_mesh_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ip, ip, i64p, ip, dp, dp, ip, ctypes.c_double]
    L.or_mesh_destroy.argtypes = [ctypes.c_void_p]
    L.or_last_error.restype = ctypes.c_char_p
    L.or_set_threads.argtypes = [ctypes.c_int]
    L.or_get_threads.restype = ctypes.c_int
    L.or_prim_to_cons.argtypes = [ctypes.c_void_p, dp, dp]
    L.or_cons_to_prim.argtypes = [ctypes.c_void_p, dp, dp]
    L.or_guardcell_fill.argtypes = [ctypes.c_void_p, dp]
    L.or_compute_dt.argtypes = [ctypes.c_void_p, dp, ctypes.c_double, ctypes.c_int, dp]
    L.or_hydro_advance.argtypes = [ctypes.c_void_p, dp, dp, ctypes.c_double, ctypes.c_int,
                                   dp, ctypes.c_int, ip]
    L.or_conserved_totals.argtypes = [ctypes.c_void_p, dp, dp]
    L.or_restrict_parents.argtypes = [ctypes.c_void_p, dp]
    L.or_hydro_advance_rk2.argtypes = [ctypes.c_void_p, dp, dp, ctypes.c_double,
                                       ctypes.c_int, dp]
    L.or_hydro_advance_rk3.argtypes = [ctypes.c_void_p, dp, dp, ctypes.c_double,
                                       ctypes.c_int, dp]
    i64p = ctypes.POINTER(ctypes.c_int64)
    L.or_mesh_set_species.argtypes = [ctypes.c_void_p, ctypes.c_int, dp, dp]
    L.or_riemann_star2.argtypes = [dp, dp, ctypes.c_double, ctypes.c_double, dp]
    L.or_riemann_sample2.argtypes = [dp, dp, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, dp]
    L.or_regrid_errors.argtypes = [ctypes.c_void_p, dp, ctypes.c_double, dp]
    L.or_regrid_plan.argtypes = [ctypes.c_void_p, dp, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_int, ctypes.c_int, ip, i64p, ip, ip, ip, ip]
    L.or_regrid_transfer.argtypes = [ctypes.c_void_p, dp, ctypes.c_void_p, ip, ip, ip,
                                     dp]
    L.or_mc.restype = ctypes.c_double
    L.or_mc.argtypes = [ctypes.c_double, ctypes.c_double]
    L.or_hllc.argtypes = [dp, dp, ctypes.c_int, ctypes.c_double, dp]
    L.or_riemann_star.argtypes = [dp, dp, ctypes.c_double, dp]
    L.or_riemann_sample.argtypes = [dp, dp, ctypes.c_double, ctypes.c_double, dp]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = _bind(ctypes.CDLL(_SO))
            _lib = L
    return _lib


_OPC_SO = os.path.join(_HERE, "liboracle_opcount.so")
_opc_lib = None


def opcount_lib():
    """The op-counting build of the oracle (opcount.cpp: oracle.c compiled as
    C++ with a counting double type, single-threaded), with the same entry
    points plus or_opcount_reset / or_opcount_get / or_opcount_close."""
    global _opc_lib
    with _lock:
        if _opc_lib is None:
            srcs = [os.path.join(_HERE, f) for f in ("opcount.cpp", "riemann_exact.c",
                                                      "oracle.c", "fx_oracle.h")]
            newest = max(os.path.getmtime(f) for f in srcs)
            if not os.path.exists(_OPC_SO) or os.path.getmtime(_OPC_SO) < newest:
                tmp = _OPC_SO + f".tmp{os.getpid()}"
                obj = tmp + ".riemann.o"
                subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-c", "-ffp-contract=off",
                                "-fno-fast-math", "-o", obj, srcs[1]], check=True)
                subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared",
                                "-ffp-contract=off", "-fno-fast-math", "-o", tmp, srcs[0], obj,
                                "-lm"], check=True)
                os.unlink(obj)
                os.replace(tmp, _OPC_SO)
            L = _bind(ctypes.CDLL(_OPC_SO))
            u64p = ctypes.POINTER(ctypes.c_uint64)
            L.or_opcount_get.argtypes = [u64p, u64p]
            _opc_lib = L
    return _opc_lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def get_threads() -> int:
    return int(lib().or_get_threads())


class OracleMesh:
    """The oracle's view of a block set; ``mesh`` is an ``inputs.Mesh``."""

    def __init__(self, mesh, gamma: float = 1.4, library=None):
        L = self._L = lib() if library is None else library
        self.mesh = mesh
        self.gamma = float(gamma)
        self._level = np.ascontiguousarray(mesh.level, dtype=np.int32)
        self._origin = np.ascontiguousarray(mesh.origin, dtype=np.int64)
        self._parent = np.ascontiguousarray(mesh.parent, dtype=np.int32)
        nroot = np.array(mesh.nroot, dtype=np.int32)
        lo = np.array(mesh.lo, dtype=np.float64)
        hi = np.array(mesh.hi, dtype=np.float64)
        bc = mesh.bc_flat()
        self._h = L.or_mesh_create(mesh.ndim, mesh.nxb, mesh.ng, mesh.nb, _ip(nroot),
                                   _ip(self._level),
                                   self._origin.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                   _ip(self._parent), _dp(lo), _dp(hi), _ip(bc), self.gamma)
        if not self._h:
            raise ValueError(L.or_last_error().decode())
        ns = int(getattr(mesh, "nspec", 0))
        if ns:
            g = np.array([sp[0] for sp in mesh.species], dtype=np.float64)
            a = np.array([sp[1] for sp in mesh.species], dtype=np.float64)
            if L.or_mesh_set_species(self._h, ns, _dp(g), _dp(a)):
                raise ValueError(L.or_last_error().decode())

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.or_mesh_destroy(h)
            self._h = None

    # -- EOS ------------------------------------------------------------
    def prim_to_cons(self, W: np.ndarray) -> np.ndarray:
        U = np.zeros_like(W)
        self._L.or_prim_to_cons(self._h, _dp(W), _dp(U))
        return U

    def cons_to_prim(self, U: np.ndarray) -> np.ndarray:
        W = np.zeros_like(U)
        self._L.or_cons_to_prim(self._h, _dp(U), _dp(W))
        return W

    # -- step pieces ------------------------------------------------------
    def guardcell_fill(self, U: np.ndarray) -> None:
        if self._L.or_guardcell_fill(self._h, _dp(U)):
            raise RuntimeError(self._L.or_last_error().decode())

    def compute_dt(self, U: np.ndarray, cfl: float = 0.8, form: int = 0) -> float:
        dt = np.zeros(1)
        self._L.or_compute_dt(self._h, _dp(U), float(cfl), int(form), _dp(dt))
        return float(dt[0])

    def hydro_advance(self, U: np.ndarray, dt: float, reflux: bool = True,
                      want_bflux: bool = False, select=None, integrator: int = 0):
        """Advance the leaves one step from ``U`` (guards filled).  Returns
        ``(Unew, status, bflux)``; ``Unew`` starts as a copy of ``U``.
        integrator 0: MUSCL-Hancock; 1: SSP-RK2; 2: SSP-RK3 (no ``select``)."""
        m = self.mesh
        Unew = U.copy()
        bflux = None
        bptr = None
        if want_bflux:
            nf = m.nxb ** (m.ndim - 1)
            bflux = np.zeros((m.nb, 2 * m.ndim, 5 + int(getattr(m, "nspec", 0)), nf))
            bptr = _dp(bflux)
        if integrator == 1:
            st = self._L.or_hydro_advance_rk2(self._h, _dp(U), _dp(Unew), float(dt), int(reflux), bptr)
            return Unew, st, bflux
        if integrator == 2:
            st = self._L.or_hydro_advance_rk3(self._h, _dp(U), _dp(Unew), float(dt), int(reflux), bptr)
            return Unew, st, bflux
        if select is not None:
            sel = np.ascontiguousarray(select, dtype=np.int32)
            st = self._L.or_hydro_advance(self._h, _dp(U), _dp(Unew), float(dt), int(reflux), bptr,
                                        len(sel), _ip(sel))
        else:
            st = self._L.or_hydro_advance(self._h, _dp(U), _dp(Unew), float(dt), int(reflux), bptr,
                                        0, None)
        return Unew, st, bflux

    def regrid_errors(self, U: np.ndarray, eps: float = 0.01) -> np.ndarray:
        """Loehner indicator per block (U guard-filled; -1 for parents)."""
        err = np.zeros(self.mesh.nb)
        self._L.or_regrid_errors(self._h, _dp(U), float(eps), _dp(err))
        return err

    def regrid(self, U: np.ndarray, refine_cutoff: float = 0.8, derefine_cutoff: float = 0.2,
               eps: float = 0.01, max_level: int | None = None):
        """One regrid of state ``U``: restriction into parents, full guard
        fill, error estimate, marking with 2:1 balance, new mesh, data
        transfer, restriction into the new parents.  Returns
        ``(OracleMesh of the new mesh, new state, errors, (kind, src, oct))``."""
        import dataclasses
        m = self.mesh
        max_level = int(m.level.max()) + 1 if max_level is None else int(max_level)
        U = U.copy()
        self.restrict_parents(U)
        self.guardcell_fill(U)
        err = self.regrid_errors(U, eps)
        level, origin, parent, kind, src, octs = self.regrid_plan(err, refine_cutoff,
                                                                 derefine_cutoff, max_level)
        new_mesh = dataclasses.replace(m, level=level, origin=origin, parent=parent, extra={})
        om = OracleMesh(new_mesh, self.gamma, self._L)
        Unew = np.zeros(new_mesh.shape)
        maps = (kind, src, octs)
        self._L.or_regrid_transfer(self._h, _dp(U), om._h, _ip(maps[0]), _ip(maps[1]),
                                 _ip(maps[2]), _dp(Unew))
        om.restrict_parents(Unew)
        return om, Unew, err, maps

    def regrid_plan(self, err: np.ndarray, refine_cutoff: float, derefine_cutoff: float,
                    max_level: int):
        """Marking and 2:1 balance for per-block indicator values ``err``
        (or_regrid_plan).  Returns ``(level, origin, parent, kind, src,
        oct)`` of the new mesh, sorted by (level, z, y, x of the origin)."""
        m = self.mesh
        err = np.ascontiguousarray(err, dtype=np.float64)
        cap = m.nb * (1 + 2 ** m.ndim)
        level = np.zeros(cap, dtype=np.int32)
        origin = np.zeros((cap, 3), dtype=np.int64)
        parent = np.zeros(cap, dtype=np.int32)
        kind = np.zeros(cap, dtype=np.int32)
        src = np.zeros(cap, dtype=np.int32)
        octs = np.zeros(cap, dtype=np.int32)
        nn = self._L.or_regrid_plan(self._h, _dp(err), float(refine_cutoff), float(derefine_cutoff),
                                  int(max_level), cap, _ip(level),
                                  origin.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                  _ip(parent), _ip(kind), _ip(src), _ip(octs))
        if nn < 0:
            raise RuntimeError(self._L.or_last_error().decode())
        return tuple(a[:nn].copy() for a in (level, origin, parent, kind, src, octs))

    def restrict_parents(self, U: np.ndarray) -> None:
        self._L.or_restrict_parents(self._h, _dp(U))

    def conserved_totals(self, U: np.ndarray) -> np.ndarray:
        out = np.zeros(5 + int(getattr(self.mesh, "nspec", 0)))
        self._L.or_conserved_totals(self._h, _dp(U), _dp(out))
        return out

    def step(self, U: np.ndarray, cfl: float = 0.8, dt: float | None = None, form: int = 0,
             reflux: bool = True, t_end: float | None = None, t: float = 0.0,
             integrator: int = 0):
        """One full step: dt, guard fill, advance.  Returns ``(Unew, dt)``."""
        U = U.copy()
        if dt is None:
            dt = self.compute_dt(U, cfl, form)
        if t_end is not None:
            dt = min(dt, t_end - t)
        self.guardcell_fill(U)
        Unew, st, _ = self.hydro_advance(U, dt, reflux, integrator=integrator)
        if st:
            raise FloatingPointError("unphysical state after step")
        return Unew, dt

    def run(self, U: np.ndarray, nsteps: int | None = None, t_end: float | None = None,
            cfl: float = 0.8, form: int = 0, reflux: bool = True, max_steps: int = 100000,
            integrator: int = 0):
        t = 0.0
        n = 0
        while True:
            if nsteps is not None and n >= nsteps:
                break
            if t_end is not None and t >= t_end * (1 - 1e-14):
                break
            if n >= max_steps:
                raise RuntimeError("too many steps")
            U, dt = self.step(U, cfl=cfl, form=form, reflux=reflux, t_end=t_end, t=t,
                              integrator=integrator)
            t += dt
            n += 1
        return U, t, n


def mc(a: float, b: float) -> float:
    return float(lib().or_mc(float(a), float(b)))


def hllc(WL, WR, direction: int, gamma: float = 1.4) -> np.ndarray:
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    F = np.zeros(5)
    lib().or_hllc(_dp(WL), _dp(WR), int(direction), float(gamma), _dp(F))
    return F


def riemann_star(WL, WR, gamma: float = 1.4) -> np.ndarray:
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    out = np.zeros(4)
    if lib().or_riemann_star(_dp(WL), _dp(WR), float(gamma), _dp(out)):
        raise ValueError("vacuum")
    return out


def riemann_sample2(WL, WR, xi, gL: float, gR: float) -> np.ndarray:
    """Exact solution of a two-gas Riemann problem ({rho, u, p} per side,
    gamma gL left of the contact, gR right) sampled at xi = x/t (array)."""
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    out = np.zeros((xi.size, 3))
    wl = np.ascontiguousarray(WL, dtype=np.float64)
    wr = np.ascontiguousarray(WR, dtype=np.float64)
    o = np.zeros(3)
    for i, x in enumerate(xi):
        if lib().or_riemann_sample2(_dp(wl), _dp(wr), float(gL), float(gR), float(x), _dp(o)):
            raise ValueError("vacuum")
        out[i] = o
    return out


def riemann_sample(WL, WR, xi, gamma: float = 1.4) -> np.ndarray:
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    out = np.zeros((xi.size, 3))
    o = np.zeros(3)
    for n, x in enumerate(xi.ravel()):
        lib().or_riemann_sample(_dp(WL), _dp(WR), float(gamma), float(x), _dp(o))
        out[n] = o
    return out
