"""Thin ctypes binding of libfx (include/fx.h).

Functions keep the C names and only marshal arguments: every step of the hot
path runs in the library's CUDA kernels.  PyTorch supplies device memory and
streams.  There is no CPU fallback: if ``libfx.so`` cannot be built or loaded,
or no CUDA device is present, these calls raise.

``BlockSet`` is a small convenience wrapper that owns the two state tensors
of one block set and forwards to the C calls.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

FX_OK = 0
FX_ERR = {-1: "FX_ERR_ARG", -2: "FX_ERR_CUDA", -3: "FX_ERR_OOM", -4: "FX_ERR_UNPHYSICAL",
          -5: "FX_ERR_TIMEOUT", -6: "FX_ERR_STATE", -7: "FX_ERR_MESH"}
FX_F64 = 0
FX_F32BULK = 1
FX_BC_OUTFLOW = 0
FX_BC_PERIODIC = 1
FX_BC_REFLECT = 2
FX_MAXVAR = 9          # 5 + at most 4 species

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None
_lock = threading.Lock()


class FxError(RuntimeError):
    def __init__(self, code, msg=""):
        self.code = code
        super().__init__(f"{FX_ERR.get(code, code)}: {msg}")


def lib_path() -> str:
    return os.path.join(_HERE, "libfx.so")


def load(build: bool = True):
    """Load libfx.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build:
            from . import _build
            _build.build()
        L = ctypes.CDLL(lib_path())
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
        i64p = ctypes.POINTER(ctypes.c_int64)
        c_int, c_double = ctypes.c_int, ctypes.c_double
        sig = {
            "fx_init": (c_int, [c_double, c_int, c_int, ctypes.POINTER(vp)]),
            "fx_finalize": (c_int, [vp]),
            "fx_set_option": (c_int, [vp, ctypes.c_char_p, c_double]),
            "fx_set_species": (c_int, [vp, c_int, dp, dp]),
            "fx_last_error": (ctypes.c_char_p, [vp]),
            "fx_blocks_create": (c_int, [vp, c_int, c_int, c_int, ip, ip, i64p, ip, dp, dp, ip,
                                         c_int, vp, vp, ctypes.POINTER(vp)]),
            "fx_blocks_destroy": (c_int, [vp]),
            "fx_blocks_current": (c_int, [vp]),
            "fx_blocks_mark_dirty": (c_int, [vp]),
            "fx_prim_to_cons": (c_int, [vp, vp, vp, vp]),
            "fx_guardcell_fill": (c_int, [vp, vp, vp]),
            "fx_guardcell_fill_amr": (c_int, [vp, vp, vp]),
            "fx_compute_dt": (c_int, [vp, vp, c_double, vp, vp]),
            "fx_hydro_advance": (c_int, [vp, vp, vp, vp]),
            "fx_step": (c_int, [vp, vp, c_double, vp, vp]),
            "fx_conserved_totals": (c_int, [vp, vp, dp, vp]),
            "fx_status": (c_int, [vp, vp]),
            "fx_run_host": (c_int, [vp, vp, vp, vp, c_int, c_double, dp, vp]),
            "fx_run_host_interior": (c_int, [vp, vp, vp, vp, c_int, c_double, dp, vp]),
            "fx_regrid_plan": (c_int, [vp, vp, c_double, c_double, c_double, c_int, vp, ip]),
            "fx_regrid_errors": (c_int, [vp, dp]),
            "fx_regrid_mesh": (c_int, [vp, ip, i64p, ip]),
            "fx_regrid_apply": (c_int, [vp, vp, vp, vp, vp]),
            "fx_regrid_plan_host": (c_int, [c_int, c_int, ip, ip, c_int, ip, i64p, ip, dp,
                                            c_double, c_double, c_int, c_int, ip, ip, i64p, ip,
                                            ip, ctypes.c_char_p, c_int]),
            "fx_block_fluxes": (vp, [vp, c_int]),
            "fx_kernel_launches": (ctypes.c_longlong, []),
            "fx_dword_selftest": (c_int, [c_int, vp, vp, vp, c_int, vp]),
            "fx_fma_probe": (c_int, [c_int, c_int, c_int, vp, vp, ctypes.POINTER(ctypes.c_double)]),
            "fx_batch_create": (c_int, [vp, c_int, ctypes.POINTER(vp)]),
            "fx_batch_destroy": (c_int, [vp]),
            "fx_batch_add": (c_int, [vp, vp, c_double, c_int, vp, ip]),
            "fx_batch_run": (c_int, [vp, c_int, vp]),
            "fx_batch_poll": (c_int, [vp, ip, vp]),
            "fx_batch_remove": (c_int, [vp, c_int, vp]),
            "fx_batch_tune": (c_int, [vp, vp, ip]),
            "fx_batch_choice": (c_int, [vp, c_int, c_int, ip, ip]),
            "fx_batch_path": (c_int, [vp, c_int, ip]),
            "fx_compute_dt_noalloc": (c_int, [vp, c_int, c_int, c_int, c_int, dp, c_double,
                                              c_double, c_int, vp, vp, ctypes.c_char_p,
                                              ctypes.c_size_t]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def _check(ctx, rc):
    if rc != FX_OK:
        msg = load().fx_last_error(ctx).decode() if ctx else ""
        raise FxError(rc, msg)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# ---------------------------------------------------------------- raw calls

def fx_init(gamma: float, nxb: int, nguard: int):
    ctx = ctypes.c_void_p()
    rc = load().fx_init(float(gamma), int(nxb), int(nguard), ctypes.byref(ctx))
    if rc != FX_OK:
        raise FxError(rc, "fx_init")
    return ctx


def fx_finalize(ctx):
    _check(None, load().fx_finalize(ctx))


def fx_set_species(ctx, species) -> None:
    """Multispecies perfect gas for block sets created afterwards:
    ``species`` = ((gamma_k, A_k), ...) (empty: the single gas)."""
    g = np.array([sp[0] for sp in species], dtype=np.float64)
    a = np.array([sp[1] for sp in species], dtype=np.float64)
    pd = ctypes.POINTER(ctypes.c_double)
    _check(ctx, load().fx_set_species(ctx, len(species), g.ctypes.data_as(pd) if len(g) else None,
                                      a.ctypes.data_as(pd) if len(a) else None))


def fx_set_option(ctx, key: str, value: float):
    _check(ctx, load().fx_set_option(ctx, key.encode(), float(value)))


def fx_blocks_create(ctx, mesh, precision: int, U0_ptr: int, U1_ptr: int):
    level = np.ascontiguousarray(mesh.level, dtype=np.int32)
    origin = np.ascontiguousarray(mesh.origin, dtype=np.int64)
    parent = np.ascontiguousarray(mesh.parent, dtype=np.int32)
    nroot = np.array(mesh.nroot, dtype=np.int32)
    lo = np.array(mesh.lo, dtype=np.float64)
    hi = np.array(mesh.hi, dtype=np.float64)
    bc = mesh.bc_flat()
    ip = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    bs = ctypes.c_void_p()
    rc = load().fx_blocks_create(ctx, mesh.ndim, mesh.nb, mesh.nxb, ip(nroot), ip(level),
                                 origin.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ip(parent),
                                 dp(lo), dp(hi), ip(bc), int(precision), ctypes.c_void_p(U0_ptr),
                                 ctypes.c_void_p(U1_ptr), ctypes.byref(bs))
    _check(ctx, rc)
    return bs


def fx_blocks_destroy(bs):
    load().fx_blocks_destroy(bs)


def fx_blocks_mark_dirty(bs):
    load().fx_blocks_mark_dirty(bs)


def fx_blocks_current(bs) -> int:
    return int(load().fx_blocks_current(bs))


def fx_prim_to_cons(ctx, bs, W_ptr: int, stream=None):
    _check(ctx, load().fx_prim_to_cons(ctx, bs, ctypes.c_void_p(W_ptr), _stream_ptr(stream)))


def fx_guardcell_fill(ctx, bs, stream=None):
    _check(ctx, load().fx_guardcell_fill(ctx, bs, _stream_ptr(stream)))


def fx_guardcell_fill_amr(ctx, bs, stream=None):
    _check(ctx, load().fx_guardcell_fill_amr(ctx, bs, _stream_ptr(stream)))


def fx_compute_dt(ctx, bs, cfl: float, dt_ptr: int, stream=None):
    _check(ctx, load().fx_compute_dt(ctx, bs, float(cfl), ctypes.c_void_p(dt_ptr), _stream_ptr(stream)))


def fx_hydro_advance(ctx, bs, dt_ptr: int, stream=None):
    _check(ctx, load().fx_hydro_advance(ctx, bs, ctypes.c_void_p(dt_ptr), _stream_ptr(stream)))


def fx_step(ctx, bs, cfl: float, dt_ptr: int, stream=None):
    _check(ctx, load().fx_step(ctx, bs, float(cfl), ctypes.c_void_p(dt_ptr), _stream_ptr(stream)))


def fx_conserved_totals(ctx, bs, stream=None, nvar: int = 5) -> np.ndarray:
    """Totals of the first ``nvar`` variables (room for every variable the
    library may write is always provided)."""
    out = np.zeros(FX_MAXVAR)
    _check(ctx, load().fx_conserved_totals(ctx, bs, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           _stream_ptr(stream)))
    return out[:nvar]


def fx_status(ctx, bs) -> int:
    return int(load().fx_status(ctx, bs))


def fx_run_host(ctx, bs, host_in: np.ndarray, host_out: np.ndarray, nsteps: int, cfl: float,
                stream=None, want_time: bool = False):
    t = np.zeros(1)
    tp = t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if want_time else None
    _check(ctx, load().fx_run_host(ctx, bs, ctypes.c_void_p(host_in.ctypes.data),
                                   ctypes.c_void_p(host_out.ctypes.data), int(nsteps), float(cfl),
                                   tp, _stream_ptr(stream)))
    return float(t[0]) if want_time else None


def fx_run_host_interior(ctx, bs, host_in: np.ndarray, host_out: np.ndarray, nsteps: int,
                         cfl: float, stream=None, want_time: bool = False):
    """``host_in``/``host_out``: packed interior cells ``[nb, nvar, nz, n, n]``."""
    t = np.zeros(1)
    tp = t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if want_time else None
    _check(ctx, load().fx_run_host_interior(ctx, bs, ctypes.c_void_p(host_in.ctypes.data),
                                            ctypes.c_void_p(host_out.ctypes.data), int(nsteps),
                                            float(cfl), tp, _stream_ptr(stream)))
    return float(t[0]) if want_time else None


def fx_compute_dt_noalloc(U_ptr: int, ndim: int, nblocks: int, nxb: int, nguard: int, dx,
                          gamma: float, cfl: float, cfl_form: int, dt_ptr: int, stream=None):
    """dt for callers that cannot allocate device memory (see fx.h).  Returns
    ``(rc, message)``; the library allocates nothing, not even for errors."""
    dxa = np.ascontiguousarray(dx, dtype=np.float64)
    buf = ctypes.create_string_buffer(256)
    rc = load().fx_compute_dt_noalloc(ctypes.c_void_p(U_ptr), int(ndim), int(nblocks), int(nxb),
                                      int(nguard), dxa.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      float(gamma), float(cfl), int(cfl_form), ctypes.c_void_p(dt_ptr),
                                      _stream_ptr(stream), buf, ctypes.sizeof(buf))
    return int(rc), buf.value.decode()


FX_NOALLOC_MAX_BLOCKS = 32768


def fx_block_fluxes(bs, b: int) -> int:
    return load().fx_block_fluxes(bs, int(b)) or 0


# ---------------------------------------------------------------- batches

class Batch:
    """Many block sets advanced together by one replayed CUDA graph per step
    (thin wrapper over the fx_batch_* calls)."""

    def __init__(self, ctx, max_requests: int):
        self.ctx = ctx
        self.max_requests = int(max_requests)
        h = ctypes.c_void_p()
        _check(ctx, load().fx_batch_create(ctx, self.max_requests, ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().fx_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, blockset, cfl: float, nsteps: int, stream=None) -> int:
        slot = ctypes.c_int(-1)
        _check(self.ctx, load().fx_batch_add(self.h, blockset.bs, float(cfl), int(nsteps),
                                             _stream_ptr(stream), ctypes.byref(slot)))
        return slot.value

    def run(self, nsteps: int = 1, stream=None):
        _check(self.ctx, load().fx_batch_run(self.h, int(nsteps), _stream_ptr(stream)))

    def poll(self, stream=None) -> np.ndarray:
        out = np.zeros(self.max_requests, dtype=np.int32)
        _check(self.ctx, load().fx_batch_poll(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                              _stream_ptr(stream)))
        return out

    def remove(self, slot: int, stream=None):
        _check(self.ctx, load().fx_batch_remove(self.h, int(slot), _stream_ptr(stream)))

    def tune(self, stream=None):
        rep = np.zeros(193, dtype=np.int32)
        _check(self.ctx, load().fx_batch_tune(self.h, _stream_ptr(stream),
                                              rep.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
        out = []
        for i in range(64):
            if rep[3 * i] == 0:
                break
            out.append((int(rep[3 * i]), int(rep[3 * i + 1]), int(rep[3 * i + 2])))
        return out

    def path(self, slot: int) -> int:
        """0: batched phases and persistent update; 1: the per-block-set
        kernels on a graph branch (the request fills the GPU)."""
        p = ctypes.c_int()
        _check(self.ctx, load().fx_batch_path(self.h, int(slot), ctypes.byref(p)))
        return p.value

    def choice(self, ndim: int, precision: int):
        t, c = ctypes.c_int(), ctypes.c_int()
        _check(self.ctx, load().fx_batch_choice(self.h, int(ndim), int(precision), ctypes.byref(t),
                                                ctypes.byref(c)))
        return t.value, c.value


def regrid_plan_host(mesh, err, refine_cutoff: float = 0.8, derefine_cutoff: float = 0.2,
                     max_level: int | None = None):
    """Plan a regrid of ``mesh`` for per-block indicator values ``err`` on
    the host (fx_regrid_plan_host; no GPU needed).  Returns ``(level, origin,
    parent, map)`` of the planned mesh, ``map[j] = (kind, source, octant)``."""
    L = load()
    ip = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    i64p = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    level = np.ascontiguousarray(mesh.level, dtype=np.int32)
    origin = np.ascontiguousarray(mesh.origin, dtype=np.int64)
    parent = np.ascontiguousarray(mesh.parent, dtype=np.int32)
    nroot = np.array(mesh.nroot, dtype=np.int32)
    bc = np.ascontiguousarray(mesh.bc_flat(), dtype=np.int32)
    err = np.ascontiguousarray(err, dtype=np.float64)
    if err.shape != (mesh.nb,):
        raise ValueError("one indicator value per block")
    max_level = int(mesh.level.max()) + 1 if max_level is None else int(max_level)
    msg = ctypes.create_string_buffer(256)
    n = ctypes.c_int(0)
    cap = 0
    while True:
        lv = np.zeros(max(cap, 1), dtype=np.int32)
        og = np.zeros((max(cap, 1), 3), dtype=np.int64)
        pa = np.zeros(max(cap, 1), dtype=np.int32)
        mp = np.zeros((max(cap, 1), 3), dtype=np.int32)
        rc = L.fx_regrid_plan_host(mesh.ndim, mesh.nxb, ip(nroot), ip(bc), mesh.nb, ip(level),
                                   i64p(origin), ip(parent),
                                   err.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   float(refine_cutoff), float(derefine_cutoff), max_level, cap,
                                   ctypes.byref(n), ip(lv), i64p(og), ip(pa), ip(mp), msg, 256)
        if rc == FX_OK:
            return lv[:n.value], og[:n.value], pa[:n.value], mp[:n.value]
        if rc == -1 and n.value > cap:   # FX_ERR_ARG: capacity below the count
            cap = n.value
            continue
        raise FxError(rc, msg.value.decode())


def fx_dword_selftest(op: int, a, b=None, stream=None):
    """One double-word operation element by element on device tensors of
    doubles (fx_dword_selftest); returns the result tensor."""
    import torch
    out = torch.empty_like(a)
    bp = b.data_ptr() if b is not None else None
    rc = load().fx_dword_selftest(int(op), a.data_ptr(), bp, out.data_ptr(), int(a.numel()),
                                  _stream_ptr(stream))
    if rc != FX_OK:
        raise FxError(rc, "fx_dword_selftest")
    return out


def fx_fma_probe(precision: int, ctas: int, iters: int, out_ptr: int, stream=None) -> float:
    """Launch the FMA throughput probe (fx_fma_probe) on ``stream``; returns the
    flops the launch performs (time it with events on the same stream)."""
    flops = ctypes.c_double(0.0)
    rc = load().fx_fma_probe(int(precision), int(ctas), int(iters), ctypes.c_void_p(out_ptr),
                             _stream_ptr(stream), ctypes.byref(flops))
    if rc != FX_OK:
        raise FxError(rc, "fx_fma_probe")
    return flops.value


# ---------------------------------------------------------------- convenience

class BlockSet:
    """One block set with its two device state buffers (torch tensors)."""

    def __init__(self, mesh, gamma: float = 1.4, precision: int = FX_F64, device="cuda",
                 options: dict | None = None, ctx=None):
        import torch
        if not torch.cuda.is_available():
            raise FxError(-2, "no CUDA device: libfx has no CPU path")
        self.mesh = mesh
        self.precision = precision
        self.dtype = torch.float64 if precision == FX_F64 else torch.float32
        self.own_ctx = ctx is None
        self.ctx = ctx if ctx is not None else fx_init(gamma, mesh.nxb, mesh.ng)
        if getattr(mesh, "species", ()) or ctx is None:
            fx_set_species(self.ctx, getattr(mesh, "species", ()))
        for k, v in (options or {}).items():
            fx_set_option(self.ctx, k, v)
        self.U = [torch.zeros(mesh.shape, dtype=self.dtype, device=device) for _ in range(2)]
        self.dt = torch.zeros(1, dtype=torch.float64, device=device)
        self.bs = fx_blocks_create(self.ctx, mesh, precision, self.U[0].data_ptr(),
                                   self.U[1].data_ptr())

    def close(self):
        if getattr(self, "bs", None):
            fx_blocks_destroy(self.bs)
            self.bs = None
        if getattr(self, "own_ctx", False) and getattr(self, "ctx", None):
            fx_finalize(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def current(self):
        return self.U[fx_blocks_current(self.bs)]

    def set_primitive(self, W, stream=None):
        """Primitive state ``W`` [nb, nvar, PZ, P, P] (numpy array, or a torch
        tensor -- page-locked host memory is copied asynchronously)."""
        import torch
        if isinstance(W, torch.Tensor):
            Wd = W.to(device=self.U[0].device, dtype=torch.float64, non_blocking=True)
        else:
            Wd = torch.as_tensor(np.ascontiguousarray(W, dtype=np.float64), device=self.U[0].device)
        fx_prim_to_cons(self.ctx, self.bs, Wd.data_ptr(), stream)
        torch.cuda.current_stream().synchronize()

    def set_conserved(self, U: np.ndarray):
        import torch
        self.current.copy_(torch.as_tensor(U, dtype=self.dtype))
        fx_blocks_mark_dirty(self.bs)

    def fill(self, stream=None):
        fx_guardcell_fill(self.ctx, self.bs, stream)

    def compute_dt(self, cfl: float = 0.8, stream=None) -> float:
        fx_compute_dt(self.ctx, self.bs, cfl, self.dt.data_ptr(), stream)
        return float(self.dt.item())

    def advance(self, dt: float | None = None, stream=None):
        if dt is not None:
            self.dt.fill_(dt)
        fx_hydro_advance(self.ctx, self.bs, self.dt.data_ptr(), stream)

    def step(self, cfl: float = 0.8, stream=None):
        fx_step(self.ctx, self.bs, cfl, self.dt.data_ptr(), stream)

    def run(self, nsteps: int, cfl: float = 0.8, stream=None):
        for _ in range(nsteps):
            self.step(cfl, stream)

    def interior_shape(self) -> tuple:
        m = self.mesh
        return (m.nb, m.nvar, m.nxb if m.ndim == 3 else 1, m.nxb, m.nxb)

    def run_host_interior(self, host_in: np.ndarray, host_out: np.ndarray, nsteps: int = 1,
                          cfl: float = 0.8, stream=None, want_time: bool = False):
        """fx_run_host_interior with shape and dtype checks: ``host_in`` and
        ``host_out`` are C-contiguous ``interior_shape()`` arrays of the block
        set's element type (page-locked memory recommended)."""
        want = np.dtype(np.float64 if self.precision == FX_F64 else np.float32)
        for a in (host_in, host_out):
            if a.shape != self.interior_shape() or a.dtype != want or not a.flags.c_contiguous:
                raise ValueError(f"expected a C-contiguous {want} array of shape "
                                 f"{self.interior_shape()}, got {a.dtype} {a.shape}")
        return fx_run_host_interior(self.ctx, self.bs, host_in, host_out, nsteps, cfl, stream,
                                    want_time)

    def regrid(self, refine_cutoff: float = 0.8, derefine_cutoff: float = 0.2,
               filt: float = 0.01, max_level: int | None = None, stream=None) -> bool:
        """Adapt the mesh to the current state (fx_regrid_plan, new state
        buffers, fx_regrid_apply).  ``self.mesh`` and the buffers follow.
        Returns whether the mesh changed; the indicator of the old mesh's
        blocks is kept in ``self.last_errors``."""
        import dataclasses
        import torch
        L = load()
        m = self.mesh
        max_level = int(m.level.max()) + 1 if max_level is None else int(max_level)
        nn = ctypes.c_int(0)
        _check(self.ctx, L.fx_regrid_plan(self.ctx, self.bs, float(refine_cutoff),
                                          float(derefine_cutoff), float(filt), max_level,
                                          _stream_ptr(stream), ctypes.byref(nn)))
        err = np.zeros(m.nb)
        _check(self.ctx, L.fx_regrid_errors(self.bs, err.ctypes.data_as(
            ctypes.POINTER(ctypes.c_double))))
        self.last_errors = err
        n = nn.value
        level = np.zeros(n, dtype=np.int32)
        origin = np.zeros((n, 3), dtype=np.int64)
        parent = np.zeros(n, dtype=np.int32)
        _check(self.ctx, L.fx_regrid_mesh(self.bs, level.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                          origin.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                          parent.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
        changed = not (n == m.nb and np.array_equal(level, m.level)
                       and np.array_equal(origin, m.origin) and np.array_equal(parent, m.parent))
        new_mesh = dataclasses.replace(m, level=level, origin=origin, parent=parent, extra={})
        dev = self.U[0].device
        U = [torch.zeros(new_mesh.shape, dtype=self.dtype, device=dev) for _ in range(2)]
        _check(self.ctx, L.fx_regrid_apply(self.ctx, self.bs, ctypes.c_void_p(U[0].data_ptr()),
                                           ctypes.c_void_p(U[1].data_ptr()),
                                           _stream_ptr(stream)))
        self.U = U
        self.mesh = new_mesh
        return changed

    def totals(self, stream=None) -> np.ndarray:
        return fx_conserved_totals(self.ctx, self.bs, stream, self.mesh.nvar)

    def status(self) -> int:
        return fx_status(self.ctx, self.bs)

    def state(self) -> np.ndarray:
        return self.current.double().cpu().numpy()
