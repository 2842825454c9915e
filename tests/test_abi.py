"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/fx.h declares.  No compute call is made here (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "fx.h")).read()
    return re.findall(r"^FX_API\s+(?:const\s+)?\w+\s*\**\s*(fx_\w+)\s*\(", text, re.M)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("fx_init", "fx_guardcell_fill", "fx_hydro_advance", "fx_compute_dt",
                     "fx_blocks_create", "fx_status", "fx_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2208_11630_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_no_cpu_fallback_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2208_11630_gb300 import fx
    # the library itself refuses to create a context without a device ...
    with pytest.raises(fx.FxError):
        fx.fx_init(1.4, 16, 4)
    # ... and the Python convenience layer refuses before touching it
    from paper_2208_11630_gb300 import inputs
    mesh = inputs.uniform_mesh(2, (1, 1), 16, 4)
    with pytest.raises(fx.FxError):
        fx.BlockSet(mesh)


def test_null_handles_are_refused_without_a_crash():
    """Every entry point given null handles returns the documented error (or
    NULL) instead of touching the device or dereferencing them; run in a
    child process so that a crash is a failure, not a lost test session."""
    import subprocess
    import sys
    code = r'''
import ctypes, sys
sys.path.insert(0, %r)
from paper_2208_11630_gb300 import _build
L = ctypes.CDLL(_build.build())
d, vp = ctypes.c_double, ctypes.c_void_p
L.fx_last_error.restype = ctypes.c_char_p
L.fx_block_fluxes.restype = vp
L.fx_kernel_launches.restype = ctypes.c_longlong
calls = {
 "fx_init": lambda: L.fx_init(d(1.4), 16, 4, None),
 "fx_set_option": lambda: L.fx_set_option(None, b"cfl_form", d(0)),
 "fx_set_species": lambda: L.fx_set_species(None, 1, None, None),
 "fx_blocks_create": lambda: L.fx_blocks_create(None, 3, 1, 16, None, None, None, None, None,
                                                None, None, 0, None, None, None),
 "fx_blocks_destroy": lambda: L.fx_blocks_destroy(None),
 "fx_blocks_mark_dirty": lambda: L.fx_blocks_mark_dirty(None),
 "fx_blocks_current": lambda: L.fx_blocks_current(None),
 "fx_prim_to_cons": lambda: L.fx_prim_to_cons(None, None, None, None),
 "fx_guardcell_fill": lambda: L.fx_guardcell_fill(None, None, None),
 "fx_guardcell_fill_amr": lambda: L.fx_guardcell_fill_amr(None, None, None),
 "fx_compute_dt": lambda: L.fx_compute_dt(None, None, d(0.8), None, None),
 "fx_hydro_advance": lambda: L.fx_hydro_advance(None, None, None, None),
 "fx_step": lambda: L.fx_step(None, None, d(0.8), None, None),
 "fx_conserved_totals": lambda: L.fx_conserved_totals(None, None, None, None),
 "fx_status": lambda: L.fx_status(None, None),
 "fx_run_host": lambda: L.fx_run_host(None, None, None, None, 1, d(0.8), None, None),
 "fx_run_host_interior": lambda: L.fx_run_host_interior(None, None, None, None, 1, d(0.8),
                                                        None, None),
 "fx_regrid_plan": lambda: L.fx_regrid_plan(None, None, d(0.8), d(0.2), d(0.01), 1, None, None),
 "fx_regrid_errors": lambda: L.fx_regrid_errors(None, None),
 "fx_regrid_mesh": lambda: L.fx_regrid_mesh(None, None, None, None),
 "fx_regrid_apply": lambda: L.fx_regrid_apply(None, None, None, None, None),
 "fx_regrid_plan_host": lambda: L.fx_regrid_plan_host(3, 16, None, None, 1, None, None, None,
                                                      None, d(0.8), d(0.2), 1, 0, None, None,
                                                      None, None, None, None, 0),
 "fx_batch_create": lambda: L.fx_batch_create(None, 4, None),
 "fx_batch_destroy": lambda: L.fx_batch_destroy(None),
 "fx_batch_add": lambda: L.fx_batch_add(None, None, d(0.8), 1, None, None),
 "fx_batch_run": lambda: L.fx_batch_run(None, 1, None),
 "fx_batch_poll": lambda: L.fx_batch_poll(None, None, None),
 "fx_batch_remove": lambda: L.fx_batch_remove(None, 0, None),
 "fx_batch_tune": lambda: L.fx_batch_tune(None, None, None),
 "fx_batch_choice": lambda: L.fx_batch_choice(None, 3, 0, None, None),
 "fx_batch_path": lambda: L.fx_batch_path(None, 0, None),
 "fx_compute_dt_noalloc": lambda: L.fx_compute_dt_noalloc(None, 3, 1, 16, 4, None, d(1.4), d(0.8),
                                                          0, None, None, None, ctypes.c_size_t(0)),
 "fx_dword_selftest": lambda: L.fx_dword_selftest(0, None, None, None, 4, None),
 "fx_fma_probe": lambda: L.fx_fma_probe(0, 1, 1, None, None, None),
}
for name, f in calls.items():
    print(name, f(), flush=True)
print("fx_finalize", L.fx_finalize(None), flush=True)
print("fx_last_error", L.fx_last_error(None).decode(), flush=True)
print("fx_block_fluxes", L.fx_block_fluxes(None, 0), flush=True)
print("fx_kernel_launches", L.fx_kernel_launches(), flush=True)
''' % ROOT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, (r.returncode, r.stdout[-2000:], r.stderr[-2000:])
    got = dict(line.split(" ", 1) for line in r.stdout.strip().splitlines())
    special = {"fx_finalize": "0", "fx_last_error": "null context", "fx_block_fluxes": "None",
               "fx_kernel_launches": "0"}
    for name in declared_symbols():
        assert name in got, name
        assert got[name] == special.get(name, "-1"), (name, got[name])
