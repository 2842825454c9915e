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
