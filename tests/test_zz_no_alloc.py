"""The allocation-free time-step entry point (fx_compute_dt_noalloc).

Some callers cannot call cudaMalloc -- they run inside a host callback or an
allocator's own bookkeeping, share the device with a runtime that owns all of
its memory, or forbid allocation after start-up -- so they cannot create a
block set.  This entry point gives them the same dt as fx_compute_dt for a
single-level array of blocks, from a fixed scratch array inside the library.

These checks call it through the C ABI, twice in a row on different states,
and compare with fx_compute_dt (same tolerance as the dt parity tests).  The
file is named to be collected last.
"""
import numpy as np
import pytest

from paper_2208_11630_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_11630_gb300 import fx as _fx
    _fx.load()
    return _fx


def _reference(fx, mesh, W, form):
    bs = fx.BlockSet(mesh, 1.4, options={"cfl_form": form})
    bs.set_primitive(W)
    dt = bs.compute_dt(0.8)
    return bs, dt


def _cases(ndim):
    if ndim == 3:
        m1 = inputs.uniform_mesh(3, (4, 4, 4), 16, 4, inputs.PERIODIC)
        m2 = inputs.uniform_mesh(3, (3, 2, 2), 16, 4, inputs.OUTFLOW)
        return [(m1, inputs.kh_state(m1)), (m2, inputs.random_blocky_state(m2, 12))]
    # 2D: one z plane, dx[2] unused -- the Sod mesh (64 blocks of 16^2) and an
    # uneven periodic one
    m1, W1, _, _ = inputs.workload("sod2d")
    m2 = inputs.uniform_mesh(2, (5, 3), 8, 4, inputs.PERIODIC)
    return [(m1, W1), (m2, inputs.random_blocky_state(m2, 13))]


@pytest.mark.parametrize("ndim", [3, 2])
@pytest.mark.parametrize("form", [0, 1])
def test_noalloc_dt_matches_library_dt_twice(fx, form, ndim):
    cases = _cases(ndim)
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for mesh, W in cases:       # two calls in a row; the second must not see the first
        bs, want = _reference(fx, mesh, W, form)
        dx = [1.0 / n for n in mesh.cells_per_axis(0)]
        rc, msg = fx.fx_compute_dt_noalloc(bs.current.data_ptr(), mesh.ndim, mesh.nb, mesh.nxb,
                                           mesh.ng, dx, 1.4, 0.8, form, out.data_ptr(), stream)
        assert rc == 0, msg
        got = float(out.item())
        assert got == pytest.approx(want, rel=1e-15)
        bs.close()


def test_noalloc_rejects_more_blocks_than_its_scratch(fx):
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc, msg = fx.fx_compute_dt_noalloc(out.data_ptr(), 3, fx.FX_NOALLOC_MAX_BLOCKS + 1, 16, 4,
                                       [1.0, 1.0, 1.0], 1.4, 0.8, 0, out.data_ptr())
    assert rc == -1
    assert "FX_NOALLOC_MAX_BLOCKS" in msg


@pytest.mark.parametrize("form", [0, 1])
def test_noalloc_dt_is_nan_for_a_cell_without_sound_speed(fx, form):
    """A cell with negative pressure early in a block (the first cell a thread
    reduces, followed by finite ones) makes dt NaN from both entry points,
    rather than a finite value that hides it."""
    mesh = inputs.uniform_mesh(3, (2, 2, 2), 16, 4, inputs.PERIODIC)
    W = inputs.uniform_state(mesh, rho=1.0, vel=(0.3, 0.0, 0.0), p=1.0)
    g = mesh.ng
    W[1, 4, g, g, g] = -0.5
    bs, want = _reference(fx, mesh, W, form)
    assert np.isnan(want)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    dx = [1.0 / n for n in mesh.cells_per_axis(0)]
    rc, msg = fx.fx_compute_dt_noalloc(bs.current.data_ptr(), 3, mesh.nb, mesh.nxb, mesh.ng, dx,
                                       1.4, 0.8, form, out.data_ptr(),
                                       torch.cuda.current_stream())
    assert rc == 0, msg
    assert np.isnan(float(out.item()))
    bs.close()
