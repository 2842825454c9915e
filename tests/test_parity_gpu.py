"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Both sides start from the same seeded primitive inputs and convert them with
their own EOS; every step runs on each side independently (its own dt, guard
fill, update, correction and restriction).  Tolerances: bit-exact for the
guard copies and restriction, 1e-15 relative for prolonged guards and dt,
1e-12 per cell after one step and 1e-10 after 100 steps (relative error
|a - b| / max(|b|, max|b_var|)).
"""
import numpy as np
import pytest

from paper_2208_11630_gb300 import inputs
from tests.helpers import leaf_interior, max_rel_err
from tests.test_oracle_scheme import O_, P_, R_, _wall_problem, mesh_2level, mesh_3level

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_11630_gb300 import fx as _fx
    _fx.load()
    return _fx


def gpu_blockset(fx, mesh, W, gamma=1.4, options=None):
    bs = fx.BlockSet(mesh, gamma=gamma, options=options)
    bs.set_primitive(W)
    return bs


def both_start(orc, fx, mesh, W, gamma=1.4, options=None):
    om = orc.OracleMesh(mesh, gamma)
    U = om.prim_to_cons(W)
    bs = gpu_blockset(fx, mesh, W, gamma, options)
    return om, U, bs


CASES = {
    "sod2d": lambda: inputs.workload("sod2d")[:2],
    "kh64": lambda: (lambda m: (m, inputs.kh_state(m)))(
        inputs.uniform_mesh(3, (4, 4, 4), 16, 4, inputs.PERIODIC)),
    "blocky3d_outflow": lambda: (lambda m: (m, inputs.random_blocky_state(m, 3)))(
        inputs.uniform_mesh(3, (3, 2, 2), 16, 4, inputs.OUTFLOW)),
    "blocky2d_nxb8": lambda: (lambda m: (m, inputs.random_blocky_state(m, 4)))(
        inputs.uniform_mesh(2, (5, 3), 8, 4, inputs.PERIODIC)),
    "smooth3d_nxb32": lambda: (lambda m: (m, inputs.random_smooth_state(m, 5)))(
        inputs.uniform_mesh(3, (2, 1, 2), 32, 4, inputs.PERIODIC)),
    "smooth3d_nxb8_ng2": lambda: (lambda m: (m, inputs.random_smooth_state(m, 6)))(
        inputs.uniform_mesh(3, (3, 3, 2), 8, 2, inputs.PERIODIC)),
    # an odd guard width: interior rows start at an odd element offset
    "smooth3d_nxb16_ng3": lambda: (lambda m: (m, inputs.random_smooth_state(m, 24)))(
        inputs.uniform_mesh(3, (2, 2, 1), 16, 3, ((O_, O_), (P_, P_), (P_, P_)))),
    "single_block_periodic": lambda: (lambda m: (m, inputs.random_smooth_state(m, 7)))(
        inputs.uniform_mesh(3, (1, 1, 1), 16, 4, inputs.PERIODIC)),
    "amr_sedov_small": lambda: (lambda m: (m, inputs.sedov_state(m)))(mesh_2level(4, 16, 4)),
    "amr_smooth_periodic": lambda: (lambda m: (m, inputs.random_smooth_state(m, 8)))(
        mesh_2level(4, 8, 4, inputs.PERIODIC)),
    "amr_2d_blocky": lambda: (lambda m: (m, inputs.random_blocky_state(m, 9)))(
        mesh_2level(4, 16, 4, inputs.OUTFLOW, ndim=2)),
    "amr_3level_sedov": lambda: (lambda m: (m, inputs.sedov_state(m)))(mesh_3level()),
    "amr_3level_periodic": lambda: (lambda m: (m, inputs.random_smooth_state(m, 15)))(
        mesh_3level(inputs.PERIODIC)),
    "smooth3d_nxb24": lambda: (lambda m: (m, inputs.random_smooth_state(m, 16)))(
        inputs.uniform_mesh(3, (2, 1, 1), 24, 4, inputs.PERIODIC)),
    "smooth3d_nxb64": lambda: (lambda m: (m, inputs.random_smooth_state(m, 17)))(
        inputs.uniform_mesh(3, (1, 1, 1), 64, 4, inputs.PERIODIC)),
    # reflecting walls: all sides, mixed with outflow and periodic, and with
    # refined blocks against a wall (mirrored prolonged guards)
    "reflect2d_blocky": lambda: (lambda m: (m, inputs.random_blocky_state(m, 18)))(
        inputs.uniform_mesh(2, (4, 3), 16, 4, inputs.REFLECT)),
    "reflect3d_mixed": lambda: (lambda m: (m, inputs.random_smooth_state(m, 19)))(
        inputs.uniform_mesh(3, (3, 2, 2), 16, 4, ((R_, O_), (P_, P_), (O_, R_)))),
    "amr_reflect_wall": lambda: _wall_problem(3, (2, 2, 2), 8, (0,),
                                              lambda c: c[0] == 0 and c[1] == 1, 22)[:2],
    "amr_2d_reflect_wall": lambda: _wall_problem(2, (4, 4), 16, (0, 1),
                                                 lambda c: c[0] == 0 and c[1] in (1, 2), 23)[:2],
}


def guard_mask(mesh):
    g, n = mesh.ng, mesh.nxb
    mask = np.ones(mesh.shape[2:], dtype=bool)
    if mesh.ndim == 3:
        mask[g:g + n, g:g + n, g:g + n] = False
    else:
        mask[:, g:g + n, g:g + n] = False
    return mask


@pytest.mark.parametrize("case", sorted(CASES))
def test_guard_fill(orc, fx, case):
    mesh, W = CASES[case]()
    om, U, bs = both_start(orc, fx, mesh, W)
    np.testing.assert_allclose(bs.state(), U, rtol=1e-15, atol=0)   # EOS conversion
    bs.set_conserved(U)                                               # same bits from here
    om.guardcell_fill(U)
    bs.fill()
    G = bs.state()
    leaf = mesh.is_leaf().astype(bool)
    mask = guard_mask(mesh)
    a, b = G[leaf][:, :, mask], U[leaf][:, :, mask]
    if mesh.level.max() == 0:
        assert np.array_equal(a, b)      # plain copies: bit-exact
    else:
        np.testing.assert_allclose(a, b, rtol=1e-15, atol=1e-300)
    # parents hold the bit-exact restriction of their children
    par = ~leaf
    if par.any():
        om.restrict_parents(U)
        assert np.array_equal(mesh.interior(G)[par], mesh.interior(U)[par])


@pytest.mark.parametrize("case", sorted(CASES))
def test_dt(orc, fx, case):
    mesh, W = CASES[case]()
    om, U, bs = both_start(orc, fx, mesh, W)
    bs.set_conserved(U)
    for form in (0, 1):
        fx.fx_set_option(bs.ctx, "cfl_form", form)
        assert bs.compute_dt(0.8) == pytest.approx(om.compute_dt(U, 0.8, form), rel=1e-15)


@pytest.mark.parametrize("case", sorted(CASES))
def test_one_step(orc, fx, case):
    mesh, W = CASES[case]()
    om, U, bs = both_start(orc, fx, mesh, W)
    bs.set_conserved(U)
    Uo, dto = om.step(U)
    bs.step(0.8)
    assert bs.status() == 0
    assert float(bs.dt.item()) == pytest.approx(dto, rel=1e-15)
    G = bs.state()
    err = max_rel_err(mesh, G, Uo)
    assert err <= 1e-12, err
    par = ~mesh.is_leaf().astype(bool)
    if par.any():   # restricted parents follow their children
        a, b = mesh.interior(G)[par], mesh.interior(Uo)[par]
        s = np.maximum(np.abs(b).max(axis=(0, 2, 3, 4), keepdims=True), 1e-300)
        assert (np.abs(a - b) / np.maximum(np.abs(b), s)).max() <= 1e-12


@pytest.mark.parametrize("case,nsteps", [("sod2d", 50), ("sod2d", 100), ("kh64", 100),
                                         ("amr_sedov_small", 100), ("amr_smooth_periodic", 100),
                                         ("amr_2d_blocky", 100), ("smooth3d_nxb32", 100),
                                         ("amr_3level_sedov", 100), ("amr_3level_periodic", 100),
                                         ("smooth3d_nxb24", 100), ("reflect2d_blocky", 100),
                                         ("reflect3d_mixed", 100), ("amr_reflect_wall", 100),
                                         ("amr_2d_reflect_wall", 100)])
def test_many_steps(orc, fx, case, nsteps):
    mesh, W = CASES[case]()
    om, U, bs = both_start(orc, fx, mesh, W)
    bs.set_conserved(U)
    Uo, t, _ = om.run(U, nsteps=nsteps)
    bs.run(nsteps, 0.8)
    assert bs.status() == 0
    err = max_rel_err(mesh, bs.state(), Uo)
    assert err <= 1e-10, err


def test_advection_100_steps(orc, fx):
    mesh = inputs.uniform_mesh(3, (4, 4, 4), 16, 4, inputs.PERIODIC)
    W = inputs.advection_state(mesh)
    om, U, bs = both_start(orc, fx, mesh, W)
    bs.set_conserved(U)
    Uo, _, _ = om.run(U, nsteps=100)
    bs.run(100, 0.8)
    assert max_rel_err(mesh, bs.state(), Uo) <= 1e-10


class _DevPtr:
    """Borrowed view of library-owned device memory (read-only use)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f8", "data": (ptr, False),
                                         "version": 2, "strides": None}


def test_reflux_registers_and_toggle(orc, fx):
    mesh, W = CASES["amr_smooth_periodic"]()
    for reflux in (1, 0):
        om, U, bs = both_start(orc, fx, mesh, W, options={"reflux": reflux})
        bs.set_conserved(U)
        om.guardcell_fill(U)
        bs.fill()
        dt = 0.5 * om.compute_dt(U)
        Uo, st, bf = om.hydro_advance(U, dt, reflux=bool(reflux), want_bflux=True)
        bs.advance(dt)
        assert max_rel_err(mesh, bs.state(), Uo) <= 1e-12
        torch.cuda.synchronize()
        nchecked = 0
        nf = 2 * mesh.ndim * 5 * mesh.nxb ** (mesh.ndim - 1)
        for b in range(mesh.nb):
            ptr = fx.fx_block_fluxes(bs.bs, b)
            if not ptr:
                continue
            got = torch.as_tensor(_DevPtr(ptr, nf), device="cuda").cpu().numpy()
            got = got.reshape(bf[b].shape)
            scale = np.abs(bf[b]).max(axis=(0, 2), keepdims=True)
            assert np.all(np.abs(got - bf[b]) <= 1e-12 * np.maximum(scale, 1e-300))
            nchecked += 1
        assert nchecked > 0
        if reflux:
            A = om.conserved_totals(np.abs(U))
            assert np.all(np.abs(bs.totals() - om.conserved_totals(U)) / A <= 1e-13)


def test_conservation_and_uniform_state(orc, fx):
    mesh = inputs.uniform_mesh(3, (2, 2, 2), 16, 4, inputs.PERIODIC)
    om, U, bs = both_start(orc, fx, mesh, inputs.kh_state(mesh))
    T0 = bs.totals()
    np.testing.assert_allclose(T0, om.conserved_totals(U), rtol=1e-14, atol=1e-15)
    bs.run(100, 0.8)
    # Roundoff of a conserved total is bounded by a small multiple of eps times
    # the magnitudes summed, at the start and at the end: sum |U(0)| alone is
    # no scale for a component that starts at exactly zero, such as m_z here
    # (v_z = 0 initially; pressure gradients along z make it nonzero).
    A = om.conserved_totals(np.abs(U)) + om.conserved_totals(np.abs(bs.state()))
    assert np.all(np.abs(bs.totals() - T0) / A <= 1e-13)
    for mesh in (mesh_2level(4, 8, 4), inputs.uniform_mesh(2, (3, 2), 16, 4)):
        bs = gpu_blockset(fx, mesh, inputs.uniform_state(mesh))
        U0 = bs.state()
        bs.run(3, 0.8)
        assert np.array_equal(leaf_interior(mesh, bs.state()), leaf_interior(mesh, U0))


def test_run_host_matches_device_path(orc, fx):
    mesh, W = CASES["kh64"]()
    bs = gpu_blockset(fx, mesh, W)
    U0 = bs.state()
    host_in = torch.from_numpy(U0).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    t = fx.fx_run_host(bs.ctx, bs.bs, host_in.numpy(), host_out.numpy(), 3, 0.8, want_time=True)
    bs2 = gpu_blockset(fx, mesh, W)
    bs2.run(3, 0.8)
    assert np.array_equal(host_out.numpy(), bs2.state())
    assert t > 0


@pytest.mark.parametrize("case", ["kh64", "sod2d", "smooth3d_nxb8_ng2", "amr_smooth_periodic",
                                  "amr_2d_reflect_wall"])
def test_run_host_interior_matches_device_path(fx, case):
    """Interior-only host round trip (chunked update with overlapped download
    on single-level meshes, plain path on AMR) equals stepping on the device,
    bit for bit, in both precisions, for one and several steps and for a
    second call on the same block set; the block set continues from it."""
    mesh, W = CASES[case]()
    for prec in (fx.FX_F64, fx.FX_F32BULK):
        bs = fx.BlockSet(mesh, 1.4, precision=prec)
        bs.set_primitive(W)
        ref = fx.BlockSet(mesh, 1.4, precision=prec)
        ref.set_primitive(W)
        U0 = bs.state()
        host_in = torch.from_numpy(np.ascontiguousarray(mesh.interior(U0))).to(bs.dtype)
        host_in = host_in.pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        with pytest.raises(ValueError):       # the element type is checked
            wrong = torch.float32 if prec == fx.FX_F64 else torch.float64
            bs.run_host_interior(host_in.to(wrong).numpy(), host_out.numpy())
        for nsteps in (1, 3):
            t = bs.run_host_interior(host_in.numpy(), host_out.numpy(), nsteps, 0.8,
                                     want_time=True)
            fx.fx_blocks_mark_dirty(ref.bs)   # an uploaded state gets a fresh dt reduction
            ref.run(nsteps, 0.8)
            assert t > 0
            assert np.array_equal(host_out.double().numpy(), mesh.interior(ref.state())), \
                (prec, nsteps)
            host_in.copy_(host_out)
        assert bs.status() == 0
        bs.step(0.8)
        ref.step(0.8)
        assert np.array_equal(mesh.interior(bs.state()), mesh.interior(ref.state()))
        bs.close()
        ref.close()


def test_unphysical_state_is_reported(fx):
    """A negative density in the input makes the update non-physical; the
    device latches it, fx_status reports FX_ERR_UNPHYSICAL once and clears."""
    mesh = inputs.uniform_mesh(2, (2, 1), 16, 4, inputs.OUTFLOW)
    W = inputs.uniform_state(mesh, rho=1.0, vel=(0, 0, 0), p=1.0)
    W[1, 0, 0, 8:12, 8:12] = -1.0
    bs = gpu_blockset(fx, mesh, W)
    bs.fill()
    bs.advance(1e-3)
    assert bs.status() == -4
    assert bs.status() == 0


def test_bad_mesh_is_rejected(fx):
    base = inputs.uniform_mesh(3, (4, 4, 4), 8, 4)
    flags = np.zeros(base.nb, dtype=bool)
    flags[0] = True
    m1 = inputs.refine(base, flags)
    # refine the child on the +x side of block 0 again: its level-2 children
    # touch the level-0 block at +x, which violates 2:1 balance
    f2 = np.zeros(m1.nb, dtype=bool)
    f2[base.nb + 1] = True
    m2 = inputs.refine(m1, f2)
    ctx = fx.fx_init(1.4, 8, 4)
    U = [torch.zeros(m2.shape, dtype=torch.float64, device="cuda") for _ in range(2)]
    with pytest.raises(fx.FxError) as e:
        fx.fx_blocks_create(ctx, m2, fx.FX_F64, U[0].data_ptr(), U[1].data_ptr())
    assert e.value.code == -7
    with pytest.raises(fx.FxError):
        fx.fx_set_option(ctx, "no_such_option", 1)
    fx.fx_finalize(ctx)


def test_full_size_kh_sampled(orc, fx):
    """The benchmark workload (256^3, 4096 blocks of 16^3, launch as timed):
    one full step on the GPU, the oracle on a sample of blocks including
    periodic corners."""
    mesh, W, gamma, cfl = inputs.workload("kh3d")
    om = orc.OracleMesh(mesh, gamma)
    U = om.prim_to_cons(W)
    bs = gpu_blockset(fx, mesh, W)
    bs.set_conserved(U)
    del W
    dto = om.compute_dt(U, cfl)
    bs.step(cfl)
    assert bs.status() == 0
    assert float(bs.dt.item()) == pytest.approx(dto, rel=1e-15)
    om.guardcell_fill(U)
    sel = [0, 15, 240, 255, 2048 + 7 * 16 + 9, 3840, 4095, 1234]
    Uo, st, _ = om.hydro_advance(U, dto, select=sel)
    G = bs.current
    for b in sel:
        got = G[b].double().cpu().numpy()
        err = max_rel_err(_one(mesh), got[None], Uo[b][None])
        assert err <= 1e-12, (b, err)


def _one(mesh):
    m = inputs.uniform_mesh(3, (1, 1, 1), mesh.nxb, mesh.ng)
    return m


@pytest.mark.parametrize("case", ["kh64", "sod2d", "amr_smooth_periodic", "amr_sedov_small"])
def test_fused_dt_equals_standalone_reduction(fx, case):
    """After an update the next dt comes from the signal speeds the update
    (and the flux correction) reduced on the fly; it must equal a fresh
    reduction over the stored state."""
    mesh, W = CASES[case]()
    for prec in (fx.FX_F64, fx.FX_F32BULK):
        bs = fx.BlockSet(mesh, 1.4, precision=prec)
        bs.set_primitive(W)
        bs.step(0.8)
        bs.step(0.8)
        fused = bs.compute_dt(0.8)
        fx.fx_blocks_mark_dirty(bs.bs)
        fresh = bs.compute_dt(0.8)
        assert fused == pytest.approx(fresh, rel=1e-15), (prec, fused, fresh)
        bs.close()


def test_full_size_sedov_amr(orc, fx):
    """The Sedov configuration at full size (8^3 coarse blocks of 16^3, 128
    refined, 1024 fine blocks; 1,408 leaves): three fused steps on the GPU
    against the oracle on every leaf, parents included."""
    mesh, W, gamma, cfl = inputs.workload("sedov_amr")
    om = orc.OracleMesh(mesh, gamma)
    U = om.prim_to_cons(W)
    bs = gpu_blockset(fx, mesh, W)
    bs.set_conserved(U)
    Uo, _, _ = om.run(U, nsteps=3)
    bs.run(3, cfl)
    assert bs.status() == 0
    G = bs.state()
    assert max_rel_err(mesh, G, Uo) <= 1e-12
    par = ~mesh.is_leaf().astype(bool)
    a, b = mesh.interior(G)[par], mesh.interior(Uo)[par]
    s = np.maximum(np.abs(b).max(axis=(0, 2, 3, 4), keepdims=True), 1e-300)
    assert (np.abs(a - b) / np.maximum(np.abs(b), s)).max() <= 1e-12


@pytest.mark.parametrize("integrator", [1, 2])
@pytest.mark.parametrize("case", ["sod2d", "kh64", "blocky2d_nxb8", "amr_smooth_periodic",
                                  "amr_sedov_small", "amr_3level_periodic", "smooth3d_nxb32",
                                  "amr_reflect_wall"])
def test_rk2_variant(orc, fx, case, integrator):
    """SSP-RK2 and SSP-RK3 with PLM and HLLC (integrator options 1 and 2)
    against the oracle's: one step at 1e-12, thirty more at 1e-10; totals
    conserved on periodic meshes (stage-weighted flux correction on AMR)."""
    mesh, W = CASES[case]()
    om, U, bs = both_start(orc, fx, mesh, W, options={"integrator": integrator})
    bs.set_conserved(U)
    Uo, dto = om.step(U, integrator=integrator)
    bs.step(0.8)
    assert bs.status() == 0
    assert float(bs.dt.item()) == pytest.approx(dto, rel=1e-15)
    assert max_rel_err(mesh, bs.state(), Uo) <= 1e-12
    Uo2, _, _ = om.run(Uo, nsteps=30, integrator=integrator)
    bs.run(30, 0.8)
    assert bs.status() == 0
    assert max_rel_err(mesh, bs.state(), Uo2) <= 1e-10
    if mesh.bc[0][0] == inputs.PERIODIC:
        # scale: magnitudes at both ends, as in the conservation test above
        A = om.conserved_totals(np.abs(U)) + om.conserved_totals(np.abs(Uo2))
        A = np.where(A == 0, 1.0, A)      # m_z of a 2D run is zero everywhere
        assert np.all(np.abs(bs.totals() - om.conserved_totals(U)) / A <= 1e-13)


@pytest.mark.parametrize("integrator", [1, 2])
def test_rk2_block_sets_are_not_batched(fx, integrator):
    mesh, W = CASES["kh64"]()
    bs = fx.BlockSet(mesh, 1.4, options={"integrator": integrator})
    bs.set_primitive(W)
    ctx = fx.fx_init(1.4, 16, 4)
    batch = fx.Batch(ctx, 2)
    with pytest.raises(fx.FxError):
        batch.add(bs, 0.8, 3)
    batch.close()
    fx.fx_finalize(ctx)


def test_rk3_interior_host_round_trip(fx):
    """SSP-RK3 through the interior-only host path (not chunked: three
    stages) equals stepping on the device, bit for bit."""
    mesh, W = CASES["kh64"]()
    bs = fx.BlockSet(mesh, 1.4, options={"integrator": 2})
    bs.set_primitive(W)
    ref = fx.BlockSet(mesh, 1.4, options={"integrator": 2})
    ref.set_primitive(W)
    host_in = torch.from_numpy(np.ascontiguousarray(mesh.interior(bs.state()))).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    bs.run_host_interior(host_in.numpy(), host_out.numpy(), 2, 0.8)
    ref.run(2, 0.8)
    assert np.array_equal(host_out.numpy(), mesh.interior(ref.state()))
