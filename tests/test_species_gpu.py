"""GPU parity of the multispecies perfect gas (fx_set_species) against the
oracle: mixture-gamma EOS, advected mass fractions, species fluxes in HLLC,
species guard cells, flux correction and regridding -- one step at 1e-12,
many steps at 1e-10 (FP64), FP32-bulk at 1e-5, species totals conserved;
the single-gas-only paths refuse multispecies block sets."""
import dataclasses

import numpy as np
import pytest

from paper_2208_11630_gb300 import inputs
from tests.helpers import leaf_interior, max_rel_err, max_rel_err_vec
from tests.test_oracle_scheme import mesh_2level

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

AIR_HE = ((1.4, 28.96), (5.0 / 3.0, 4.0))
FOUR = ((1.4, 28.0), (5.0 / 3.0, 4.0), (1.3, 16.0), (1.2, 44.0))


@pytest.fixture(scope="module")
def fx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_11630_gb300 import fx as _fx
    _fx.load()
    return _fx


def species_state(mesh, W5, seed):
    """A single-gas primitive state W5 with random smooth-ish mass fractions
    (positive, summing to one) appended."""
    ns = mesh.nspec
    W = np.zeros(mesh.shape)
    W[:, :5] = W5[:, :5]
    rng = np.random.default_rng(seed)
    g, n = mesh.ng, mesh.nxb
    nz = n if mesh.ndim == 3 else 1
    for b in range(mesh.nb):
        x, y, z = mesh.cell_centers(b)
        raw = np.stack([1.0 + 0.8 * np.sin(2 * np.pi * (x * (k + 1) + y * (2 - k) + z) +
                                           rng.uniform(0, 6.3)) *
                        np.ones((nz, n, n)) for k in range(ns)])
        raw = np.abs(raw) + 0.05
        X = raw / raw.sum(axis=0)
        if mesh.ndim == 3:
            W[b, 5:, g:g + n, g:g + n, g:g + n] = X
        else:
            W[b, 5:, 0, g:g + n, g:g + n] = X[:, 0]
    return W


CASES = {
    "smooth3d_2sp": lambda: (lambda m: (m, species_state(m, inputs.random_smooth_state(m, 71), 72)))(
        inputs.uniform_mesh(3, (3, 2, 2), 16, 4, inputs.PERIODIC, species=AIR_HE)),
    "amr_3sp": lambda: (lambda m: (m, species_state(m, inputs.random_smooth_state(m, 73), 74)))(
        dataclasses.replace(mesh_2level(4, 8, 4, inputs.PERIODIC), species=AIR_HE + ((1.3, 16.0),))),
    "blocky2d_4sp": lambda: (lambda m: (m, species_state(m, inputs.random_blocky_state(m, 75), 76)))(
        inputs.uniform_mesh(2, (4, 3), 16, 4, inputs.OUTFLOW, species=FOUR)),
    "smooth3d_1sp_nxb8": lambda: (lambda m: (m, species_state(m, inputs.random_smooth_state(m, 77), 78)))(
        inputs.uniform_mesh(3, (2, 2, 2), 8, 4, inputs.REFLECT, species=((1.4, 28.96),))),
}


def _both(orc, fx, mesh, W, prec=0):
    om = orc.OracleMesh(mesh)
    U = om.prim_to_cons(W)
    bs = fx.BlockSet(mesh, 1.4, precision=prec)
    bs.set_primitive(W)
    return om, U, bs


@pytest.mark.parametrize("case", sorted(CASES))
def test_species_one_and_many_steps(orc, fx, case):
    mesh, W = CASES[case]()
    om, U, bs = _both(orc, fx, mesh, W)
    # EOS conversion: the mixture gamma adds roundings (1/(gamma-1) vs p/(gamma-1))
    np.testing.assert_allclose(leaf_interior(mesh, bs.state()), leaf_interior(mesh, U),
                               rtol=4e-15, atol=1e-300)
    bs.set_conserved(U)
    assert bs.compute_dt(0.8) == pytest.approx(om.compute_dt(U, 0.8), rel=1e-15)
    Uo, dto = om.step(U)
    bs.step(0.8)
    assert bs.status() == 0
    assert float(bs.dt.item()) == pytest.approx(dto, rel=1e-15)
    assert max_rel_err(mesh, bs.state(), Uo) <= 1e-12
    Uo2, _, _ = om.run(Uo, nsteps=20)
    bs.run(20, 0.8)
    assert bs.status() == 0
    err = max_rel_err(mesh, bs.state(), Uo2)
    print(f"\n{case}: 21 steps GPU vs oracle {err:.2e}")
    assert err <= 1e-10
    # the fused next-step dt equals a fresh reduction
    fused = bs.compute_dt(0.8)
    fx.fx_blocks_mark_dirty(bs.bs)
    assert bs.compute_dt(0.8) == pytest.approx(fused, rel=1e-15)
    if mesh.bc[0][0] == inputs.PERIODIC:   # species (and all) totals conserved
        T0, T1 = om.conserved_totals(U), bs.totals()
        A = om.conserved_totals(np.abs(U)) + om.conserved_totals(np.abs(Uo2))
        A = np.where(A == 0, 1.0, A)
        assert np.all(np.abs(T1 - T0) / A <= 1e-13), (T1 - T0) / A
    bs.close()


def test_species_guard_fill(orc, fx):
    mesh, W = CASES["amr_3sp"]()
    om, U, bs = _both(orc, fx, mesh, W)
    bs.set_conserved(U)
    om.guardcell_fill(U)
    bs.fill()
    G = bs.state()
    leaf = mesh.is_leaf().astype(bool)
    np.testing.assert_allclose(G[leaf], U[leaf], rtol=1e-15, atol=1e-300)
    bs.close()


def test_species_two_gas_shock_tube(orc, fx):
    mesh = inputs.uniform_mesh(2, (8, 1), 16, 4, inputs.OUTFLOW,
                               species=((1.4, 1.0), (5.0 / 3.0, 1.0)))
    W = np.zeros(mesh.shape)
    for b in range(mesh.nb):
        x, _, _ = mesh.cell_centers(b)
        left = (x < 0.5)[0]
        W[b, 0, 0, 4:20, 4:20] = np.where(left, 1.0, 0.125)
        W[b, 4, 0, 4:20, 4:20] = np.where(left, 1.0, 0.1)
        W[b, 5, 0, 4:20, 4:20] = np.where(left, 1.0, 0.0)
        W[b, 6, 0, 4:20, 4:20] = np.where(left, 0.0, 1.0)
    om, U, bs = _both(orc, fx, mesh, W)
    bs.set_conserved(U)
    Uo, _, _ = om.run(U, nsteps=60)
    bs.run(60, 0.8)
    assert bs.status() == 0
    assert max_rel_err(mesh, bs.state(), Uo) <= 1e-10
    bs.close()


def test_species_fp32bulk(orc, fx):
    mesh, W = CASES["smooth3d_2sp"]()
    om, U, bs = _both(orc, fx, mesh, W, prec=fx.FX_F32BULK)
    Uo, _ = om.step(U)
    bs.step(0.8)
    assert bs.status() == 0
    err = max_rel_err_vec(mesh, bs.state(), Uo)
    print(f"\nFP32-bulk two species one step: {err:.2e}")
    assert err <= 1e-5
    bs.close()


def test_species_regrid_and_host_round_trip(orc, fx):
    base = inputs.uniform_mesh(3, (4, 4, 4), 8, 4, inputs.OUTFLOW, species=AIR_HE)
    W5 = inputs.sedov_state(dataclasses.replace(base, species=()), e_blast=0.5)
    W = species_state(base, W5, 79)
    om, U, bs = _both(orc, fx, base, W)
    om2, U2, err_o, _ = om.regrid(U, max_level=2)
    bs.regrid(max_level=2)
    assert np.array_equal(bs.mesh.level, om2.mesh.level)
    assert np.array_equal(bs.mesh.origin, om2.mesh.origin)
    leaf = base.is_leaf().astype(bool)
    np.testing.assert_allclose(bs.last_errors[leaf], err_o[leaf], rtol=1e-12, atol=1e-14)
    assert max_rel_err(bs.mesh, bs.state(), U2) <= 1e-14
    # interior-only host round trip with species
    m2 = bs.mesh
    ref = fx.BlockSet(m2, 1.4)
    ref.set_conserved(bs.state())
    host_in = torch.from_numpy(np.ascontiguousarray(m2.interior(bs.state()))).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    bs.run_host_interior(host_in.numpy(), host_out.numpy(), 2, 0.8)
    ref.run(2, 0.8)
    assert np.array_equal(host_out.numpy(), m2.interior(ref.state()))
    bs.close()
    ref.close()


def test_species_refused_by_single_gas_paths(fx):
    mesh, W = CASES["smooth3d_2sp"]()
    bs = fx.BlockSet(mesh, 1.4, options={"integrator": 1})
    bs.set_primitive(W)
    with pytest.raises(fx.FxError):
        bs.step(0.8)
    bs.close()
    bs = fx.BlockSet(mesh, 1.4)
    bs.set_primitive(W)
    ctx = fx.fx_init(1.4, 16, 4)
    batch = fx.Batch(ctx, 2)
    with pytest.raises(fx.FxError):
        batch.add(bs, 0.8, 2)
    batch.close()
    fx.fx_finalize(ctx)
    bs.close()
