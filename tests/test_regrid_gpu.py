"""GPU parity of regridding (fx_regrid_plan / fx_regrid_apply) against the
oracle: the per-leaf indicator (1e-12 relative), the planned mesh (identical
levels, origins and parents -- the two sides implement the marking and the
2:1 balance with different algorithms), the transferred state (1e-14), a
dynamic Sedov run that regrids every few steps (meshes identical at every
regrid, state within 1e-10, mass and energy conserved), hand-worked forced
refinements across a periodic wrap, and FP32-bulk block sets."""
import numpy as np
import pytest

from paper_2208_11630_gb300 import inputs
from tests.helpers import max_rel_err, max_rel_err_vec
from tests.test_oracle_regrid import _state_from_fields, assert_balanced
from tests.test_oracle_scheme import _wall_problem, mesh_2level

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

R_, O_, P_ = inputs.REFLECT, inputs.OUTFLOW, inputs.PERIODIC


@pytest.fixture(scope="module")
def fx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_11630_gb300 import fx as _fx
    _fx.load()
    return _fx


def _cases():
    m_kh = inputs.uniform_mesh(3, (4, 4, 4), 16, 4, P_)
    m_sed = mesh_2level(4, 8, 4)
    m_2d = inputs.uniform_mesh(2, (6, 4), 16, 4, O_)
    m_w, W_w = _wall_problem(3, (2, 2, 2), 8, (0,), lambda c: c[0] == 0 and c[1] == 1, 41)[:2]
    # 32^3 blocks: the indicator's shared-memory window exceeds 48 KB
    m_32 = inputs.uniform_mesh(3, (2, 2, 2), 32, 4, P_)
    return {
        "smooth3d": (m_kh, inputs.random_smooth_state(m_kh, 43)),
        "smooth3d_nxb32": (m_32, inputs.random_smooth_state(m_32, 44)),
        "sedov_amr": (m_sed, inputs.sedov_state(m_sed)),
        "blocky2d": (m_2d, inputs.random_blocky_state(m_2d, 42)),
        "walled_amr": (m_w, W_w),
    }


def _cutoffs(err, lo_q=0.5, hi_q=0.85):
    """Refine / derefine cutoffs placed in gaps of the error distribution,
    so that no block sits within 1e-9 of either."""
    e = np.sort(err[err >= 0])
    def gap_at(q):
        i = int(q * (len(e) - 1))
        for j in range(i, len(e) - 1):
            if e[j + 1] - e[j] > 1e-6:
                return 0.5 * (e[j] + e[j + 1])
        return e[-1] + 1.0
    dc = gap_at(lo_q)
    rc = max(gap_at(hi_q), dc + 1e-6)
    return rc, dc


@pytest.mark.parametrize("case", ["smooth3d", "smooth3d_nxb32", "sedov_amr", "blocky2d",
                                  "walled_amr"])
def test_plan_and_transfer_match_oracle(orc, fx, case):
    mesh, W = _cases()[case]
    bs = fx.BlockSet(mesh, 1.4)
    bs.set_primitive(W)
    U = bs.state()
    om = orc.OracleMesh(mesh)
    # the oracle's indicator on the same state (after its own fill)
    Uf = U.copy()
    om.restrict_parents(Uf)
    om.guardcell_fill(Uf)
    err_o = om.regrid_errors(Uf)
    rc, dc = _cutoffs(err_o)
    om2, U2, err_o2, maps = om.regrid(U, refine_cutoff=rc, derefine_cutoff=dc, max_level=2)
    assert np.array_equal(err_o2, err_o)
    changed = bs.regrid(refine_cutoff=rc, derefine_cutoff=dc, max_level=2)
    err_g = bs.last_errors
    leaf = mesh.is_leaf().astype(bool)
    assert np.all(err_g[~leaf] == -1.0)
    np.testing.assert_allclose(err_g[leaf], err_o[leaf], rtol=1e-12, atol=1e-14)
    m2 = bs.mesh
    assert changed == (om2.mesh.nb != mesh.nb or not np.array_equal(om2.mesh.level, mesh.level))
    print(f"\n{case}: {mesh.nb} -> {m2.nb} blocks, levels {np.bincount(m2.level).tolist()}, "
          f"cutoffs {rc:.4f} / {dc:.4f}")
    assert np.array_equal(m2.level, om2.mesh.level)
    assert np.array_equal(m2.origin, om2.mesh.origin)
    assert np.array_equal(m2.parent, om2.mesh.parent)
    assert_balanced(m2)
    G = bs.state()
    assert max_rel_err(m2, G, U2) <= 1e-14
    np.testing.assert_array_equal(np.isfinite(m2.interior(G)), True)
    # and the new block set steps on
    bs.step(0.8)
    Uo, _ = om2.step(U2)
    assert bs.status() == 0
    assert max_rel_err(m2, bs.state(), Uo) <= 1e-12
    bs.close()


def test_dynamic_sedov_regrid_every_three_steps(orc, fx):
    base = inputs.uniform_mesh(3, (4, 4, 4), 8, 4, O_)
    W = inputs.sedov_state(base, e_blast=1.0, r_cells=2.5)
    bs = fx.BlockSet(base, 1.4)
    bs.set_primitive(W)
    om = orc.OracleMesh(base)
    U = om.prim_to_cons(W)
    T0 = bs.totals()
    nlev = []
    for cycle in range(4):
        om, U, err_o, _ = om.regrid(U, refine_cutoff=0.8, derefine_cutoff=0.2, max_level=2)
        bs.regrid(refine_cutoff=0.8, derefine_cutoff=0.2, max_level=2)
        assert np.array_equal(bs.mesh.level, om.mesh.level), cycle
        assert np.array_equal(bs.mesh.origin, om.mesh.origin), cycle
        assert np.array_equal(bs.mesh.parent, om.mesh.parent), cycle
        nlev.append(np.bincount(bs.mesh.level).tolist())
        U, _, _ = om.run(U, nsteps=3)
        bs.run(3, 0.8)
        assert bs.status() == 0
    err = max_rel_err(bs.mesh, bs.state(), U)
    print(f"\ndynamic Sedov (regrid every 3 steps), levels {nlev}: GPU vs oracle {err:.2e}")
    assert err <= 1e-10
    assert int(bs.mesh.level.max()) == 2
    T1 = bs.totals()
    A = np.abs(T0) + np.abs(T1)
    A = np.where(A == 0, 1.0, A)
    assert abs(T1[0] - T0[0]) / A[0] <= 1e-12 and abs(T1[4] - T0[4]) / A[4] <= 1e-12
    bs.close()


def test_forced_refinement_across_periodic_wrap(fx):
    mesh = inputs.uniform_mesh(2, (4, 4), 8, 4, P_)
    bs = fx.BlockSet(mesh, 1.4)
    bs.set_primitive(_state_from_fields(mesh, lambda X, Y, Z: 1.0 + 0.5 * ((X == 3) & (Y == 4)),
                                        lambda X, Y, Z: np.ones(np.shape(X))))
    bs.regrid(max_level=2)
    m2 = bs.mesh
    assert np.bincount(m2.level).tolist() == [16, 4]
    W2 = _state_from_fields(m2, lambda X, Y, Z: 1.0 + 0.5 * ((X == 1) & (Y == 2)),
                            lambda X, Y, Z: np.ones(np.shape(X)))
    for b in range(m2.nb):
        if m2.level[b] == 0:
            W2[b, 0] = np.where(W2[b, 0] != 0, 1.0, 0.0)
    bs.set_primitive(W2)
    bs.regrid(max_level=2)
    m3 = bs.mesh
    assert_balanced(m3)
    lvl0_refined = sorted(tuple(m3.origin[b, :2] // 8) for b in range(m3.nb)
                          if m3.level[b] == 0 and not m3.is_leaf()[b])
    assert lvl0_refined == [(0, 0), (0, 3), (3, 0), (3, 3)]
    bs.close()


def test_fp32bulk_regrid(orc, fx):
    mesh = mesh_2level(4, 8, 4)
    W = inputs.sedov_state(mesh, e_blast=0.01)
    bs = fx.BlockSet(mesh, 1.4, precision=fx.FX_F32BULK)
    bs.set_primitive(W)
    U = bs.state()                    # FP32 values, as doubles
    om = orc.OracleMesh(mesh)
    om2, U2, err_o, _ = om.regrid(U, max_level=2)
    bs.regrid(max_level=2)
    leaf = mesh.is_leaf().astype(bool)
    np.testing.assert_allclose(bs.last_errors[leaf], err_o[leaf], rtol=1e-12, atol=1e-14)
    assert np.array_equal(bs.mesh.level, om2.mesh.level)
    assert np.array_equal(bs.mesh.origin, om2.mesh.origin)
    # prolongation in FP64, one rounding to FP32
    assert max_rel_err_vec(bs.mesh, bs.state(), U2) <= 1e-7
    bs.step(0.8)
    assert bs.status() == 0
    bs.close()


def test_regrid_refused_inside_a_batch(fx):
    mesh = inputs.uniform_mesh(3, (2, 2, 2), 16, 4, P_)
    bs = fx.BlockSet(mesh, 1.4)
    bs.set_primitive(inputs.kh_state(mesh))
    ctx = fx.fx_init(1.4, 16, 4)
    batch = fx.Batch(ctx, 2)
    slot = batch.add(bs, 0.8, 2)
    with pytest.raises(fx.FxError):
        bs.regrid()
    batch.run(2)
    batch.remove(slot)
    assert bs.regrid(refine_cutoff=2.0, derefine_cutoff=-1.0) is False
    batch.close()
    fx.fx_finalize(ctx)
    bs.close()
