"""GPU parity of the double-word update (fx_set_option "f64_arith" = 1).

An FP64 block set updated in double-word arithmetic (pairs of FP32 numbers,
about 2^-47 relative precision) is held to the same tolerances against the
FP64 oracle as the FP64 update: 1e-12 relative per cell after one step, 1e-10
after 100 steps.  The momentum components share one scale, the largest
momentum magnitude (``max_rel_err_vec``): a component that vanishes over the
whole domain, like m_z of the 3D shear layer after one step (at most 3e-4),
would otherwise have its absolute roundoff judged against its own vanishing
maximum.  A separate check shows that the mode is really in use (its result
differs from the FP64 update's, by roundoff only).
"""
import numpy as np
import pytest

from tests.helpers import max_rel_err_vec
from tests.test_parity_gpu import CASES, both_start

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DW = {"f64_arith": 1}


@pytest.fixture(scope="module")
def fx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_11630_gb300 import fx as _fx
    _fx.load()
    return _fx


@pytest.mark.parametrize("case", sorted(CASES))
def test_dword_one_step(orc, fx, case):
    mesh, W = CASES[case]()
    om, U, bs = both_start(orc, fx, mesh, W, options=DW)
    bs.set_conserved(U)
    Uo, dto = om.step(U)
    bs.step(0.8)
    assert bs.status() == 0
    # the first dt comes from the FP64 reduction of the uploaded state
    assert float(bs.dt.item()) == pytest.approx(dto, rel=1e-15)
    err = max_rel_err_vec(mesh, bs.state(), Uo)
    assert err <= 1e-12, err
    bs.close()


@pytest.mark.parametrize("case", ["sod2d", "kh64", "amr_sedov_small", "amr_3level_periodic",
                                  "smooth3d_nxb32", "reflect3d_mixed", "amr_2d_reflect_wall"])
def test_dword_100_steps(orc, fx, case):
    mesh, W = CASES[case]()
    om, U, bs = both_start(orc, fx, mesh, W, options=DW)
    bs.set_conserved(U)
    Uo, _, _ = om.run(U, nsteps=100)
    bs.run(100, 0.8)
    assert bs.status() == 0
    err = max_rel_err_vec(mesh, bs.state(), Uo)
    assert err <= 1e-10, err
    bs.close()


def test_dword_mode_is_in_use(orc, fx):
    """Same start, one step each way: the double-word result is not the FP64
    update's bit for bit, and the two agree to roundoff."""
    mesh, W = CASES["kh64"]()
    _, U, native = both_start(orc, fx, mesh, W)
    _, _, dword = both_start(orc, fx, mesh, W, options=DW)
    native.set_conserved(U)
    dword.set_conserved(U)
    native.step(0.8)
    dword.step(0.8)
    a, b = dword.state(), native.state()
    assert not np.array_equal(mesh.interior(a), mesh.interior(b))
    assert max_rel_err_vec(mesh, a, b) <= 1e-13
    native.close()
    dword.close()


def test_dword_host_round_trip(fx):
    """The overlapped host path (fx_run_host_interior) takes the option too:
    its result equals stepping the same block set kind on the device."""
    mesh, W = CASES["kh64"]()
    bs = fx.BlockSet(mesh, 1.4, options=DW)
    bs.set_primitive(W)
    ref = fx.BlockSet(mesh, 1.4, options=DW)
    ref.set_primitive(W)
    host_in = torch.from_numpy(np.ascontiguousarray(mesh.interior(bs.state()))).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    bs.run_host_interior(host_in.numpy(), host_out.numpy(), 3, 0.8)
    ref.run(3, 0.8)
    assert np.array_equal(host_out.numpy(), mesh.interior(ref.state()))
    bs.close()
    ref.close()


def test_dword_option_values(fx):
    ctx = fx.fx_init(1.4, 16, 4)
    try:
        for bad in (3, -1, 0.5):     # 0 FP64, 1 double-word, 2 FP32 arithmetic
            with pytest.raises(fx.FxError):
                fx.fx_set_option(ctx, "f64_arith", bad)
        fx.fx_set_option(ctx, "f64_arith", 2)
        fx.fx_set_option(ctx, "f64_arith", 1)
        fx.fx_set_option(ctx, "f64_arith", 0)
    finally:
        fx.fx_finalize(ctx)


def test_dword_requests_in_a_batch(orc, fx):
    """Double-word FP64 requests share a batch with FP64 and FP32-bulk ones:
    each double-word request equals the same block set stepped alone (within
    roundoff of the differently compiled batched kernel) and the oracle, the
    FP64 request is untouched by its neighbours' mode, and the tuner picks a
    launch for the double-word class."""
    from paper_2208_11630_gb300 import inputs
    from tests.test_batch_gpu import _cases
    from tests.test_oracle_scheme import mesh_2level
    by_name = {c[0]: c for c in _cases()}
    m_sed = mesh_2level(4, 16, 4)
    reqs = [  # (name, mesh, W, precision, steps, double-word)
        ("kh_dw", *by_name["kh_f64"][1:3], 0, 7, True),
        ("amr_dw", *by_name["amr_f64"][1:3], 0, 5, True),
        ("sedov_dw", m_sed, inputs.sedov_state(m_sed), 0, 6, True),
        ("kh_f64", *by_name["kh_f64"][1:3], 0, 7, False),
        ("kh_f32", *by_name["kh_f32"][1:3], 1, 8, False),
    ]
    ctx = fx.fx_init(1.4, 16, 4)
    batch = fx.Batch(ctx, 8)
    sets, slots = [], []
    for name, mesh, W, prec, k, dwm in reqs:
        bs = fx.BlockSet(mesh, 1.4, precision=prec, options=DW if dwm else None)
        bs.set_primitive(W)
        slots.append(batch.add(bs, 0.8, k))
        sets.append(bs)
    batch.tune()
    tile, ctas = batch.choice(3, 2)
    assert tile in (8, 16) and ctas >= 1
    batch.run(max(r[4] for r in reqs) + 1)
    for (name, mesh, W, prec, k, dwm), bs, slot in zip(reqs, sets, slots):
        batch.remove(slot)
        assert bs.status() == 0, name
        ref = fx.BlockSet(mesh, 1.4, precision=prec, options=DW if dwm else None)
        ref.set_primitive(W)
        ref.run(k, 0.8)
        tol = 1e-5 if prec == 1 else 1e-12
        assert max_rel_err_vec(mesh, bs.state(), ref.state()) <= tol, name
        if prec == 0:
            om = orc.OracleMesh(mesh)
            Uo, _, _ = om.run(om.prim_to_cons(W), nsteps=k)
            assert max_rel_err_vec(mesh, bs.state(), Uo) <= 1e-12, name
        bs.close()
        ref.close()
    batch.close()
    fx.fx_finalize(ctx)


@pytest.mark.parametrize("integrator", [1, 2])
@pytest.mark.parametrize("case", ["sod2d", "kh64", "amr_sedov_small", "amr_2d_reflect_wall"])
def test_dword_ssp_rk(orc, fx, case, integrator):
    """SSP-RK2 / SSP-RK3 stages in double-word arithmetic against the oracle's
    integrator: one step at 1e-12, thirty more at 1e-10."""
    mesh, W = CASES[case]()
    om, U, bs = both_start(orc, fx, mesh, W, options={"integrator": integrator, **DW})
    bs.set_conserved(U)
    Uo, dto = om.step(U, integrator=integrator)
    bs.step(0.8)
    assert bs.status() == 0
    assert float(bs.dt.item()) == pytest.approx(dto, rel=1e-15)
    assert max_rel_err_vec(mesh, bs.state(), Uo) <= 1e-12
    Uo2, _, _ = om.run(Uo, nsteps=30, integrator=integrator)
    bs.run(30, 0.8)
    assert bs.status() == 0
    assert max_rel_err_vec(mesh, bs.state(), Uo2) <= 1e-10
    bs.close()


@pytest.mark.parametrize("case", ["smooth3d_2sp", "amr_3sp", "blocky2d_4sp",
                                  "smooth3d_1sp_nxb8"])
def test_dword_species(orc, fx, case):
    """The multispecies update in double-word arithmetic against the oracle:
    one step at 1e-12, twenty more at 1e-10."""
    from tests.test_species_gpu import CASES as SP_CASES
    mesh, W = SP_CASES[case]()
    om = orc.OracleMesh(mesh)
    U = om.prim_to_cons(W)
    bs = fx.BlockSet(mesh, 1.4, options=DW)
    bs.set_conserved(U)
    Uo, dto = om.step(U)
    bs.step(0.8)
    assert bs.status() == 0
    assert float(bs.dt.item()) == pytest.approx(dto, rel=1e-15)
    assert max_rel_err_vec(mesh, bs.state(), Uo) <= 1e-12
    Uo2, _, _ = om.run(Uo, nsteps=20)
    bs.run(20, 0.8)
    assert bs.status() == 0
    assert max_rel_err_vec(mesh, bs.state(), Uo2) <= 1e-10
    bs.close()


def test_dword_operations_within_their_bounds(fx):
    """Each double-word operation against FP64 on 2^18 random operands with
    magnitudes log-uniform over 1e-15..1e15 and both signs: the error of the
    result, relative to the scale the operation's bound refers to, stays
    within a few units of 2^-47 (the conversion within 2^-48)."""
    rng = np.random.default_rng(2024)
    n = 1 << 18

    def draw(signed=True):
        x = 10.0 ** rng.uniform(-15, 15, n)
        return x * (rng.choice([-1.0, 1.0], n) if signed else 1.0)

    a, b, pos = draw(), draw(), draw(signed=False)
    dev = lambda x: torch.from_numpy(x).cuda()
    run = lambda op, x, y=None: fx.fx_dword_selftest(op, dev(x), None if y is None else dev(y)).cpu().numpy()
    u = 2.0 ** -47
    checks = [  # op, inputs, exact (FP64) result, scale of the bound, bound in units of u
        (6, (a,), a, np.abs(a), 0.5),
        (0, (a, b), a + b, np.abs(a) + np.abs(b), 4),
        (1, (a, b), a - b, np.abs(a) + np.abs(b), 4),
        (2, (a, b), a * b, np.abs(a * b), 4),
        (3, (a, b), a / b, np.abs(a / b), 16),
        (4, (pos,), np.sqrt(pos), np.sqrt(pos), 4),
        (5, (pos,), 1.0 / np.sqrt(pos), 1.0 / np.sqrt(pos), 8),
        (7, (a, b), a * b + a, np.abs(a * b) + np.abs(a), 8),
    ]
    for op, args, exact, scale, k in checks:
        got = run(op, *args)
        err = np.abs(got - exact) / scale
        print(f"op {op}: max error {err.max() / u:.3f} x 2^-47 (bound {k})")
        # FP64's own rounding of the reference is 2^-53, far inside the bound
        assert err.max() <= k * u, (op, err.max() / u)
    with pytest.raises(fx.FxError):
        fx.fx_dword_selftest(9, dev(a), dev(b))
