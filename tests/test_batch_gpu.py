"""Batched, graph-replayed stepping of many block sets (fx_batch_*).

Checks: a batch of mixed requests (2D/3D, uniform/AMR, FP64/FP32-bulk,
nxb 8/16/32, different block counts and step counts) gives, per request, the
same state as stepping that block set alone and, for FP64, the oracle, both
within the parity tolerance 1e-12 (the batched and single-set kernels are the
same device code but compiled in different kernels, so FMA contraction may
round differently); a request's result is bit-identical alone and in the mix;
finished requests stop; tuning leaves every state unchanged.
"""
import numpy as np
import pytest

from paper_2208_11630_gb300 import inputs
from tests.helpers import leaf_interior, max_rel_err, max_rel_err_vec
from tests.test_oracle_scheme import _wall_problem, mesh_2level

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_11630_gb300 import fx as _fx
    _fx.load()
    return _fx


def _cases():
    m_kh = inputs.uniform_mesh(3, (3, 2, 2), 16, 4, inputs.PERIODIC)
    m_sod = inputs.uniform_mesh(2, (8, 4), 16, 4, inputs.OUTFLOW)
    m_amr = mesh_2level(4, 8, 4, inputs.PERIODIC)
    m_sed = mesh_2level(4, 16, 4)
    m_32 = inputs.uniform_mesh(3, (2, 1, 1), 32, 4, inputs.PERIODIC)
    m_8 = inputs.uniform_mesh(3, (3, 3, 2), 8, 4, inputs.OUTFLOW)
    m_wall, W_wall = _wall_problem(3, (2, 2, 2), 8, (0,), lambda c: c[0] == 0 and c[1] == 1,
                                   24)[:2]
    return [
        ("kh_f64", m_kh, inputs.kh_state(m_kh), 0, 7),
        ("sod_f64", m_sod, inputs.sod_state(m_sod), 0, 12),
        ("amr_f64", m_amr, inputs.random_smooth_state(m_amr, 3), 0, 5),
        ("sedov_f32", m_sed, inputs.sedov_state(m_sed), 1, 6),
        ("nxb32_f32", m_32, inputs.random_smooth_state(m_32, 4), 1, 9),
        ("nxb8_f64", m_8, inputs.random_blocky_state(m_8, 5), 0, 4),
        ("kh_f32", m_kh, inputs.kh_state(m_kh), 1, 8),
        ("reflect_f64", m_wall, W_wall, 0, 6),
        ("reflect_f32", m_wall, W_wall, 1, 5),
    ]


def _blockset(fx, mesh, W, prec, ctx=None):
    bs = fx.BlockSet(mesh, 1.4, precision=prec, ctx=ctx)
    bs.set_primitive(W)
    return bs


def test_batch_matches_single_and_oracle(orc, fx):
    cases = _cases()
    ctx = fx.fx_init(1.4, 16, 4)
    batch = fx.Batch(ctx, 16)
    sets, slots = [], []
    for name, mesh, W, prec, k in cases:
        bs = _blockset(fx, mesh, W, prec)
        slots.append(batch.add(bs, 0.8, k))
        sets.append(bs)
    kmax = max(c[4] for c in cases)
    batch.run(kmax + 2)                  # extra steps: finished requests must stop
    assert np.all(batch.poll()[:len(cases)] == 0)
    for (name, mesh, W, prec, k), bs, slot in zip(cases, sets, slots):
        batch.remove(slot)
        assert bs.status() == 0, name
        ref = _blockset(fx, mesh, W, prec)
        ref.run(k, 0.8)
        got, want = bs.state(), ref.state()
        tol = 1e-12 if prec == 0 else 1e-5   # FP32-bulk: FP32 rounding differences
        assert max_rel_err_vec(mesh, got, want) <= tol, name
        if prec == 0:
            om = orc.OracleMesh(mesh)
            Uo, _, _ = om.run(om.prim_to_cons(W), nsteps=k)
            assert max_rel_err(mesh, got, Uo) <= 1e-12, name
        # a released block set continues on its own (fused dt carried over)
        bs.step(0.8)
        ref.step(0.8)
        assert max_rel_err_vec(mesh, bs.state(), ref.state()) <= tol, name
    batch.close()
    fx.fx_finalize(ctx)


def test_alone_equals_in_the_mix_bitwise(fx):
    cases = _cases()
    name, mesh, W, prec, k = cases[0]
    ctx = fx.fx_init(1.4, 16, 4)
    alone = fx.Batch(ctx, 4)
    a = _blockset(fx, mesh, W, prec)
    sa = alone.add(a, 0.8, k)
    alone.run(k)
    alone.remove(sa)
    mix = fx.Batch(ctx, 16)
    others = []
    for c in cases[1:]:
        bs = _blockset(fx, c[1], c[2], c[3])
        mix.add(bs, 0.8, c[4])
        others.append(bs)
    b = _blockset(fx, mesh, W, prec)
    sb = mix.add(b, 0.8, k)
    mix.run(k)
    mix.remove(sb)
    assert np.array_equal(a.state(), b.state())
    alone.close()
    mix.close()
    fx.fx_finalize(ctx)


def test_tuning_leaves_states_unchanged_and_picks_a_choice(fx):
    ctx = fx.fx_init(1.4, 16, 4)
    batch = fx.Batch(ctx, 8)
    sets, slots = [], []
    cases = _cases()[:4]
    for name, mesh, W, prec, k in cases:
        bs = _blockset(fx, mesh, W, prec)
        slots.append(batch.add(bs, 0.8, 3))
        sets.append(bs)
    cur = [bs.state() for bs in sets]
    report = batch.tune()
    assert report, "tuner timed no candidate"
    for (t, c, us) in report:
        assert t in (8, 16) and c >= 1 and us > 0
    for (name, mesh, W, prec, k), bs, c0 in zip(cases, sets, cur):
        # leaf interiors of the current state are untouched (the tuner fills
        # guards and parents, and the other buffer may receive a copy)
        assert np.array_equal(leaf_interior(mesh, bs.state()), leaf_interior(mesh, c0)), name
    tile, ctas = batch.choice(3, 0)
    assert tile in (8, 16)
    batch.run(3)
    assert np.all(batch.poll()[:4] == 0)
    # whatever tile the tuner picked, results equal the single-set path
    for (name, mesh, W, prec, k), bs, slot in zip(cases, sets, slots):
        batch.remove(slot)
        ref = _blockset(fx, mesh, W, prec)
        ref.run(3, 0.8)
        tol = 1e-12 if prec == 0 else 1e-5
        assert max_rel_err_vec(mesh, bs.state(), ref.state()) <= tol, name
    batch.close()
    fx.fx_finalize(ctx)


def test_large_requests_step_through_the_per_set_kernels(orc, fx):
    """A request with at least one full wave of the per-block-set update's
    CTAs (2 per SM for FP64 16x16 tiles, 4 for FP32-bulk; one tile per 16^3
    block) is stepped by the per-block-set kernels of every phase (those of
    fx_step) on a branch of the batch graph, its buffers alternating between
    the two captured graphs; so its batched state is bitwise that of stepping
    it alone.  Covered: FP64 and FP32-bulk uniform requests and an FP64 AMR
    one (copies, prolongation, reflux, restriction) beside small requests in
    the batched phases, step counts of both parities, a request admitted after
    an odd number of replays (re-capture from the device's buffer parity),
    finished requests left in the graph while others run on, and release back
    to single-set stepping; the AMR request also against the oracle."""
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    m64 = inputs.uniform_mesh(3, (8, 8, 5), 16, 4, inputs.PERIODIC)
    m32 = inputs.uniform_mesh(3, (8, 8, 10), 16, 4, inputs.PERIODIC)
    mamr = mesh_2level(6, 16, 4, central=4)
    if m64.nb < 2 * nsm or m32.nb < 4 * nsm or int(mamr.is_leaf().sum()) < 2 * nsm:
        pytest.skip("meshes smaller than one wave on this GPU")
    big = [("big_f64", m64, inputs.kh_state(m64), 0, 5),
           ("big_f32", m32, inputs.kh_state(m32), 1, 4)]
    small = _cases()[:3]
    late = ("big_amr_f64", mamr, inputs.sedov_state(mamr), 0, 3)
    ctx = fx.fx_init(1.4, 16, 4)
    batch = fx.Batch(ctx, 8)
    entries = []
    for c in big + small:
        bs = _blockset(fx, c[1], c[2], c[3])
        entries.append((c, bs, batch.add(bs, 0.8, c[4])))
    batch.run(1)                          # odd: the next capture starts from parity 1
    bs = _blockset(fx, late[1], late[2], late[3])
    entries.append((late, bs, batch.add(bs, 0.8, late[4])))
    batch.run(11)                         # everyone finishes (the small ones take up to 12)
    assert np.all(batch.poll()[:len(entries)] == 0)
    for (name, mesh, W, prec, k), bs, slot in entries:
        assert batch.path(slot) == (1 if name.startswith("big") else 0), name
    for (name, mesh, W, prec, k), bs, slot in entries:
        batch.remove(slot)
        assert bs.status() == 0, name
        ref = _blockset(fx, mesh, W, prec)
        ref.run(k, 0.8)
        tol = 1e-12 if prec == 0 else 1e-5
        if name.startswith("big"):
            assert np.array_equal(bs.state(), ref.state()), name
        else:
            assert max_rel_err_vec(mesh, bs.state(), ref.state()) <= tol, name
        if "amr" in name:
            om = orc.OracleMesh(mesh)
            Uo, _, _ = om.run(om.prim_to_cons(W), nsteps=k)
            assert max_rel_err(mesh, bs.state(), Uo) <= 1e-12, name
        bs.step(0.8)                      # released: continues on its own
        ref.step(0.8)
        if name.startswith("big"):
            assert np.array_equal(bs.state(), ref.state()), name
        else:
            assert max_rel_err_vec(mesh, bs.state(), ref.state()) <= tol, name
        bs.close()
        ref.close()
    batch.close()
    fx.fx_finalize(ctx)


def test_empty_batch_and_refused_requests(fx):
    """A batch with no requests replays an empty step and polls as all-empty
    slots; block sets the batch does not step (SSP-RK, species, the FP32
    arithmetic ablation) are refused at admission with FX_ERR_ARG."""
    ctx = fx.fx_init(1.4, 16, 4)
    batch = fx.Batch(ctx, 4)
    batch.run(3)
    assert np.all(batch.poll() == -1)
    m = inputs.uniform_mesh(3, (2, 2, 2), 16, 4, inputs.PERIODIC)
    for opts in ({"integrator": 1}, {"f64_arith": 2}):
        bs = fx.BlockSet(m, 1.4, options=opts)
        bs.set_primitive(inputs.kh_state(m))
        with pytest.raises(fx.FxError):
            batch.add(bs, 0.8, 1)
        bs.close()
    # after the refusals the batch still steps an admitted request
    bs = _blockset(fx, m, inputs.kh_state(m), 0)
    slot = batch.add(bs, 0.8, 2)
    batch.run(2)
    assert batch.poll()[slot] == 0
    batch.remove(slot)
    assert bs.status() == 0
    bs.close()
    batch.close()
    fx.fx_finalize(ctx)
