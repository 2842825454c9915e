"""Pins of the oracle's whole step: guard fill, hydro update, flux correction,
restriction, time step.  Each check compares against something other than the
oracle itself: the exact Riemann solution, conservation, exact invariants,
symmetry, brute-force indexing, textbook special cases and closed forms."""
import numpy as np
import pytest

from paper_2208_11630_gb300 import inputs
from tests.helpers import assemble, leaf_interior, rel_err

GAMMA = 1.4


def mesh_2level(nblk=4, nxb=8, ng=4, bc=inputs.OUTFLOW, central=None, ndim=3):
    """Coarse ``nblk^ndim`` grid with the central ``central^ndim`` blocks
    refined (default: half the blocks per axis)."""
    central = central or nblk // 2
    base = inputs.uniform_mesh(ndim, (nblk,) * ndim, nxb, ng, bc)
    flags = []
    lo = (nblk - central) // 2
    for b in range(base.nb):
        bc_ = base.origin[b] // nxb
        flags.append(all(lo <= bc_[d] < lo + central for d in range(ndim)))
    return inputs.refine(base, np.array(flags))


def mesh_3level(bc=inputs.OUTFLOW, nxb=8):
    """4^3 coarse blocks, the central 2^3 refined, and the central 2^3 of the
    resulting fine blocks refined again (64 blocks per level, 2:1 balanced)."""
    m2 = mesh_2level(4, nxb, 4, bc)
    leaf = m2.is_leaf()
    flags = np.zeros(m2.nb, dtype=bool)
    for b in range(m2.nb):
        if m2.level[b] == 1 and leaf[b]:
            o = m2.origin[b] // nxb
            flags[b] = all(3 <= o[d] < 5 for d in range(3))
    return inputs.refine(m2, flags)


# ------------------------------------------------------------------ guard fill

R_, O_, P_ = inputs.REFLECT, inputs.OUTFLOW, inputs.PERIODIC


@pytest.mark.parametrize("ndim,bc", [(2, inputs.PERIODIC), (2, inputs.OUTFLOW),
                                     (3, inputs.PERIODIC), (3, inputs.OUTFLOW),
                                     (3, ((P_, P_), (O_, O_), (P_, P_))),
                                     (2, inputs.REFLECT),
                                     (3, ((R_, O_), (P_, P_), (O_, R_)))])
def test_guard_fill_brute_force(orc, ndim, bc):
    """Guards of a uniform mesh equal global-array indexing with wrap
    (periodic), clip (outflow) or mirror about the wall with the normal
    momentum negated (reflecting) per side -- bitwise."""
    nblk = (3, 2, 2)[:ndim]
    mesh = inputs.uniform_mesh(ndim, nblk, 8, 4, bc)
    om = orc.OracleMesh(mesh)
    rng = np.random.default_rng(1)
    U = rng.uniform(-1, 1, mesh.shape)
    G = assemble(mesh, U)
    om.guardcell_fill(U)
    N = mesh.cells_per_axis(0)
    bcs = mesh.bc
    for b in range(mesh.nb):
        idx, sign = [], []
        for d in range(3):
            if d >= ndim:
                idx.append(np.zeros(1, dtype=int))
                sign.append(np.ones(1))
                continue
            g = mesh.origin[b, d] + np.arange(mesh.P) - mesh.ng
            sg = np.ones(mesh.P)
            for side, beyond in ((0, g < 0), (1, g >= N[d])):
                kind = bcs[d][side]
                if kind == inputs.PERIODIC:
                    g = np.where(beyond, np.mod(g, N[d]), g)
                elif kind == inputs.REFLECT:
                    g = np.where(beyond, (-1 - g) if side == 0 else (2 * N[d] - 1 - g), g)
                    sg = np.where(beyond, -1.0, sg)
                else:
                    g = np.where(beyond, 0 if side == 0 else N[d] - 1, g)
            idx.append(g)
            sign.append(sg)
        want = G[:, idx[2][:, None, None], idx[1][None, :, None], idx[0][None, None, :]].copy()
        want[1] *= sign[0][None, None, :]
        want[2] *= sign[1][None, :, None]
        want[3] *= sign[2][:, None, None]
        assert np.array_equal(U[b], want)


def test_prolongation_linear_exact(orc):
    """Conservative MC prolongation reproduces a linear field exactly (to
    roundoff) in the guards of fine blocks next to coarse leaves."""
    mesh = mesh_2level(4, 8, 4)
    om = orc.OracleMesh(mesh)
    a = np.array([1.0, -0.5, 0.25, 2.0, 3.0])
    grad = np.array([[0.3, -0.2, 0.1], [0.5, 0.4, -0.6], [-0.2, 0.1, 0.05],
                     [0.7, 0.0, 0.3], [1.0, -1.0, 0.5]])
    U = np.zeros(mesh.shape)

    def lin(b, ii, jj, kk):
        lev = int(mesh.level[b])
        dx = 1.0 / mesh.cells_per_axis(lev)[0]
        x = (mesh.origin[b, 0] + ii - mesh.ng + 0.5) * dx
        y = (mesh.origin[b, 1] + jj - mesh.ng + 0.5) * dx
        z = (mesh.origin[b, 2] + kk - mesh.ng + 0.5) * dx
        return [a[v] + grad[v, 0] * x + grad[v, 1] * y + grad[v, 2] * z for v in range(5)]

    P = mesh.P
    kk, jj, ii = np.meshgrid(np.arange(P), np.arange(P), np.arange(P), indexing="ij")
    for b in range(mesh.nb):
        vals = lin(b, ii, jj, kk)
        for v in range(5):
            U[b, v] = vals[v]
    exact = U.copy()
    U2 = U.copy()
    U2[:, :, :, :, :] = np.where(np.ones_like(U2, dtype=bool), U2, 0)
    # wipe guards, then fill
    g, n = mesh.ng, mesh.nxb
    mask = np.ones(mesh.shape[2:], dtype=bool)
    mask[g:g + n, g:g + n, g:g + n] = False
    U2[:, :, mask] = 0.0
    om.guardcell_fill(U2)
    leaf = mesh.is_leaf()
    checked = 0
    for b in range(mesh.nb):
        if mesh.level[b] != 1 or not leaf[b]:
            continue
        # guard cells within 2 fine cells of the interior have coarse
        # stencils far from the physical boundary
        sel = mask.copy()
        sel[:g - 2] = sel[g + n + 2:] = False
        sel[:, :g - 2] = sel[:, g + n + 2:] = False
        sel[:, :, :g - 2] = sel[:, :, g + n + 2:] = False
        np.testing.assert_allclose(U2[b][:, sel], exact[b][:, sel], rtol=1e-13, atol=1e-13)
        checked += 1
    assert checked == 64


def test_restriction_of_prolongation_is_identity(orc):
    """The 2^d fine guard cells prolonged from one coarse cell average back to
    that coarse cell's value."""
    mesh = mesh_2level(4, 8, 4)
    om = orc.OracleMesh(mesh)
    W = inputs.random_smooth_state(mesh, seed=21)
    U = om.prim_to_cons(W)
    om.guardcell_fill(U)
    n, g = mesh.nxb, mesh.ng
    leaf = mesh.is_leaf()
    # index the coarse leaves by block coordinate
    coarse = {tuple(mesh.origin[b] // n): b for b in range(mesh.nb)
              if mesh.level[b] == 0 and leaf[b]}
    count = 0
    for b in range(mesh.nb):
        if mesh.level[b] != 1:
            continue
        for (ax, side) in [(0, -1), (0, 1), (1, -1), (1, 1), (2, -1), (2, 1)]:
            # face guard slab of depth ng (2 coarse cells)
            sl = [slice(g, g + n)] * 3
            sl[2 - ax] = slice(0, g) if side < 0 else slice(g + n, g + n + g)
            fine = U[b][:, sl[0], sl[1], sl[2]]
            # fine global origin of the slab
            fo = [int(mesh.origin[b, d]) for d in range(3)]
            fo[ax] += -g if side < 0 else n
            cpos = [fo[d] // 2 for d in range(3)]
            cb = tuple(cp // n for cp in cpos)
            if cb not in coarse:
                continue  # same-level neighbour: plain copy
            c = coarse[cb]
            avg = fine.reshape(5, fine.shape[1] // 2, 2, fine.shape[2] // 2, 2,
                               fine.shape[3] // 2, 2).mean(axis=(2, 4, 6))
            lc = [cpos[d] - int(mesh.origin[c, d]) + g for d in range(3)]
            sh = [fine.shape[3] // 2, fine.shape[2] // 2, fine.shape[1] // 2]
            want = U[c][:, lc[2]:lc[2] + sh[2], lc[1]:lc[1] + sh[1], lc[0]:lc[0] + sh[0]]
            np.testing.assert_allclose(avg, want, rtol=1e-14, atol=1e-14)
            count += 1
    assert count > 0


# ------------------------------------------------------------------ invariants

@pytest.mark.parametrize("case", ["2d_outflow", "3d_periodic", "3d_outflow", "amr", "amr3"])
def test_uniform_state_bitwise(orc, case):
    if case == "2d_outflow":
        mesh = inputs.uniform_mesh(2, (3, 2), 8, 4, inputs.OUTFLOW)
    elif case == "3d_periodic":
        mesh = inputs.uniform_mesh(3, (2, 2, 2), 8, 4, inputs.PERIODIC)
    elif case == "3d_outflow":
        mesh = inputs.uniform_mesh(3, (2, 1, 2), 8, 4, inputs.OUTFLOW)
    elif case == "amr":
        mesh = mesh_2level(4, 8, 4)
    else:
        mesh = mesh_3level()
    om = orc.OracleMesh(mesh)
    U0 = om.prim_to_cons(inputs.uniform_state(mesh))
    U, t, n = om.run(U0.copy(), nsteps=3)
    assert np.array_equal(leaf_interior(mesh, U), leaf_interior(mesh, U0))


def test_conservation_periodic_kh(orc):
    mesh = inputs.uniform_mesh(3, (2, 2, 2), 8, 4, inputs.PERIODIC)
    om = orc.OracleMesh(mesh)
    U = om.prim_to_cons(inputs.kh_state(mesh))
    T0 = om.conserved_totals(U)
    U, t, n = om.run(U, nsteps=100)
    T1 = om.conserved_totals(U)
    A = om.conserved_totals(np.abs(U))
    assert np.all(np.abs(T1 - T0) / A <= 1e-13), (T1 - T0) / A


def test_conservation_amr_needs_reflux(orc):
    """On a periodic 2-level mesh the totals are conserved to roundoff only
    with the fine-to-coarse flux correction."""
    mesh = mesh_2level(4, 8, 4, inputs.PERIODIC)
    om = orc.OracleMesh(mesh)
    U0 = om.prim_to_cons(inputs.random_smooth_state(mesh, seed=4))
    T0 = om.conserved_totals(U0)
    A = om.conserved_totals(np.abs(U0))
    U1, _, _ = om.run(U0.copy(), nsteps=20, reflux=True)
    U2, _, _ = om.run(U0.copy(), nsteps=20, reflux=False)
    d1 = np.abs(om.conserved_totals(U1) - T0) / A
    d2 = np.abs(om.conserved_totals(U2) - T0) / A
    assert np.all(d1 <= 1e-13), d1
    assert d2.max() > 1e-8, d2


def test_conservation_three_levels(orc):
    """Three levels, periodic: flux correction at both coarse-fine interfaces
    keeps the totals to roundoff."""
    mesh = mesh_3level(inputs.PERIODIC)
    om = orc.OracleMesh(mesh)
    U0 = om.prim_to_cons(inputs.random_smooth_state(mesh, seed=14))
    T0 = om.conserved_totals(U0)
    U1, _, _ = om.run(U0.copy(), nsteps=10)
    A = om.conserved_totals(np.abs(U1)) + om.conserved_totals(np.abs(U0))
    d = np.abs(om.conserved_totals(U1) - T0) / A
    assert np.all(d <= 1e-13), d


def test_reflux_matches_geometric_face_average(orc):
    """The correction of each coarse cell at a coarse-fine face equals
    +-dt/dx (F_c - mean of the fine fluxes whose face centres lie on that
    coarse face), with fine faces matched by physical position."""
    mesh = mesh_2level(4, 8, 4, inputs.PERIODIC)
    om = orc.OracleMesh(mesh)
    U = om.prim_to_cons(inputs.random_smooth_state(mesh, seed=9))
    om.guardcell_fill(U)
    dt = 0.3 * om.compute_dt(U)
    Ur, _, bf = om.hydro_advance(U, dt, reflux=True, want_bflux=True)
    Un, _, _ = om.hydro_advance(U, dt, reflux=False)
    n, g = mesh.nxb, mesh.ng
    leaf = mesh.is_leaf()
    # physical face centres of every fine boundary face
    fine_faces = {}
    for b in range(mesh.nb):
        if mesh.level[b] != 1:
            continue
        dx = 1.0 / mesh.cells_per_axis(1)[0]
        for d in range(3):
            a1, a2 = [e for e in range(3) if e != d]
            for s in range(2):
                pos_d = (mesh.origin[b, d] + (n if s else 0)) * dx % 1.0
                for t2 in range(n):
                    for t1 in range(n):
                        p = [0.0] * 3
                        p[d] = round(pos_d, 12)
                        p[a1] = round((mesh.origin[b, a1] + t1 + 0.5) * dx, 12)
                        p[a2] = round((mesh.origin[b, a2] + t2 + 0.5) * dx, 12)
                        fine_faces[(d, tuple(p))] = bf[b, 2 * d + s, :, t2 * n + t1]
    dxc = 1.0 / mesh.cells_per_axis(0)[0]
    checked = 0
    for c in range(mesh.nb):
        if mesh.level[c] != 0 or not leaf[c]:
            continue
        diff = mesh.interior(Ur[c:c + 1])[0] - mesh.interior(Un[c:c + 1])[0]
        want = np.zeros_like(diff)
        for d in range(3):
            a1, a2 = [e for e in range(3) if e != d]
            for s in range(2):
                pos_d = round((mesh.origin[c, d] + (n if s else 0)) * dxc % 1.0, 12)
                for t2 in range(n):
                    for t1 in range(n):
                        fl = []
                        for o2 in (0.25, 0.75):
                            for o1 in (0.25, 0.75):
                                p = [0.0] * 3
                                p[d] = pos_d
                                p[a1] = round((mesh.origin[c, a1] + t1 + o1) * dxc, 12)
                                p[a2] = round((mesh.origin[c, a2] + t2 + o2) * dxc, 12)
                                key = (d, tuple(p))
                                if key in fine_faces:
                                    fl.append(fine_faces[key])
                        if not fl:
                            continue
                        assert len(fl) == 4
                        fbar = np.mean(fl, axis=0)
                        fc = bf[c, 2 * d + s, :, t2 * n + t1]
                        corr = dt * (fc - fbar) / dxc * (1 if s else -1)
                        cell = [0] * 3
                        cell[d] = n - 1 if s else 0
                        cell[a1], cell[a2] = t1, t2
                        want[:, cell[2], cell[1], cell[0]] += corr
                        checked += 1
        np.testing.assert_allclose(diff, want, rtol=1e-9, atol=1e-13)
    assert checked > 0


def test_two_d_rows_identical_and_w_zero(orc):
    mesh, W, g, cfl = inputs.workload("sod2d")
    om = orc.OracleMesh(mesh, g)
    U, t, n = om.run(om.prim_to_cons(W), nsteps=50)
    G = assemble(mesh, U)
    assert np.array_equal(G, np.broadcast_to(G[:, :, :1, :], G.shape))
    assert np.all(G[2] == 0.0) and np.all(G[3] == 0.0)


def test_sod_mirror_symmetry(orc):
    mesh = inputs.uniform_mesh(2, (8, 1), 16, 4, inputs.OUTFLOW)
    om = orc.OracleMesh(mesh)
    Ua, _, _ = om.run(om.prim_to_cons(inputs.sod_state(mesh)), nsteps=40)
    Ub, _, _ = om.run(om.prim_to_cons(inputs.sod_state(mesh, mirror=True)), nsteps=40)
    Ga, Gb = assemble(mesh, Ua), assemble(mesh, Ub)
    Gm = Gb[:, :, :, ::-1].copy()
    Gm[1] = -Gm[1]
    for v in range(5):
        s = np.abs(Ga[v]).max() or 1.0
        assert np.abs(Ga[v] - Gm[v]).max() <= 1e-14 * s


def test_shear_layer_mirror_symmetry(orc):
    """The shear layer with its random perturbation replaced by one mode,
    v_y = 0.01 sin(2 pi x) sin(4 pi y) -- odd about y = 1/2, while the band
    |y - 1/2| < 1/4 and v_x are even -- is symmetric under y -> 1 - y with
    v_y -> -v_y, and the scheme keeps it so to roundoff (periodic, 2D, with
    the transverse predictor terms and both flux directions active)."""
    mesh = inputs.uniform_mesh(2, (4, 4), 16, 4, inputs.PERIODIC)
    W = inputs.kh_state(mesh)
    I = mesh.interior(W)
    for b in range(mesh.nb):
        x, y, _ = mesh.cell_centers(b)
        I[b, 2] = 0.01 * np.sin(2 * np.pi * x) * np.sin(4 * np.pi * y)
    om = orc.OracleMesh(mesh)
    U, _, _ = om.run(om.prim_to_cons(W), nsteps=30)
    G = assemble(mesh, U)
    Gm = G[:, :, ::-1, :].copy()
    Gm[2] = -Gm[2]
    assert np.abs(G[2]).max() > 1e-3   # the mode is there and has grown
    for v in range(5):
        s = np.abs(G[v]).max()
        assert np.abs(G[v] - Gm[v]).max() <= 1e-12 * s, v


def test_sod_axis_equivalence(orc):
    """Sod along y equals the transposed Sod along x."""
    mesh = inputs.uniform_mesh(2, (4, 4), 16, 4, inputs.OUTFLOW)
    om = orc.OracleMesh(mesh)
    Ux, _, _ = om.run(om.prim_to_cons(inputs.sod_state(mesh, axis=0)), nsteps=20)
    Uy, _, _ = om.run(om.prim_to_cons(inputs.sod_state(mesh, axis=1)), nsteps=20)
    Gx, Gy = assemble(mesh, Ux), assemble(mesh, Uy)
    Gt = Gy.transpose(0, 1, 3, 2)[[0, 2, 1, 3, 4]]
    np.testing.assert_allclose(Gx, Gt, rtol=0, atol=1e-15)


def test_sod_exact_solution_l1_convergence(orc):
    """L1 density error against the exact Riemann solution at t = 0.2 halves
    with each doubling of resolution (first order, shock-limited)."""
    errs = []
    for nx in (64, 128, 256):
        mesh = inputs.uniform_mesh(2, (nx // 16, 1), 16, 4, inputs.OUTFLOW)
        om = orc.OracleMesh(mesh)
        U, t, _ = om.run(om.prim_to_cons(inputs.sod_state(mesh)), t_end=0.2)
        assert t == pytest.approx(0.2, rel=1e-12)
        rho = assemble(mesh, U)[0, 0, 0]
        x = (np.arange(nx) + 0.5) / nx
        ex = orc.riemann_sample([1, 0, 1], [0.125, 0, 0.1], (x - 0.5) / t)[:, 0]
        errs.append(np.abs(rho - ex).mean())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[1] < 0.005
    assert np.all(orders > 0.85) and np.all(orders < 1.3), (errs, orders)


def test_scalar_advection_special_case(orc):
    """With uniform velocity and pressure the mass update reduces to the
    textbook MC-limited MUSCL-Hancock scheme for linear advection:
    rho_i - nu (rho*_{i+1/2} - rho*_{i-1/2}), rho*_{i+1/2} = rho_i + (1-nu)/2 s_i."""
    mesh = inputs.uniform_mesh(2, (4, 1), 16, 4, inputs.PERIODIC)
    om = orc.OracleMesh(mesh)
    W = inputs.uniform_state(mesh, rho=1.0, vel=(0.8, 0.0, 0.0), p=1.0)
    N = 64
    rng = np.random.default_rng(3)
    prof = 1.0 + 0.5 * rng.random(N)
    for b in range(mesh.nb):
        o = int(mesh.origin[b, 0])
        W[b, 0, 0, 4:20, 4:20] = prof[o:o + 16][None, :]
    U = om.prim_to_cons(W)
    om.guardcell_fill(U)
    dt = 0.5 / N  # nu = 0.8 * dt * N = 0.4
    Un, st, _ = om.hydro_advance(U, dt)
    assert st == 0
    nu = 0.8 * dt * N
    rm, rp = np.roll(prof, 1), np.roll(prof, -1)
    a, b_ = prof - rm, rp - prof
    s = np.where(a * b_ <= 0, 0.0,
                 np.sign(a) * np.minimum(np.minimum(2 * np.abs(a), 2 * np.abs(b_)),
                                         0.5 * np.abs(a + b_)))
    face = prof + 0.5 * (1 - nu) * s          # upwind state at i+1/2
    want = prof - nu * (face - np.roll(face, 1))
    got = assemble(mesh, Un)[0, 0, 0]
    np.testing.assert_allclose(got, want, rtol=1e-13)


def test_decomposition_invariance(orc):
    """One 8^3 block == 8 blocks of 4^3 == 64 blocks of 2^3 (periodic), bitwise."""
    res = []
    for nxb, nblk in ((8, 1), (4, 2), (2, 4)):
        mesh = inputs.uniform_mesh(3, (nblk,) * 3, nxb, 2, inputs.PERIODIC)
        om = orc.OracleMesh(mesh)
        U, _, _ = om.run(om.prim_to_cons(inputs.random_smooth_state(mesh, seed=2)), nsteps=3)
        res.append(assemble(mesh, U))
    assert np.array_equal(res[0], res[1])
    assert np.array_equal(res[0], res[2])


def test_all_fine_two_level_equals_uniform_fine(orc):
    base = inputs.uniform_mesh(3, (2, 2, 2), 8, 4, inputs.PERIODIC)
    mesh = inputs.refine(base, np.ones(base.nb, dtype=bool))
    fine = inputs.uniform_mesh(3, (4, 4, 4), 8, 4, inputs.PERIODIC)
    om, of = orc.OracleMesh(mesh), orc.OracleMesh(fine)
    Ua, _, _ = om.run(om.prim_to_cons(inputs.random_smooth_state(mesh, seed=5)), nsteps=3)
    Ub, _, _ = of.run(of.prim_to_cons(inputs.random_smooth_state(fine, seed=5)), nsteps=3)
    assert np.array_equal(assemble(mesh, Ua), assemble(fine, Ub))


def test_sedov_cube_symmetry(orc):
    """Sedov on a symmetric 2-level mesh stays invariant under axis swaps and
    reflections (roundoff only)."""
    mesh = mesh_2level(4, 8, 4)
    om = orc.OracleMesh(mesh)
    W = inputs.sedov_state(mesh)
    U, _, _ = om.run(om.prim_to_cons(W), nsteps=10)
    G = assemble(mesh, U)
    rho, E = G[0], G[4]
    m = G[1:4]
    for v, f in ((0, rho), (4, E)):
        s = np.abs(f).max()
        for perm in ((0, 2, 1), (1, 0, 2), (2, 1, 0)):
            assert np.abs(f - f.transpose(perm)).max() <= 1e-12 * s
        for ax in range(3):
            assert np.abs(f - np.flip(f, axis=ax)).max() <= 1e-12 * s
    # momentum: m_x(x) is odd under x -> -x and maps to m_y under x <-> y
    s = np.abs(m).max()
    assert np.abs(m[0] + np.flip(m[0], axis=2)).max() <= 1e-12 * s
    assert np.abs(m[0] - m[1].transpose(0, 2, 1)).max() <= 1e-12 * s
    assert np.abs(m[0] - m[2].transpose(2, 1, 0)).max() <= 1e-12 * s


def test_advection_pressure_velocity_stay_uniform(orc):
    mesh = inputs.uniform_mesh(3, (2, 2, 2), 8, 4, inputs.PERIODIC)
    om = orc.OracleMesh(mesh)
    U, _, _ = om.run(om.prim_to_cons(inputs.advection_state(mesh)), nsteps=10)
    W = om.cons_to_prim(U)
    Wi = leaf_interior(mesh, W)
    assert np.abs(Wi[:, 4] - 1.0).max() <= 1e-13
    assert np.abs(Wi[:, 1] - 1.0).max() <= 1e-13
    assert np.abs(Wi[:, 2] - 0.5).max() <= 1e-13
    assert np.abs(Wi[:, 3] - 0.25).max() <= 1e-13


def test_advection_second_order_convergence(orc):
    """Smooth 3D advection of a single Fourier mode converges at close to
    second order (MC clips extrema) against the exactly translated profile."""
    errs = []
    for nblk in (2, 4):
        mesh = inputs.uniform_mesh(3, (nblk,) * 3, 8, 4, inputs.PERIODIC)
        om = orc.OracleMesh(mesh)
        kw = dict(seed=1, nmodes=1, kmax=1, amp=0.1)
        U, t, _ = om.run(om.prim_to_cons(inputs.advection_state(mesh, **kw)), t_end=0.25)
        err = 0.0
        for b in range(mesh.nb):
            x, y, z = mesh.cell_centers(b)
            ex = inputs.advection_density(x, y, z, t, **kw)
            err += np.abs(mesh.interior(U[b:b + 1])[0, 0] - ex).sum()
        errs.append(err / (nblk * 8) ** 3)
    order = np.log2(errs[0] / errs[1])
    assert order > 1.5, (errs, order)


def test_dt_uniform_closed_form(orc):
    mesh = inputs.uniform_mesh(3, (2, 1, 1), 8, 4, inputs.OUTFLOW,
                               hi=(2.0, 1.0, 0.5))
    om = orc.OracleMesh(mesh)
    W = inputs.uniform_state(mesh, rho=1.3, vel=(0.3, -0.2, 0.1), p=0.7)
    U = om.prim_to_cons(W)
    c = np.sqrt(GAMMA * 0.7 / 1.3)
    dx = np.array([2.0 / 16, 1.0 / 8, 0.5 / 8])
    sp = (np.array([0.3, 0.2, 0.1]) + c) / dx
    assert om.compute_dt(U, 0.8, 0) == pytest.approx(0.8 / sp.sum(), rel=1e-14)
    assert om.compute_dt(U, 0.8, 1) == pytest.approx(0.8 / sp.max(), rel=1e-14)


@pytest.mark.parametrize("where", ["first", "middle", "last"])
def test_dt_of_a_cell_without_sound_speed_is_nan(orc, where):
    """A cell whose energy is below its kinetic energy has negative pressure
    and no sound speed; the CFL bound of a state that holds it is undefined,
    so dt is NaN in both forms wherever the cell sits (first cell a thread
    visits, or last), on one thread and on several."""
    mesh = inputs.uniform_mesh(3, (2, 2, 1), 8, 4, inputs.PERIODIC)
    om = orc.OracleMesh(mesh)
    U = om.prim_to_cons(inputs.uniform_state(mesh, rho=1.0, vel=(0.5, 0, 0), p=1.0))
    g, n = mesh.ng, mesh.nxb
    b, k, j, i = {"first": (0, 0, 0, 0), "middle": (1, 3, 5, 2),
                  "last": (mesh.nb - 1, n - 1, n - 1, n - 1)}[where]
    U[b, 4, g + k, g + j, g + i] = 0.01          # E < |m|^2 / (2 rho) = 0.125
    old = orc.get_threads()
    try:
        for nthreads in (1, 4):
            orc.set_threads(nthreads)
            for form in (0, 1):
                assert np.isnan(om.compute_dt(U, 0.8, form)), (nthreads, form)
    finally:
        orc.set_threads(old)
    U[b, 4, g + k, g + j, g + i] = 1.0 / (GAMMA - 1.0) + 0.125   # physical again
    assert np.isfinite(om.compute_dt(U, 0.8, 1))


def test_positivity_fallback_keeps_123_problem_positive(orc):
    """Two strong rarefactions (Toro's test 2) push face states towards
    vacuum; the first-order fallback keeps every cell positive."""
    mesh = inputs.uniform_mesh(2, (8, 1), 16, 4, inputs.OUTFLOW)
    W = inputs.uniform_state(mesh, rho=1.0, vel=(0, 0, 0), p=0.4)
    for b in range(mesh.nb):
        x, _, _ = mesh.cell_centers(b)
        W[b, 1, 0, 4:20, 4:20] = np.where(x < 0.5, -2.0, 2.0)
    om = orc.OracleMesh(mesh)
    U, t, n = om.run(om.prim_to_cons(W), t_end=0.15)
    Wi = leaf_interior(mesh, om.cons_to_prim(U))
    assert np.all(Wi[:, 0] > 0) and np.all(Wi[:, 4] > 0)


def test_thread_count_independent(orc):
    mesh = mesh_2level(4, 8, 4, inputs.PERIODIC)
    om = orc.OracleMesh(mesh)
    U0 = om.prim_to_cons(inputs.random_smooth_state(mesh, seed=8))
    old = orc.get_threads()
    try:
        orc.set_threads(1)
        Ua, _, _ = om.run(U0.copy(), nsteps=3)
        orc.set_threads(4)
        Ub, _, _ = om.run(U0.copy(), nsteps=3)
    finally:
        orc.set_threads(old)
    assert np.array_equal(leaf_interior(mesh, Ua), leaf_interior(mesh, Ub))


def _wave_errors(orc, kind, ns=(32, 64, 128), eps=1e-5, t_end=0.25):
    """L1 error (relative to the amplitude) of a small-amplitude smooth wave
    along x after ``t_end``, against its exact linear translation."""
    errs = []
    for nx in ns:
        mesh = inputs.uniform_mesh(2, (nx // 16, 1), 16, 4, inputs.PERIODIC)
        om = orc.OracleMesh(mesh)
        W = inputs.uniform_state(mesh, rho=1.0, vel=(0, 0, 0), p=1.0 / GAMMA)
        for b in range(mesh.nb):
            x, _, _ = mesh.cell_centers(b)
            s = np.sin(2 * np.pi * x)[0]
            if kind == "acoustic":   # rho0 = 1, c0 = 1: dp = drho = du
                W[b, 0, 0, 4:20, 4:20] = 1.0 + eps * s
                W[b, 1, 0, 4:20, 4:20] = eps * s
                W[b, 4, 0, 4:20, 4:20] = 1.0 / GAMMA + eps * s
            else:                    # shear wave carried by u = 1
                W[b, 1, 0, 4:20, 4:20] = 1.0
                W[b, 2, 0, 4:20, 4:20] = eps * s
        U, t, _ = om.run(om.prim_to_cons(W), t_end=t_end)
        G = assemble(mesh, U)
        x = (np.arange(nx) + 0.5) / nx
        ex = np.sin(2 * np.pi * (x - t))
        if kind == "acoustic":
            got = (G[0, 0, 0] - 1.0) / eps
        else:
            got = G[2, 0, 0] / eps       # rho = 1 exactly, so m_y = v
        errs.append(np.abs(got - ex).mean())
    return np.array(errs)


@pytest.mark.parametrize("kind", ["acoustic", "shear"])
def test_linear_waves_second_order(orc, kind):
    """Small-amplitude acoustic and shear waves converge at close to second
    order: every term of the Hancock predictor matters for these."""
    errs = _wave_errors(orc, kind)
    orders = np.log2(errs[:-1] / errs[1:])
    assert np.all(orders > 1.6), (errs, orders)


# ------------------------------------------------------------------ SSP-RK2 variant

def test_rk2_scalar_advection_special_case(orc):
    """With uniform velocity and pressure the SSP-RK2 mass update is the
    textbook Heun scheme on MC-limited upwind PLM:
    L(r)_i = -nu (r_i + s_i/2 - r_{i-1} - s_{i-1}/2),
    r1 = r + L(r), r_new = (r + r1 + L(r1)) / 2."""
    mesh = inputs.uniform_mesh(2, (4, 1), 16, 4, inputs.PERIODIC)
    om = orc.OracleMesh(mesh)
    W = inputs.uniform_state(mesh, rho=1.0, vel=(0.8, 0.0, 0.0), p=1.0)
    N = 64
    rng = np.random.default_rng(13)
    prof = 1.0 + 0.5 * rng.random(N)
    for b in range(mesh.nb):
        o = int(mesh.origin[b, 0])
        W[b, 0, 0, 4:20, 4:20] = prof[o:o + 16][None, :]
    U = om.prim_to_cons(W)
    om.guardcell_fill(U)
    dt = 0.5 / N
    nu = 0.8 * dt * N

    def L(r):
        a, bb = r - np.roll(r, 1), np.roll(r, -1) - r
        s = np.where(a * bb <= 0, 0.0,
                     np.sign(a) * np.minimum(np.minimum(2 * np.abs(a), 2 * np.abs(bb)),
                                             0.5 * np.abs(a + bb)))
        face = r + 0.5 * s
        return -nu * (face - np.roll(face, 1))

    r1 = prof + L(prof)
    want = 0.5 * (prof + (r1 + L(r1)))
    Un, st, _ = om.hydro_advance(U, dt, integrator=1)
    assert st == 0
    np.testing.assert_allclose(assemble(mesh, Un)[0, 0, 0], want, rtol=1e-13)


def test_rk2_sod_convergence_and_linear_waves(orc):
    errs = []
    for nx in (64, 128, 256):
        mesh = inputs.uniform_mesh(2, (nx // 16, 1), 16, 4, inputs.OUTFLOW)
        om = orc.OracleMesh(mesh)
        U, t, _ = om.run(om.prim_to_cons(inputs.sod_state(mesh)), t_end=0.2, integrator=1)
        rho = assemble(mesh, U)[0, 0, 0]
        x = (np.arange(nx) + 0.5) / nx
        ex = orc.riemann_sample([1, 0, 1], [0.125, 0, 0.1], (x - 0.5) / t)[:, 0]
        errs.append(np.abs(rho - ex).mean())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 0.75) and np.all(orders < 1.3), (errs, orders)
    # smooth acoustic wave at second order
    errs = []
    eps = 1e-5
    for nx in (32, 64, 128):
        mesh = inputs.uniform_mesh(2, (nx // 16, 1), 16, 4, inputs.PERIODIC)
        om = orc.OracleMesh(mesh)
        W = inputs.uniform_state(mesh, rho=1.0, vel=(0, 0, 0), p=1.0 / GAMMA)
        for b in range(mesh.nb):
            x, _, _ = mesh.cell_centers(b)
            s = np.sin(2 * np.pi * x)[0]
            W[b, 0, 0, 4:20, 4:20] = 1.0 + eps * s
            W[b, 1, 0, 4:20, 4:20] = eps * s
            W[b, 4, 0, 4:20, 4:20] = 1.0 / GAMMA + eps * s
        U, t, _ = om.run(om.prim_to_cons(W), t_end=0.25, integrator=1)
        xg = (np.arange(nx) + 0.5) / nx
        got = (assemble(mesh, U)[0, 0, 0] - 1.0) / eps
        errs.append(np.abs(got - np.sin(2 * np.pi * (xg - t))).mean())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.6), (errs, orders)


def test_rk2_conservation_uniform_and_amr(orc):
    for mesh, W in ((inputs.uniform_mesh(3, (2, 2, 2), 8, 4, inputs.PERIODIC), None),
                    (mesh_2level(4, 8, 4, inputs.PERIODIC), None)):
        W = inputs.random_smooth_state(mesh, seed=18)
        om = orc.OracleMesh(mesh)
        U0 = om.prim_to_cons(W)
        T0 = om.conserved_totals(U0)
        U1, _, _ = om.run(U0.copy(), nsteps=15, integrator=1)
        A = om.conserved_totals(np.abs(U0)) + om.conserved_totals(np.abs(U1))
        d = np.abs(om.conserved_totals(U1) - T0) / A
        assert np.all(d <= 1e-13), d
        if mesh.level.max() > 0:       # without the stage-averaged correction it drifts
            U2, _, _ = om.run(U0.copy(), nsteps=15, integrator=1, reflux=False)
            assert (np.abs(om.conserved_totals(U2) - T0) / A).max() > 1e-8
    mesh = mesh_2level(4, 8, 4)
    om = orc.OracleMesh(mesh)
    U0 = om.prim_to_cons(inputs.uniform_state(mesh))
    U, _, _ = om.run(U0.copy(), nsteps=3, integrator=1)
    assert np.array_equal(leaf_interior(mesh, U), leaf_interior(mesh, U0))


def test_rk3_scalar_advection_special_case(orc):
    """With uniform velocity and pressure the SSP-RK3 mass update is the
    textbook Shu-Osher scheme on MC-limited upwind PLM:
    r1 = r + L(r), r2 = 3/4 r + 1/4 (r1 + L(r1)), r_new = 1/3 r + 2/3 (r2 + L(r2))."""
    mesh = inputs.uniform_mesh(2, (4, 1), 16, 4, inputs.PERIODIC)
    om = orc.OracleMesh(mesh)
    W = inputs.uniform_state(mesh, rho=1.0, vel=(0.8, 0.0, 0.0), p=1.0)
    N = 64
    rng = np.random.default_rng(17)
    prof = 1.0 + 0.5 * rng.random(N)
    for b in range(mesh.nb):
        o = int(mesh.origin[b, 0])
        W[b, 0, 0, 4:20, 4:20] = prof[o:o + 16][None, :]
    U = om.prim_to_cons(W)
    om.guardcell_fill(U)
    dt = 0.5 / N
    nu = 0.8 * dt * N

    def L(r):
        a, bb = r - np.roll(r, 1), np.roll(r, -1) - r
        s = np.where(a * bb <= 0, 0.0,
                     np.sign(a) * np.minimum(np.minimum(2 * np.abs(a), 2 * np.abs(bb)),
                                             0.5 * np.abs(a + bb)))
        face = r + 0.5 * s
        return -nu * (face - np.roll(face, 1))

    r1 = prof + L(prof)
    r2 = 0.75 * prof + 0.25 * (r1 + L(r1))
    want = prof / 3.0 + 2.0 / 3.0 * (r2 + L(r2))
    Un, st, _ = om.hydro_advance(U, dt, integrator=2)
    assert st == 0
    np.testing.assert_allclose(assemble(mesh, Un)[0, 0, 0], want, rtol=1e-13)


def _front_errors(orc, integrator, cfls=(0.8, 0.4, 0.2), ref_cfl=0.025, t_end=0.2):
    """L1 distance of the density at t_end from a run with a much smaller dt,
    on one mesh (so only the time discretisation differs): a smooth tanh front
    advected at u = 0.8 through uniform pressure, where the MC limiter takes
    the central slope and the spatial operator is linear (Fromm)."""
    nx = 128
    mesh = inputs.uniform_mesh(2, (nx // 16, 1), 16, 4, inputs.OUTFLOW)
    om = orc.OracleMesh(mesh)
    W = inputs.uniform_state(mesh, rho=1.0, vel=(0.8, 0.0, 0.0), p=1.0)
    for b in range(mesh.nb):
        x, _, _ = mesh.cell_centers(b)
        W[b, 0, 0, 4:20, 4:20] = 1.5 + 0.4 * np.tanh((x[0] - 0.3) / 0.08)
    U0 = om.prim_to_cons(W)
    dx = 1.0 / nx
    amax = 0.8 + np.sqrt(GAMMA * 1.0 / 1.1)

    def run(cfl):
        dt = cfl * dx / amax
        n = int(round(t_end / dt))
        U = U0.copy()
        for _ in range(n):
            U, _ = om.step(U, dt=t_end / n, integrator=integrator)
        return assemble(mesh, U)[0, 0, 0]

    ref = run(ref_cfl)
    return [np.abs(run(c) - ref).mean() for c in cfls]


def test_rk3_third_order_in_time(orc):
    """Halving dt on a fixed mesh cuts the time-discretisation error ~8x for
    SSP-RK3 (~4x for SSP-RK2, which this test also checks so that it can tell
    the two apart)."""
    e3 = _front_errors(orc, 2)
    o3 = np.log2(np.array(e3[:-1]) / np.array(e3[1:]))
    assert np.all(o3 > 2.6), (e3, o3)
    e2 = _front_errors(orc, 1)
    o2 = np.log2(np.array(e2[:-1]) / np.array(e2[1:]))
    assert np.all(o2 > 1.7) and np.all(o2 < 2.4), (e2, o2)


def test_rk3_conservation_uniform_and_amr(orc):
    for mesh in (inputs.uniform_mesh(3, (2, 2, 2), 8, 4, inputs.PERIODIC),
                 mesh_2level(4, 8, 4, inputs.PERIODIC)):
        W = inputs.random_smooth_state(mesh, seed=19)
        om = orc.OracleMesh(mesh)
        U0 = om.prim_to_cons(W)
        T0 = om.conserved_totals(U0)
        U1, _, _ = om.run(U0.copy(), nsteps=12, integrator=2)
        A = om.conserved_totals(np.abs(U0)) + om.conserved_totals(np.abs(U1))
        d = np.abs(om.conserved_totals(U1) - T0) / A
        assert np.all(d <= 1e-13), d
        if mesh.level.max() > 0:       # without the stage-weighted correction it drifts
            U2, _, _ = om.run(U0.copy(), nsteps=12, integrator=2, reflux=False)
            assert (np.abs(om.conserved_totals(U2) - T0) / A).max() > 1e-8
    mesh = mesh_2level(4, 8, 4)
    om = orc.OracleMesh(mesh)
    U0 = om.prim_to_cons(inputs.uniform_state(mesh))
    U, _, _ = om.run(U0.copy(), nsteps=3, integrator=2)
    assert np.array_equal(leaf_interior(mesh, U), leaf_interior(mesh, U0))


# ------------------------------------------------------------------ reflecting walls

def _wall_problem(ndim, nblk, nxb, walls, refine_at, seed):
    """A problem with reflecting walls on both sides of the axes in ``walls``
    (periodic elsewhere), and its mirror-image extension: the periodic
    problem on the domain doubled to [-1, 1] along each wall axis, with the
    initial data mirrored there (density, pressure and the tangential
    velocities even, the normal velocity odd).  By symmetry the periodic
    solution restricted to [0, 1] is the walled one.  ``refine_at(c)`` says
    whether the level-0 block with block coordinates ``c`` of the walled
    domain is refined once.  The initial data are random per level-0 cell."""
    bc_r = tuple((R_, R_) if d in walls else (P_, P_) for d in range(3))
    m_r = inputs.uniform_mesh(ndim, nblk, nxb, 4, bc_r)
    nb_p = tuple(2 * nblk[d] if d in walls else nblk[d] for d in range(ndim))
    lo_p = tuple(-1.0 if d in walls else 0.0 for d in range(3))
    m_p = inputs.uniform_mesh(ndim, nb_p, nxb, 4, P_, lo=lo_p)

    def mirror_coord(c):
        return tuple((c[d] - nblk[d] if c[d] >= nblk[d] else nblk[d] - 1 - c[d])
                     if d in walls else c[d] for d in range(ndim))

    f_r = [refine_at(tuple(m_r.origin[b, :ndim] // nxb)) for b in range(m_r.nb)]
    f_p = [refine_at(mirror_coord(tuple(m_p.origin[b, :ndim] // nxb))) for b in range(m_p.nb)]
    if any(f_r):
        m_r, m_p = inputs.refine(m_r, np.array(f_r)), inputs.refine(m_p, np.array(f_p))
    rng = np.random.default_rng(seed)
    N = m_r.cells_per_axis(0)
    Gr = np.empty((5, N[2], N[1], N[0]))
    Gr[0] = rng.uniform(0.5, 2.0, Gr[0].shape)
    for d in range(3):
        Gr[1 + d] = rng.uniform(-1.0, 1.0, Gr[0].shape) if d < ndim else 0.0
    Gr[4] = rng.uniform(0.5, 2.0, Gr[0].shape)
    Gp = Gr
    for d in walls:
        ax = 3 - d
        half = np.flip(Gp, axis=ax).copy()
        half[1 + d] = -half[1 + d]
        Gp = np.concatenate([half, Gp], axis=ax)

    def fill(mesh, G):
        W = np.zeros(mesh.shape)
        for b in range(mesh.nb):
            gx, gy, gz = mesh.global_index(b)
            s = int(mesh.level[b])
            vals = G[:, gz >> s, gy >> s, gx >> s]
            if ndim == 3:
                W[b, :, 4:-4, 4:-4, 4:-4] = vals
            else:
                W[b, :, 0, 4:-4, 4:-4] = vals[:, 0]
        return W

    return m_r, fill(m_r, Gr), m_p, fill(m_p, Gp)


@pytest.mark.parametrize("case", ["2d_box", "3d_xz", "3d_amr_wall"])
def test_reflecting_equals_mirrored_periodic(orc, case):
    """Reflecting walls reproduce the mirror-symmetric periodic solution on
    the doubled domain (up to roundoff: the periodic run is mirror-symmetric
    only to rounding), uniform and with refined blocks against a wall."""
    if case == "2d_box":
        args = (2, (2, 2), 8, (0, 1), lambda c: False)
    elif case == "3d_xz":
        args = (3, (2, 1, 2), 8, (0, 2), lambda c: False)
    else:
        args = (3, (2, 2, 2), 8, (0,), lambda c: c[0] == 0 and c[1] == 1)
    m_r, W_r, m_p, W_p = _wall_problem(*args, seed=21)
    walls = args[3]
    o_r, o_p = orc.OracleMesh(m_r), orc.OracleMesh(m_p)
    U_r, U_p = o_r.prim_to_cons(W_r), o_p.prim_to_cons(W_p)
    dt = 0.5 * o_r.compute_dt(U_r, 0.8)
    for _ in range(6):
        U_r, _ = o_r.step(U_r, dt=dt)
        U_p, _ = o_p.step(U_p, dt=dt)
    G_r, G_p = assemble(m_r, U_r), assemble(m_p, U_p)
    for d in walls:
        ax = 3 - d
        n = G_r.shape[ax]
        G_p = np.take(G_p, np.arange(n, 2 * n), axis=ax)
    assert not np.isnan(G_r).any()
    err = rel_err(G_r, G_p, axis_var=0).max()
    assert err <= 1e-12, err
    # the walls did something: the state differs from an outflow run
    bc_o = tuple((O_, O_) if d in walls else (P_, P_) for d in range(3))
    m_o = inputs.Mesh(**{**m_r.__dict__, "bc": bc_o, "extra": {}})
    o_o = orc.OracleMesh(m_o)
    U_o = o_o.prim_to_cons(W_r)
    for _ in range(6):
        U_o, _ = o_o.step(U_o, dt=dt)
    assert rel_err(assemble(m_o, U_o), G_p, axis_var=0).max() > 1e-3


@pytest.mark.parametrize("ndim", [2, 3])
def test_closed_box_conserves_mass_and_energy(orc, ndim):
    """All walls reflecting on a 2-level mesh: no mass or energy crosses a
    wall, so both totals stay constant to roundoff (momentum does not: the
    walls push back)."""
    mesh = mesh_2level(4, 8, 4, inputs.REFLECT, ndim=ndim)
    om = orc.OracleMesh(mesh)
    U0 = om.prim_to_cons(inputs.random_smooth_state(mesh, seed=8))
    T0 = om.conserved_totals(U0)
    U1, _, _ = om.run(U0.copy(), nsteps=15)
    A = om.conserved_totals(np.abs(U1)) + om.conserved_totals(np.abs(U0))
    d = np.abs(om.conserved_totals(U1) - T0) / np.where(A == 0, 1.0, A)
    assert d[0] <= 1e-13 and d[4] <= 1e-13, d
