"""Pins of the oracle's multispecies perfect gas (Section 2.2: the perfect-gas
EOS has a multispecies variant).  Species k has ratio of specific heats
gamma_k and molar mass A_k; the state carries rho X_k; a cell's gamma follows
the ideal-gas mixture rule.  Pinned by: the mixture EOS closed form; one
species with the gas's own gamma equal to the single gas; two identical
species equal to the single gas with exact species transport; the
scalar-advection special case for a mass fraction; the exact two-gas
Riemann solver (reduces to the one-gas solver, jump conditions per side);
L1 convergence of a two-gas shock tube to that exact solution."""
import dataclasses

import numpy as np
import pytest

from paper_2208_11630_gb300 import inputs
from tests.helpers import assemble, leaf_interior

GAMMA = 1.4
P_, O_ = inputs.PERIODIC, inputs.OUTFLOW


def _with_species(W, mesh, X):
    """Append mass fractions X [ns][...] (broadcast per block interior) to a
    single-gas primitive state W."""
    ns = len(mesh.species)
    Wn = np.zeros(mesh.shape)
    Wn[:, :5] = W
    g, n = mesh.ng, mesh.nxb
    for k in range(ns):
        for b in range(mesh.nb):
            if mesh.ndim == 3:
                Wn[b, 5 + k, g:g + n, g:g + n, g:g + n] = X(k, b)
            else:
                Wn[b, 5 + k, 0, g:g + n, g:g + n] = X(k, b)
    return Wn


def test_mixture_eos_closed_form(orc):
    """Helium (5/3, 4) and nitrogen (7/5, 28) in mass fractions 0.3 / 0.7:
    c_v ~ sum X/(A (g-1)), c_p ~ sum X g/(A (g-1)), gamma = c_p / c_v."""
    sp = ((5.0 / 3.0, 4.0), (1.4, 28.0))
    mesh = inputs.uniform_mesh(2, (1, 1), 8, 4, P_, species=sp)
    om = orc.OracleMesh(mesh)
    X = (0.3, 0.7)
    cv = sum(x / (a * (g - 1)) for x, (g, a) in zip(X, sp))
    cp = sum(x * g / (a * (g - 1)) for x, (g, a) in zip(X, sp))
    gam = cp / cv
    rho, u, p = 1.7, (0.3, -0.2, 0.0), 2.5
    W = np.zeros(mesh.shape)
    W[:, 0], W[:, 1], W[:, 2], W[:, 4] = rho, u[0], u[1], p
    W[:, 5], W[:, 6] = X
    U = om.prim_to_cons(W)
    E = p / (gam - 1) + 0.5 * rho * (u[0] ** 2 + u[1] ** 2)
    np.testing.assert_allclose(U[0, 4], E, rtol=1e-14)
    np.testing.assert_allclose(U[0, 5], rho * 0.3, rtol=1e-15)
    np.testing.assert_allclose(om.cons_to_prim(U)[0, 4], p, rtol=1e-14)


def test_one_species_equals_single_gas(orc):
    mesh = inputs.uniform_mesh(3, (2, 2, 2), 8, 4, P_)
    W = inputs.random_smooth_state(mesh, 61)
    ms = dataclasses.replace(mesh, species=((GAMMA, 2.0),))
    Ws = _with_species(W, ms, lambda k, b: 1.0)
    o1, o2 = orc.OracleMesh(mesh), orc.OracleMesh(ms)
    U1, _, _ = o1.run(o1.prim_to_cons(W), nsteps=8)
    U2, _, _ = o2.run(o2.prim_to_cons(Ws), nsteps=8)
    L1, L2 = leaf_interior(mesh, U1), leaf_interior(ms, U2)
    np.testing.assert_allclose(L2[:, :5], L1, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(L2[:, 5], L2[:, 0], rtol=1e-13)


def test_two_identical_species_transport(orc):
    """Two species with the same gamma and A: the flow is the single gas's
    and each species mass is conserved exactly; X1 + X2 stays 1 and each X
    stays within [0, 1] (MC reconstruction is TVD)."""
    mesh = inputs.uniform_mesh(3, (2, 2, 2), 8, 4, P_)
    W = inputs.random_smooth_state(mesh, 62)
    ms = dataclasses.replace(mesh, species=((GAMMA, 2.0), (GAMMA, 2.0)))
    rng = np.random.default_rng(63)
    X1 = rng.uniform(0.0, 1.0, (mesh.nb, 8, 8, 8))
    Ws = _with_species(W, ms, lambda k, b: X1[b] if k == 0 else 1.0 - X1[b])
    o1, o2 = orc.OracleMesh(mesh), orc.OracleMesh(ms)
    U0 = o2.prim_to_cons(Ws)
    T0 = o2.conserved_totals(U0)
    U1, _, _ = o1.run(o1.prim_to_cons(W), nsteps=10)
    U2, _, _ = o2.run(U0, nsteps=10)
    L1, L2 = leaf_interior(mesh, U1), leaf_interior(ms, U2)
    np.testing.assert_allclose(L2[:, :5], L1, rtol=1e-12, atol=1e-13)
    T1 = o2.conserved_totals(U2)
    assert np.all(np.abs(T1[5:] - T0[5:]) <= 1e-13 * np.abs(T0[5:]))
    X = L2[:, 5:] / L2[:, :1]
    np.testing.assert_allclose(X.sum(axis=1), 1.0, atol=1e-13)
    assert X.min() >= -1e-13 and X.max() <= 1 + 1e-13


def test_mass_fraction_scalar_advection_special_case(orc):
    """Uniform density, velocity and pressure with two species of equal
    gamma: the mass fraction update is the textbook MC-limited
    MUSCL-Hancock scheme for linear advection."""
    mesh = inputs.uniform_mesh(2, (4, 1), 16, 4, P_, species=((GAMMA, 1.0), (GAMMA, 1.0)))
    om = orc.OracleMesh(mesh)
    N = 64
    rng = np.random.default_rng(64)
    prof = 0.2 + 0.6 * rng.random(N)
    W = np.zeros(mesh.shape)
    W[:, 0], W[:, 1], W[:, 4] = 1.0, 0.8, 1.0
    for b in range(mesh.nb):
        o = int(mesh.origin[b, 0])
        W[b, 5, 0, 4:20, 4:20] = prof[o:o + 16][None, :]
        W[b, 6, 0, 4:20, 4:20] = 1.0 - prof[o:o + 16][None, :]
    U = om.prim_to_cons(W)
    om.guardcell_fill(U)
    dt = 0.5 / N
    Un, st, _ = om.hydro_advance(U, dt)
    assert st == 0
    nu = 0.8 * dt * N
    a, b_ = prof - np.roll(prof, 1), np.roll(prof, -1) - prof
    s = np.where(a * b_ <= 0, 0.0,
                 np.sign(a) * np.minimum(np.minimum(2 * np.abs(a), 2 * np.abs(b_)),
                                         0.5 * np.abs(a + b_)))
    face = prof + 0.5 * (1 - nu) * s
    want = prof - nu * (face - np.roll(face, 1))
    got = assemble(mesh, Un)[5, 0, 0]
    np.testing.assert_allclose(got, want, rtol=1e-13)


@pytest.mark.parametrize("WL,WR,gL,gR", [
    ([1.0, 0.0, 1.0], [0.125, 0.0, 0.1], 1.4, 5.0 / 3.0),
    ([1.0, 0.75, 1.0], [0.125, 0.0, 0.1], 1.2, 1.6),
    ([3.0, 0.0, 10.0], [1.0, 0.0, 1.0], 5.0 / 3.0, 1.3),
])
def test_two_gas_exact_riemann(orc, WL, WR, gL, gR):
    """With gL = gR the two-gas solver is the one-gas solver; otherwise each
    side's star state satisfies that side's jump conditions (shock) or
    isentropic relations (rarefaction) with its own gamma, and u, p are
    continuous across the contact."""
    import ctypes
    L = orc.lib()
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    wl, wr = np.array(WL), np.array(WR)
    s1, s2 = np.zeros(4), np.zeros(4)
    L.or_riemann_star(dp(wl), dp(wr), ctypes.c_double(gL), dp(s1))
    L.or_riemann_star2(dp(wl), dp(wr), gL, gL, dp(s2))
    assert np.array_equal(s1, s2)
    L.or_riemann_star2(dp(wl), dp(wr), gL, gR, dp(s2))
    ps, us, rsl, rsr = s2
    for (r, u, p), rs, g, sgn in ((WL, rsl, gL, 1), (WR, rsr, gR, -1)):
        if ps > p:
            S = (rs * us - r * u) / (rs - r)
            E1 = p / (g - 1) + 0.5 * r * u * u
            E2 = ps / (g - 1) + 0.5 * rs * us * us
            assert abs(r * u * (u - S) + p - (rs * us * (us - S) + ps)) <= 1e-10 * max(ps, p)
            assert abs((E1 + p) * u - S * E1 - ((E2 + ps) * us - S * E2)) <= \
                1e-10 * max(abs((E2 + ps) * us), abs(S * E2), 1.0)
        else:
            assert ps / rs ** g == pytest.approx(p / r ** g, rel=1e-12)
            c, cs = np.sqrt(g * p / r), np.sqrt(g * ps / rs)
            assert u + sgn * 2 * c / (g - 1) == pytest.approx(us + sgn * 2 * cs / (g - 1),
                                                              rel=1e-12, abs=1e-12)
    # sampling either side of the contact gives the star pressure and velocity
    out = orc.riemann_sample2(WL, WR, [us - 1e-9, us + 1e-9], gL, gR)
    np.testing.assert_allclose(out[:, 1], us, rtol=1e-12)
    np.testing.assert_allclose(out[:, 2], ps, rtol=1e-12)


def test_two_gas_shock_tube_converges_to_exact(orc):
    """Sod's states with gamma 1.4 (left gas) and 5/3 (right gas): the
    density converges in L1 to the exact two-gas solution at first order
    (shock-limited), despite the small pressure oscillations that a
    conservative scheme produces at a contact between gases of different
    gamma."""
    sp = ((1.4, 1.0), (5.0 / 3.0, 1.0))
    errs = []
    for nx in (64, 128, 256):
        mesh = inputs.uniform_mesh(2, (nx // 16, 1), 16, 4, O_, species=sp)
        om = orc.OracleMesh(mesh)
        W = np.zeros(mesh.shape)
        for b in range(mesh.nb):
            x, _, _ = mesh.cell_centers(b)
            left = (x < 0.5)[0]
            W[b, 0, 0, 4:20, 4:20] = np.where(left, 1.0, 0.125)
            W[b, 4, 0, 4:20, 4:20] = np.where(left, 1.0, 0.1)
            W[b, 5, 0, 4:20, 4:20] = np.where(left, 1.0, 0.0)
            W[b, 6, 0, 4:20, 4:20] = np.where(left, 0.0, 1.0)
        U, t, _ = om.run(om.prim_to_cons(W), t_end=0.2)
        rho = assemble(mesh, U)[0, 0, 0]
        x = (np.arange(nx) + 0.5) / nx
        ex = orc.riemann_sample2([1, 0, 1], [0.125, 0, 0.1], (x - 0.5) / t, 1.4, 5.0 / 3.0)[:, 0]
        errs.append(np.abs(rho - ex).mean())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    print(f"\ntwo-gas shock tube L1 {errs}, orders {orders}")
    assert errs[-1] < 0.01 and np.all(orders > 0.6), (errs, orders)
