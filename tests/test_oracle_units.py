"""Pins of the oracle's point functions: MC limiter, HLLC flux, exact Riemann
solver, EOS.  These check the oracle against hand values, textbook tables,
closed forms and invariants, never against itself."""
import os

import numpy as np
import pytest

GAMMA = 1.4
HERE = os.path.dirname(os.path.abspath(__file__))


def euler_flux(W, d, g=GAMMA):
    """Physical Euler flux along axis d of a primitive state (closed form)."""
    rho, p = W[0], W[4]
    vel = np.array(W[1:4])
    E = p / (g - 1) + 0.5 * rho * vel @ vel
    F = np.zeros(5)
    un = vel[d]
    F[0] = rho * un
    F[1:4] = rho * un * vel
    F[1 + d] += p
    F[4] = un * (E + p)
    return F


# ---------------------------------------------------------------- MC limiter

@pytest.mark.parametrize("a,b,want", [
    (1, 1, 1), (1, -1, 0), (1, 3, 2), (1, 10, 2), (-1, -3, -2), (0, 5, 0),
    (2, 1, 1.5), (-2, -1, -1.5), (3, 0, 0), (1e-3, 1e-3, 1e-3), (4, 5, 4.5),
])
def test_mc_hand_values(orc, a, b, want):
    # van Leer's MC: 0 on sign change, else sign(a) min(2|a|, 2|b|, |a+b|/2)
    assert orc.mc(a, b) == want


def test_mc_linear_data_exact(orc):
    for s in (0.3, -7.25, 1e-8):
        assert orc.mc(s, s) == s


# ---------------------------------------------------------------- HLLC

def _random_states(rng, n, supersonic=False):
    out = []
    for _ in range(n):
        rho = rng.uniform(0.2, 3.0)
        p = rng.uniform(0.1, 5.0)
        vel = rng.uniform(-2, 2, 3)
        if supersonic:
            vel[0] = 3.0 + np.sqrt(GAMMA * p / rho) * rng.uniform(1.1, 2)
        out.append(np.array([rho, *vel, p]))
    return out


@pytest.mark.parametrize("d", [0, 1, 2])
def test_hllc_consistency_identical_states(orc, d):
    rng = np.random.default_rng(5)
    for W in _random_states(rng, 20):
        F = orc.hllc(W, W, d)
        np.testing.assert_allclose(F, euler_flux(W, d), rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_hllc_stationary_contact(orc, d):
    # u_n = 0 on both sides and equal pressure: a stationary contact, which
    # HLLC resolves exactly: no mass or energy flux, normal momentum flux = p.
    for (rL, rR, p) in [(1.0, 0.125, 0.7), (3.0, 0.2, 2.0)]:
        WL = np.array([rL, 0.0, 0.0, 0.0, p])
        WR = np.array([rR, 0.0, 0.0, 0.0, p])
        WL[1 + (d + 1) % 3] = 0.4   # transverse velocities may jump
        WR[1 + (d + 1) % 3] = -0.9
        F = orc.hllc(WL, WR, d)
        assert abs(F[0]) <= 1e-15 * rL
        assert abs(F[4]) <= 1e-15 * p
        assert F[1 + d] == pytest.approx(p, rel=1e-15)
        for t in range(3):
            if t != d:
                assert abs(F[1 + t]) <= 1e-15


def test_hllc_supersonic_upwind(orc):
    rng = np.random.default_rng(6)
    L = _random_states(rng, 10, supersonic=True)
    R = _random_states(rng, 10, supersonic=True)
    for WL, WR in zip(L, R):
        F = orc.hllc(WL, WR, 0)
        assert np.array_equal(F, euler_flux(WL, 0)) or np.allclose(F, euler_flux(WL, 0), rtol=1e-15)
        # mirrored: supersonic to the left picks the right state
        mL = WR.copy(); mL[1] = -mL[1]
        mR = WL.copy(); mR[1] = -mR[1]
        F2 = orc.hllc(mL, mR, 0)
        np.testing.assert_allclose(F2, euler_flux(mR, 0), rtol=1e-15, atol=1e-15)


def test_hllc_direction_permutation(orc):
    # The flux along y of a state equals the x flux of the state with the x
    # and y velocity components swapped, with the momentum components swapped.
    rng = np.random.default_rng(7)
    for WL, WR in zip(_random_states(rng, 20), _random_states(rng, 20)):
        perm = [0, 2, 1, 3, 4]
        Fy = orc.hllc(WL, WR, 1)
        Fx = orc.hllc(WL[perm], WR[perm], 0)
        scale = np.abs(Fx).max()
        np.testing.assert_allclose(Fy, Fx[perm], rtol=0, atol=1e-14 * scale)
        perm = [0, 3, 2, 1, 4]
        Fz = orc.hllc(WL, WR, 2)
        Fx = orc.hllc(WL[perm], WR[perm], 0)
        # only the order of the kinetic-energy sum differs: roundoff level
        np.testing.assert_allclose(Fz, Fx[perm], rtol=0, atol=1e-14 * scale)


def test_hllc_mirror_symmetry(orc):
    rng = np.random.default_rng(8)
    for WL, WR in zip(_random_states(rng, 30), _random_states(rng, 30)):
        F = orc.hllc(WL, WR, 0)
        mL = WR.copy(); mL[1] = -mL[1]
        mR = WL.copy(); mR[1] = -mR[1]
        G = orc.hllc(mL, mR, 0)
        want = -F
        want[1] = F[1]          # the normal momentum flux is even under mirroring
        scale = np.abs(F).max()
        np.testing.assert_allclose(G, want, rtol=0, atol=1e-14 * scale)


def test_hllc_conservation_form_across_contact_wave(orc):
    # A moving contact (uniform u, p; density jump) is transported exactly:
    # mass flux rho_upwind * u, energy flux u (E_upwind + p).
    for u in (0.7, -0.4):
        WL = np.array([1.0, u, 0.0, 0.0, 1.0])
        WR = np.array([0.3, u, 0.0, 0.0, 1.0])
        up = WL if u > 0 else WR
        F = orc.hllc(WL, WR, 0)
        np.testing.assert_allclose(F, euler_flux(up, 0), rtol=1e-14, atol=1e-14)


# ---------------------------------------------------------------- exact Riemann

def _golden(name):
    vals = {}
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()
            vals[k] = float(v)
    return vals


def test_riemann_sod_star_textbook(orc):
    g = _golden("sod_star_toro.txt")
    s = orc.riemann_star([1.0, 0.0, 1.0], [0.125, 0.0, 0.1])
    for got, key in zip(s, ["p_star", "u_star", "rho_star_left", "rho_star_right"]):
        assert abs(got - g[key]) <= 0.5e-5, (key, got, g[key])


@pytest.mark.parametrize("WL,WR", [
    ([1.0, 0.0, 1.0], [0.125, 0.0, 0.1]),          # Sod: left rarefaction, right shock
    ([1.0, -2.0, 0.4], [1.0, 2.0, 0.4]),           # two rarefactions
    ([1.0, 0.0, 1000.0], [1.0, 0.0, 0.01]),        # strong shock
    ([5.99924, 19.5975, 460.894], [5.99242, -6.19633, 46.0950]),  # two shocks
])
def test_riemann_jump_conditions(orc, WL, WR):
    """Star states satisfy Rankine-Hugoniot across shocks and the isentropic
    relations plus the Riemann invariant across rarefactions."""
    g = GAMMA
    ps, us, rsl, rsr = orc.riemann_star(WL, WR)
    for side, (r, u, p), rs in (("L", WL, rsl), ("R", WR, rsr)):
        c = np.sqrt(g * p / r)
        cs = np.sqrt(g * ps / rs)
        if ps > p:   # shock: mass, momentum, energy fluxes equal in the shock frame
            m1 = r * u
            m2 = rs * us
            S = (m2 - m1) / (rs - r)
            E1 = p / (g - 1) + 0.5 * r * u * u
            E2 = ps / (g - 1) + 0.5 * rs * us * us
            assert abs((r * (u - S)) - (rs * (us - S))) <= 1e-10 * abs(r * (u - S)) + 1e-12
            lhs = r * u * (u - S) + p
            rhs = rs * us * (us - S) + ps
            assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), ps)
            lhs = (E1 + p) * u - S * E1
            rhs = (E2 + ps) * us - S * E2
            assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), abs(rhs), 1.0)
        else:        # rarefaction: isentropic, Riemann invariant conserved
            assert ps / rs ** g == pytest.approx(p / r ** g, rel=1e-12)
            sgn = 1 if side == "L" else -1
            assert u + sgn * 2 * c / (g - 1) == pytest.approx(us + sgn * 2 * cs / (g - 1),
                                                              rel=1e-12, abs=1e-12)


def test_riemann_sample_fan_is_isentropic(orc):
    WL, WR = [1.0, 0.0, 1.0], [0.125, 0.0, 0.1]
    xi = np.linspace(-1.18, -0.08, 23)   # inside the left fan of Sod
    s = orc.riemann_sample(WL, WR, xi)
    ent = s[:, 2] / s[:, 0] ** GAMMA
    np.testing.assert_allclose(ent, 1.0, rtol=1e-12)
    c = np.sqrt(GAMMA * s[:, 2] / s[:, 0])
    np.testing.assert_allclose(s[:, 1] + 2 * c / (GAMMA - 1), 2 * np.sqrt(GAMMA) / (GAMMA - 1),
                               rtol=1e-12)
    # self-similar fan: u - c = xi inside the fan
    np.testing.assert_allclose(s[:, 1] - c, xi, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- EOS

def test_eos_round_trip(orc):
    from paper_2208_11630_gb300 import inputs
    mesh = inputs.uniform_mesh(3, (2, 1, 1), 8, 2, inputs.PERIODIC)
    W = inputs.random_blocky_state(mesh, seed=3)
    om = orc.OracleMesh(mesh)
    U = om.prim_to_cons(W)
    W2 = om.cons_to_prim(U)
    Wi, W2i = mesh.interior(W), mesh.interior(W2)
    np.testing.assert_allclose(W2i, Wi, rtol=1e-13, atol=1e-13)
    # closed form of the total energy of an ideal gas
    Ui = mesh.interior(U)
    E = Wi[:, 4] / 0.4 + 0.5 * Wi[:, 0] * (Wi[:, 1] ** 2 + Wi[:, 2] ** 2 + Wi[:, 3] ** 2)
    np.testing.assert_allclose(Ui[:, 4], E, rtol=1e-14)
