"""Pins of the oracle's regridding (dynamic refinement): the Loehner error
indicator, the marking with 2:1 balance, and the data transfer.

The indicator is pinned by what its definition fixes independently of any
implementation: zero on linear fields, a value in [0, 1], invariance under
affine maps of the field (filter off), under axis permutations and mirror
images, and hand-derived closed forms on a step and on a single-cell spike.
The marking is checked by brute force (the new octree is valid and 2:1
balanced over faces, edges and corners, requested refinements are present,
coarsening only where every sibling asked for it) and on hand-worked cases.
The transfer conserves the totals, keeps uniform states bitwise and
reproduces linear fields.
"""
import dataclasses
import itertools

import numpy as np
import pytest

from paper_2208_11630_gb300 import inputs
from tests.helpers import leaf_interior
from tests.test_oracle_scheme import mesh_2level

R_, O_, P_ = inputs.REFLECT, inputs.OUTFLOW, inputs.PERIODIC


def _state_from_fields(mesh, rho_fn, p_fn):
    """Primitive state at rest with rho = rho_fn(X, Y, Z), p = p_fn(X, Y, Z)
    evaluated on finest-lattice-independent cell indices of each block's own
    level (X, Y, Z integer arrays)."""
    W = np.zeros(mesh.shape)
    g, n = mesh.ng, mesh.nxb
    for b in range(mesh.nb):
        X, Y, Z = mesh.global_index(b)
        X, Y, Z = np.broadcast_arrays(X, Y, Z)
        r, p = rho_fn(X, Y, Z), p_fn(X, Y, Z)
        if mesh.ndim == 3:
            W[b, 0, g:g + n, g:g + n, g:g + n] = r
            W[b, 4, g:g + n, g:g + n, g:g + n] = p
        else:
            W[b, 0, 0, g:g + n, g:g + n] = r[0]
            W[b, 4, 0, g:g + n, g:g + n] = p[0]
    return W


def _errors(orc, mesh, W, eps=0.01):
    om = orc.OracleMesh(mesh)
    U = om.prim_to_cons(W)
    om.guardcell_fill(U)
    return om.regrid_errors(U, eps)


def _interior_blocks(mesh):
    """Level-0 blocks that do not touch the domain boundary."""
    N = [mesh.nroot[d] for d in range(mesh.ndim)]
    out = []
    for b in range(mesh.nb):
        c = mesh.origin[b, :mesh.ndim] // mesh.nxb
        if all(0 < c[d] < N[d] - 1 for d in range(mesh.ndim)):
            out.append(b)
    return out


# ------------------------------------------------------------------ indicator

@pytest.mark.parametrize("ndim", [2, 3])
def test_indicator_zero_on_linear_fields(orc, ndim):
    mesh = inputs.uniform_mesh(ndim, (4,) * ndim, 8, 4, O_)
    W = _state_from_fields(mesh, lambda X, Y, Z: 2.0 + 0.125 * X + 0.25 * Y - 0.0625 * Z,
                           lambda X, Y, Z: 3.0 - 0.03125 * X + 0.0625 * Y + 0.125 * Z)
    err = _errors(orc, mesh, W)
    inner = _interior_blocks(mesh)
    assert inner and np.all(err[inner] == 0.0)
    assert np.all(err[[b for b in range(mesh.nb) if b not in inner]] >= 0.0)


@pytest.mark.parametrize("ndim", [2, 3])
def test_indicator_bounds_and_symmetries(orc, ndim):
    mesh = inputs.uniform_mesh(ndim, (3,) * ndim, 8, 4, P_)
    W = inputs.random_blocky_state(mesh, seed=31)
    err = _errors(orc, mesh, W)
    assert np.all((err >= 0.0) & (err <= 1.0))
    # affine invariance with the filter off: rho -> 3 rho + 2, p -> 0.5 p + 7
    W2 = W.copy()
    W2[:, 0] = np.where(W[:, 0] != 0, 3.0 * W[:, 0] + 2.0, 0.0)
    W2[:, 4] = np.where(W[:, 4] != 0, 0.5 * W[:, 4] + 7.0, 0.0)
    np.testing.assert_allclose(_errors(orc, mesh, W2, eps=0.0), _errors(orc, mesh, W, eps=0.0),
                               rtol=1e-12)
    # mirror image along x: block (i, j, k) <-> (N-1-i, j, k), cells reversed
    Wm = np.zeros_like(W)
    N = mesh.nroot[0]
    for b in range(mesh.nb):
        o = mesh.origin[b] // mesh.nxb
        t = [bb for bb in range(mesh.nb)
             if (mesh.origin[bb] // mesh.nxb)[0] == N - 1 - o[0]
             and all((mesh.origin[bb] // mesh.nxb)[1:] == o[1:])][0]
        Wm[t] = W[b][..., ::-1]
    err_m = _errors(orc, mesh, Wm)
    for b in range(mesh.nb):
        o = mesh.origin[b] // mesh.nxb
        t = [bb for bb in range(mesh.nb)
             if (mesh.origin[bb] // mesh.nxb)[0] == N - 1 - o[0]
             and all((mesh.origin[bb] // mesh.nxb)[1:] == o[1:])][0]
        assert err_m[t] == pytest.approx(err[b], rel=1e-12)
    if ndim == 3:     # axis permutation x <-> y (block order follows)
        Wt = np.zeros_like(W)
        for b in range(mesh.nb):
            o = mesh.origin[b] // mesh.nxb
            t = [bb for bb in range(mesh.nb) if (mesh.origin[bb] // mesh.nxb)[0] == o[1]
                 and (mesh.origin[bb] // mesh.nxb)[1] == o[0]
                 and (mesh.origin[bb] // mesh.nxb)[2] == o[2]][0]
            Wt[t] = W[b].swapaxes(-1, -2)
        err_t = _errors(orc, mesh, Wt)
        for b in range(mesh.nb):
            o = mesh.origin[b] // mesh.nxb
            t = [bb for bb in range(mesh.nb) if (mesh.origin[bb] // mesh.nxb)[0] == o[1]
                 and (mesh.origin[bb] // mesh.nxb)[1] == o[0]
                 and (mesh.origin[bb] // mesh.nxb)[2] == o[2]][0]
            assert err_t[t] == pytest.approx(err[b], rel=1e-12)


@pytest.mark.parametrize("ndim", [2, 3])
def test_indicator_closed_forms(orc, ndim):
    """Filter off, a step u = A (x < x0), B (x >= x0) constant across: at a
    cell next to the jump the x second difference equals the x first-
    difference sum |B - A|; a cross pair (x, t) has a zero numerator and the
    denominator |B - A| / 2 (x differences at t -+ 1), a pair (t, x) zero
    numerator and denominator (t differences vanish), and the transverse
    terms vanish, so E = 1 / sqrt(1 + (d-1) / 4).  With the filter on, a single-cell spike
    u0 = 1 + h in u = 1: N_kk = -2h, D_kk = 2h + eps (4 + 2h), cross pairs
    N = 0, D = eps, so E^2 = d (2h)^2 / (d D_kk^2 + d (d-1) eps^2)."""
    mesh = inputs.uniform_mesh(ndim, (4,) * ndim, 8, 4, O_)
    x0 = 13
    W = _state_from_fields(mesh, lambda X, Y, Z: np.where(X < x0, 1.5, 4.0),
                           lambda X, Y, Z: np.ones(np.shape(X)))
    err = _errors(orc, mesh, W, eps=0.0)
    want = 1.0 / np.sqrt(1.0 + (ndim - 1) / 4.0)
    assert err.max() == pytest.approx(want, rel=1e-14)
    h, eps = 0.75, 0.01
    c = (12, 9, 10)
    W = _state_from_fields(mesh, lambda X, Y, Z: 1.0 + h * ((X == c[0]) & (Y == c[1]) &
                                                            ((Z == c[2]) | (ndim == 2))),
                           lambda X, Y, Z: np.ones(np.shape(X)))
    err = _errors(orc, mesh, W, eps=eps)
    Dkk = 2 * h + eps * (4 + 2 * h)
    want = np.sqrt(ndim * (2 * h) ** 2 / (ndim * Dkk ** 2 + ndim * (ndim - 1) * eps ** 2))
    assert err.max() == pytest.approx(want, rel=1e-14)


# ------------------------------------------------------------------ marking

def _leaf_level_lattice(mesh, Lf):
    """Level of the leaf covering each block of the level-Lf lattice."""
    nd = mesh.ndim
    gn = [mesh.nroot[d] << Lf if d < nd else 1 for d in range(3)]
    G = -np.ones(gn[::-1], dtype=int)
    leaf = mesh.is_leaf()
    for b in range(mesh.nb):
        if not leaf[b]:
            continue
        s = Lf - int(mesh.level[b])
        lo = [int(mesh.origin[b, d] // mesh.nxb) << s if d < nd else 0 for d in range(3)]
        w = [1 << s if d < nd else 1 for d in range(3)]
        G[lo[2]:lo[2] + w[2], lo[1]:lo[1] + w[1], lo[0]:lo[0] + w[0]] = int(mesh.level[b])
    assert np.all(G >= 0), "leaves do not tile the domain"
    return G


def assert_balanced(mesh):
    """Touching leaves (faces, edges, corners; periodic axes wrap) differ by
    at most one level."""
    Lf = int(mesh.level.max())
    G = _leaf_level_lattice(mesh, Lf)
    nd = mesh.ndim
    for off in itertools.product(*([(-1, 0, 1)] * nd)):
        if not any(off):
            continue
        H = G
        valid = np.ones(G.shape, dtype=bool)
        for d, o in enumerate(off):
            ax = 2 - d
            if o == 0:
                continue
            H = np.roll(H, -o, axis=ax)
            if mesh.bc[d][0] != P_:        # no wrap: drop the rolled-in edge
                idx = [slice(None)] * 3
                idx[ax] = -1 if o > 0 else 0
                valid[tuple(idx)] = False
        assert np.all(np.abs(H - G)[valid] <= 1), off


def _children_of(mesh, b):
    return [c for c in range(mesh.nb) if mesh.parent[c] == b]


def test_no_requests_no_change(orc):
    mesh = mesh_2level(4, 8, 4, P_)
    om = orc.OracleMesh(mesh)
    U = om.prim_to_cons(inputs.random_smooth_state(mesh, 3))
    om2, U2, err, (kind, src, octs) = om.regrid(U, refine_cutoff=np.inf, derefine_cutoff=-np.inf)
    assert om2.mesh.nb == mesh.nb and np.all(kind == 0)
    # blocks re-sorted by (level, z, y, x); the state follows its block
    for nb_, b in enumerate(src):
        assert om2.mesh.level[nb_] == mesh.level[b]
        assert np.array_equal(om2.mesh.origin[nb_], mesh.origin[b])
        assert np.array_equal(mesh.interior(U2)[nb_], mesh.interior(U)[b]) or not mesh.is_leaf()[b]


def test_hand_worked_refinement_and_forced_neighbours(orc):
    """2D, 4x4 level-0 blocks, outflow.  A bump inside block (1, 1) refines
    that block only.  A bump in its child at the lower-left corner then asks
    for level 2 there, which forces the three level-0 blocks touching that
    child's corner region -- (0, 0), (1, 0), (0, 1) -- to level 1."""
    mesh = inputs.uniform_mesh(2, (4, 4), 8, 4, O_)
    om = orc.OracleMesh(mesh)
    W = _state_from_fields(mesh, lambda X, Y, Z: 1.0 + 0.5 * ((X == 10) & (Y == 11)),
                           lambda X, Y, Z: np.ones(np.shape(X)))
    om2, U2, err, _ = om.regrid(om.prim_to_cons(W), max_level=2)
    m2 = om2.mesh
    refined = [tuple(mesh.origin[b, :2] // 8) for b in range(mesh.nb) if err[b] > 0.8]
    assert refined == [(1, 1)]
    assert m2.nb == 16 + 4 and np.bincount(m2.level).tolist() == [16, 4]
    assert_balanced(m2)
    # second pass: a bump in the child whose level-1 origin is (16, 16)
    W2 = _state_from_fields(m2, lambda X, Y, Z: 1.0 + 0.5 * ((X == 17) & (Y == 18)) *
                            (1.0 if True else 0.0), lambda X, Y, Z: np.ones(np.shape(X)))
    # the bump must only appear on level-1 blocks
    for b in range(m2.nb):
        if m2.level[b] == 0:
            W2[b, 0] = np.where(W2[b, 0] != 0, 1.0, 0.0)
    om3, U3, err3, _ = om2.regrid(om2.prim_to_cons(W2), max_level=2)
    m3 = om3.mesh
    assert_balanced(m3)
    lvl0_refined = sorted(tuple(m3.origin[b, :2] // 8) for b in range(m3.nb)
                          if m3.level[b] == 0 and not m3.is_leaf()[b])
    assert lvl0_refined == [(0, 0), (0, 1), (1, 0), (1, 1)]
    assert np.bincount(m3.level).tolist() == [16, 16, 4]


@pytest.mark.parametrize("bc", [O_, P_])
def test_random_regrids_are_valid_and_honour_requests(orc, bc):
    rng = np.random.default_rng(5)
    mesh = mesh_2level(4, 8, 4, bc)
    om = orc.OracleMesh(mesh)
    U = om.prim_to_cons(inputs.random_smooth_state(mesh, 9))
    for it in range(3):
        m = om.mesh
        rc, dc = rng.uniform(0.3, 0.6), rng.uniform(0.05, 0.3)
        om2, U2, err, (kind, src, octs) = om.regrid(U, refine_cutoff=rc, derefine_cutoff=dc,
                                                    max_level=2)
        m2 = om2.mesh
        assert_balanced(m2)
        leaf = m.is_leaf()
        index2 = {(int(m2.level[b]), *map(int, m2.origin[b])): b for b in range(m2.nb)}
        leaf2 = m2.is_leaf()
        for b in range(m.nb):
            key = (int(m.level[b]), *map(int, m.origin[b]))
            if leaf[b] and err[b] > rc and m.level[b] < 2:
                # requested: b is now a parent
                assert key in index2 and not leaf2[index2[key]]
            if m.parent[b] >= 0 and key not in index2:
                # removed: every sibling was a leaf asking for coarsening
                sib = _children_of(m, m.parent[b])
                assert all(leaf[s] and err[s] < dc for s in sib)
        # conservation of the transfer
        T0, T1 = om.conserved_totals(U), om2.conserved_totals(U2)
        A = om.conserved_totals(np.abs(U))
        assert np.all(np.abs(T1 - T0) <= 1e-13 * np.maximum(A, 1e-300)), (T1 - T0) / A
        om, U = om2, U2
        U, _, _ = om.run(U, nsteps=1)


def test_hand_worked_forced_refinement_across_periodic_wrap(orc):
    """2D, 4x4 periodic.  Refine block (0, 0), then its child at the domain
    corner to level 2: the level-0 blocks touching that child across the
    periodic wrap -- (3, 0), (0, 3), (3, 3) -- are forced to level 1."""
    mesh = inputs.uniform_mesh(2, (4, 4), 8, 4, P_)
    om = orc.OracleMesh(mesh)
    W = _state_from_fields(mesh, lambda X, Y, Z: 1.0 + 0.5 * ((X == 3) & (Y == 4)),
                           lambda X, Y, Z: np.ones(np.shape(X)))
    om2, U2, err, _ = om.regrid(om.prim_to_cons(W), max_level=2)
    m2 = om2.mesh
    assert np.bincount(m2.level).tolist() == [16, 4]
    W2 = _state_from_fields(m2, lambda X, Y, Z: 1.0 + 0.5 * ((X == 1) & (Y == 2)),
                            lambda X, Y, Z: np.ones(np.shape(X)))
    for b in range(m2.nb):
        if m2.level[b] == 0:
            W2[b, 0] = np.where(W2[b, 0] != 0, 1.0, 0.0)
    om3, U3, _, _ = om2.regrid(om2.prim_to_cons(W2), max_level=2)
    m3 = om3.mesh
    assert_balanced(m3)
    lvl0_refined = sorted(tuple(m3.origin[b, :2] // 8) for b in range(m3.nb)
                          if m3.level[b] == 0 and not m3.is_leaf()[b])
    assert lvl0_refined == [(0, 0), (0, 3), (3, 0), (3, 3)]


def test_coarsening_happens_and_is_blocked_by_finer_neighbours(orc):
    """A 3-level mesh with a uniform state: every parent whose children are
    leaves asks to coarsen, but the level-1 parents next to level-2 leaves...
    all level-2 leaves are removed (their parents' siblings permit it), and
    the result is balanced."""
    from tests.test_oracle_scheme import mesh_3level
    mesh = mesh_3level(P_)
    om = orc.OracleMesh(mesh)
    U = om.prim_to_cons(inputs.uniform_state(mesh))
    om2, U2, err, _ = om.regrid(U, refine_cutoff=0.8, derefine_cutoff=0.2)
    m2 = om2.mesh
    assert_balanced(m2)
    assert int(m2.level.max()) == 1          # the level-2 leaves coarsened
    assert np.array_equal(leaf_interior(m2, U2)[:, :, 0, 0, 0],
                          np.broadcast_to(leaf_interior(mesh, U)[0, :, 0, 0, 0],
                                          leaf_interior(m2, U2)[:, :, 0, 0, 0].shape))
    om3, U3, _, _ = om2.regrid(U2)
    assert int(om3.mesh.level.max()) == 0


# ------------------------------------------------------------------ transfer

def test_transfer_linear_field_exact_and_uniform_bitwise(orc):
    mesh = inputs.uniform_mesh(3, (4, 4, 4), 8, 4, P_)
    om = orc.OracleMesh(mesh)
    # a linear density in x on an interior band (the MC slope of a linear
    # field is its exact slope; prolongation reproduces it)
    W = _state_from_fields(mesh, lambda X, Y, Z: 2.0 + 0.125 * X,
                           lambda X, Y, Z: np.ones(np.shape(X)))
    W[:, 4] = np.where(W[:, 0] != 0, 1.0, 0.0)
    U = om.prim_to_cons(W)
    # request refinement of the block at (1, 1, 1) only (errors are zero)
    om.guardcell_fill(U)
    om2, U2, err, (kind, src, octs) = om.regrid(U, refine_cutoff=-1.0, derefine_cutoff=-1.0,
                                                max_level=1)
    m2 = om2.mesh
    for b in range(m2.nb):
        if kind[b] != 1:
            continue
        o = m2.origin[b] // 8
        if not (2 <= o[0] < 6):
            continue          # children near the periodic wrap see the jump
        X, Y, Z = m2.global_index(b)
        # the coarse line 2 + I/8 at the fine centres, coarse coordinate X/2 - 1/4
        want = np.broadcast_to(2.0 + 0.0625 * X - 0.03125, (8, 8, 8))
        got = m2.interior(U2)[b, 0]
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-14)
    # uniform state: bitwise uniform after refinement everywhere
    Wu = inputs.uniform_state(mesh)
    om3, U3, _, _ = om.regrid(om.prim_to_cons(Wu), refine_cutoff=-1.0, derefine_cutoff=-1.0,
                              max_level=1)
    Li = leaf_interior(om3.mesh, U3)
    ref = leaf_interior(mesh, om.prim_to_cons(Wu))[0, :, 0, 0, 0]
    assert np.all(Li == ref[None, :, None, None, None])


def test_transfer_injects_where_linear_prolongation_is_not_positive(orc):
    """Density 1, momentum m = 2x (coarse cells ..., -2, 0, 2, ...), energy
    kinetic + 100, except kinetic + 1e-3 in the column where m = 0: there the
    MC slope of E vanishes (E has a minimum) while the momentum slope does
    not, so the linear children would carry m = +-1/2 with the coarse energy
    and a negative pressure.  They take the coarse value instead; elsewhere
    the prolongation stays linear; totals are conserved exactly."""
    mesh = inputs.uniform_mesh(2, (2, 2), 8, 4, O_)
    om = orc.OracleMesh(mesh)
    U = np.zeros(mesh.shape)
    tiny = 1e-3
    for b in range(mesh.nb):
        X, Y, _ = mesh.global_index(b)
        X, Y = np.broadcast_arrays(X, Y)
        m = 2.0 * (X[0] - 7)
        U[b, 0, 0, 4:12, 4:12] = 1.0
        U[b, 1, 0, 4:12, 4:12] = m
        U[b, 4, 0, 4:12, 4:12] = 0.5 * m * m + np.where(X[0] == 7, tiny, 100.0)
    om2, U2, err, (kind, src, octs) = om.regrid(U, refine_cutoff=-1.0, derefine_cutoff=-1.0,
                                                max_level=1)
    m2 = om2.mesh
    W2 = om2.cons_to_prim(U2)
    leaf = m2.is_leaf().astype(bool)
    assert np.all(m2.interior(W2)[leaf][:, 4] > 0.0)
    # the children of coarse column x = 7 (m = 0) carry exactly the coarse state
    for b in range(m2.nb):
        if not leaf[b]:
            continue
        X, Y, _ = m2.global_index(b)
        X = np.broadcast_to(X, (1, 8, 8))[0]
        cols = (X // 2 == 7)
        if cols.any():
            assert np.all(m2.interior(U2)[b, 1, 0][cols] == 0.0)
            assert np.all(m2.interior(U2)[b, 4, 0][cols] == tiny)
        far = (X // 2 == 3)
        if far.any():              # a linear profile: children split the slope
            got = m2.interior(U2)[b, 1, 0][far]
            assert set(np.unique(got)) == {-8.5, -7.5}
    T0, T1 = om.conserved_totals(U), om2.conserved_totals(U2)
    assert np.all(T1 == T0)
