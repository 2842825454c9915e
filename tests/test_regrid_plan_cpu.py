"""The library's regrid planner (fx_regrid_plan_host, host code) against the
oracle's (or_regrid_plan), two independent implementations of the same
marking and 2:1 balance rules (Section 2: the Grid unit refines and
derefines the octree).  Every split the balance loop adds or merge it
cancels is forced, so the result does not depend on the order in which
leaves are visited: the two must agree exactly -- levels, origins, parents
and the transfer map -- on random multi-level meshes.  No GPU is used."""
import dataclasses
import zlib

import numpy as np
import pytest

from paper_2208_11630_gb300 import fx, inputs

O_, P_, R_ = inputs.OUTFLOW, inputs.PERIODIC, inputs.REFLECT


def _mesh(ndim, nblk, bc):
    m = inputs.uniform_mesh(ndim, nblk, 8, 4, O_)
    return dataclasses.replace(m, bc=bc)


def _regridded(mesh, level, origin, parent):
    return dataclasses.replace(mesh, level=np.asarray(level, dtype=np.int32),
                               origin=np.asarray(origin, dtype=np.int64),
                               parent=np.asarray(parent, dtype=np.int32), extra={})


def _indicator(rng, mesh, mode, centre):
    """Per-block indicator: independent draws, or a bump around ``centre``
    plus noise (clustered refinement, whose balance cascades reach further)."""
    if mode == "random":
        return rng.uniform(0.0, 1.0, mesh.nb)
    err = np.empty(mesh.nb)
    for b in range(mesh.nb):
        ncell = np.array([mesh.nroot[d] * mesh.nxb * 2 ** int(mesh.level[b]) for d in range(3)])
        mid = (mesh.origin[b] + mesh.nxb / 2) / ncell
        r = np.linalg.norm((mid - centre)[:mesh.ndim])
        err[b] = np.exp(-(r / 0.3) ** 2) + 0.05 * rng.uniform()
    return err


CASES = {
    "2d_outflow": (2, (4, 4), ((O_, O_), (O_, O_), (O_, O_))),
    "2d_periodic": (2, (4, 3), ((P_, P_), (P_, P_), (O_, O_))),
    "2d_mixed": (2, (3, 4), ((P_, P_), (R_, O_), (O_, O_))),
    "3d_outflow": (3, (3, 2, 2), ((O_, O_), (O_, O_), (O_, O_))),
    "3d_periodic": (3, (2, 2, 2), ((P_, P_), (P_, P_), (P_, P_))),
    "3d_mixed": (3, (2, 3, 2), ((R_, R_), (P_, P_), (O_, R_))),
}


@pytest.mark.parametrize("mode", ["random", "clustered"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_host_planner_equals_oracle_planner(orc, case, mode):
    ndim, nblk, bc = CASES[case]
    rng = np.random.default_rng(zlib.crc32(f"{case}/{mode}".encode()))
    mesh = _mesh(ndim, nblk, bc)
    max_level = 3 if ndim == 2 else 2
    refined = coarsened = deepest = 0
    centre = rng.uniform(0.0, 1.0, 3)
    for it in range(8):
        if it % 3 == 2:   # the bump moves: its old region coarsens, a new one refines
            centre = rng.uniform(0.0, 1.0, 3)
        err = _indicator(rng, mesh, mode, centre)
        # pairs of refining stages (a regrid adds at most one level) alternate
        # with mixed ones, whose high derefine cutoff merges many sibling
        # groups (and balance cancels some)
        if it % 3 != 2:
            rc, dc = rng.uniform(0.3, 0.7), rng.uniform(0.0, 0.1)
        else:
            rc, dc = rng.uniform(0.6, 0.95), rng.uniform(0.5, 0.9)
        om = orc.OracleMesh(mesh)
        lo, oo, po, ko, so, octo = om.regrid_plan(err, rc, dc, max_level)
        lf, of, pf, mf = fx.regrid_plan_host(mesh, err, rc, dc, max_level)
        assert np.array_equal(lf, lo) and np.array_equal(of, oo) and np.array_equal(pf, po), it
        assert np.array_equal(mf[:, 0], ko) and np.array_equal(mf[:, 1], so), it
        # the octant is meaningful for new children only
        new = ko == 1
        assert np.array_equal(mf[new, 2], octo[new]), it
        refined += int(np.any(ko == 1))
        coarsened += int(np.count_nonzero(ko == 0) < mesh.nb)
        mesh = _regridded(mesh, lf, of, pf)
        deepest = max(deepest, int(mesh.level.max()))
    # the sequence really refines (beyond one level) and coarsens
    assert refined >= 2 and coarsened >= 1 and deepest >= 2, (refined, coarsened, deepest)


def test_host_planner_count_query_and_errors():
    mesh = _mesh(2, (4, 4), ((O_, O_), (O_, O_), (O_, O_)))
    L = fx.load()
    import ctypes
    ip = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    i64p = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    level = np.ascontiguousarray(mesh.level, dtype=np.int32)
    origin = np.ascontiguousarray(mesh.origin, dtype=np.int64)
    parent = np.ascontiguousarray(mesh.parent, dtype=np.int32)
    nroot = np.array(mesh.nroot, dtype=np.int32)
    bc = mesh.bc_flat()
    err = np.zeros(mesh.nb)
    err[5] = 1.0                                  # one block splits: 16 + 4 blocks
    dp = err.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    n = ctypes.c_int(-1)
    msg = ctypes.create_string_buffer(128)

    def call(lv=level, og=origin, pa=parent, nxb=8, cap=0, out=None):
        o = out or (None, None, None, None)
        return L.fx_regrid_plan_host(2, nxb, ip(nroot), ip(bc), mesh.nb, ip(lv), i64p(og), ip(pa),
                                     dp, 0.8, 0.2, 2, cap, ctypes.byref(n), *o, msg, 128)

    # cap 0 asks for the count
    assert call() == -1 and n.value == 20
    lv, og, pa, mp = (np.zeros(20, np.int32), np.zeros((20, 3), np.int64), np.zeros(20, np.int32),
                      np.zeros((20, 3), np.int32))
    assert call(cap=20, out=(ip(lv), i64p(og), ip(pa), ip(mp))) == 0 and n.value == 20
    assert sorted(np.bincount(lv).tolist()) == [4, 16] and (mp[:, 0] == 1).sum() == 4
    # meshes fx_blocks_create refuses are refused here too
    bad_origin = origin.copy()
    bad_origin[3, 0] += 4                         # off the block lattice
    assert call(og=bad_origin) == -7 and b"lattice" in msg.value
    dup = origin.copy()
    dup[3] = dup[2]
    assert call(og=dup) == -7 and b"same position" in msg.value
    orphan = level.copy()
    orphan[0] = 1
    assert call(lv=orphan) == -7
    assert call(nxb=12) == -1 and b"nxb" in msg.value
    # an unbalanced mesh is the planner's own error: block (1, 1) refined,
    # and its upper-right child refined again, so that level-2 blocks touch
    # the level-0 blocks (2, 1), (1, 2) and (2, 2)
    lv1, og1, pa1, _ = fx.regrid_plan_host(mesh, err, 0.8, 0.2, 2)
    c = int(np.flatnonzero((lv1 == 1) & (og1[:, 0] == 24) & (og1[:, 1] == 24))[0])
    kids = [(48, 48), (56, 48), (48, 56), (56, 56)]
    m2 = _regridded(mesh, np.concatenate([lv1, [2] * 4]),
                    np.concatenate([og1, [[x, y, 0] for x, y in kids]]),
                    np.concatenate([pa1, [c] * 4]))
    with pytest.raises(fx.FxError, match="balanced"):
        fx.regrid_plan_host(m2, np.zeros(m2.nb), 0.8, 0.2, 2)
