"""Test helpers: assembling block data into global arrays and comparing states.

Nothing here computes the finite-volume method; it only rearranges arrays.
"""
from __future__ import annotations

import numpy as np


def assemble(mesh, U, level=None, leaves_only=True):
    """Assemble interior cells of ``U`` ``[nb, 5, PZ, P, P]`` into a global
    array ``[5, Nz, Ny, Nx]`` at ``level`` (default: the finest).  Coarser
    leaves are repeated 2x per axis per level; finer data is not averaged
    (a finer leaf inside a coarser region at ``level`` is skipped)."""
    lmax = int(mesh.level.max())
    level = lmax if level is None else level
    n = mesh.nxb
    N = mesh.cells_per_axis(level)
    G = np.full((U.shape[1], N[2], N[1], N[0]), np.nan)
    leaf = mesh.is_leaf()
    for b in range(mesh.nb):
        lb = int(mesh.level[b])
        if leaves_only and not leaf[b]:
            continue
        if lb > level:
            continue
        r = 2 ** (level - lb)
        blk = mesh.interior(U[b:b + 1])[0]
        if r > 1:
            blk = blk.repeat(r, axis=3).repeat(r, axis=2)
            if mesh.ndim == 3:
                blk = blk.repeat(r, axis=1)
        o = [int(mesh.origin[b, d]) * r for d in range(3)]
        if mesh.ndim == 3:
            G[:, o[2]:o[2] + n * r, o[1]:o[1] + n * r, o[0]:o[0] + n * r] = blk
        else:
            G[:, 0:1, o[1]:o[1] + n * r, o[0]:o[0] + n * r] = blk
    return G


def rel_err(a, b, axis_var=1):
    """Per-cell relative error |a - b| / max(|b|, s_var), with s_var the
    largest |b| of that variable over the compared cells."""
    a = np.asarray(a)
    b = np.asarray(b)
    nv = a.shape[axis_var]
    moved_a = np.moveaxis(a, axis_var, 0).reshape(nv, -1)
    moved_b = np.moveaxis(b, axis_var, 0).reshape(nv, -1)
    s = np.abs(moved_b).max(axis=1, keepdims=True)
    s = np.where(s == 0, 1.0, s)
    den = np.maximum(np.abs(moved_b), s)
    return np.abs(moved_a - moved_b) / den


def max_rel_err(mesh, a, b):
    """Max of ``rel_err`` over the leaf interior cells."""
    leaf = mesh.is_leaf().astype(bool)
    ia = mesh.interior(a)[leaf]
    ib = mesh.interior(b)[leaf]
    return float(rel_err(ia, ib).max())


def leaf_interior(mesh, U):
    leaf = mesh.is_leaf().astype(bool)
    return mesh.interior(U)[leaf]


def max_rel_err_vec(mesh, a, b):
    """Like ``max_rel_err`` but the three momentum components share one scale,
    the largest momentum magnitude |m| over the compared cells.  Used where a
    component is near zero everywhere (e.g. m_z of a 3D shear layer after one
    step), so that its absolute roundoff is judged against the flow's
    momentum rather than against its own vanishing maximum."""
    leaf = mesh.is_leaf().astype(bool)
    nv = a.shape[1]
    ia = np.moveaxis(mesh.interior(a)[leaf], 1, 0).reshape(nv, -1)
    ib = np.moveaxis(mesh.interior(b)[leaf], 1, 0).reshape(nv, -1)
    s = np.abs(ib).max(axis=1)
    s[1:4] = np.sqrt((ib[1:4] ** 2).sum(axis=0)).max()
    s = np.where(s == 0, 1.0, s)[:, None]
    return float((np.abs(ia - ib) / np.maximum(np.abs(ib), s)).max())
