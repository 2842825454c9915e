"""Sharding plan of a block set over several ranks (one rank per GPU).

Paper: Flash-X (arXiv 2208.11630), Section 1 -- FLASH was designed for
distributed memory, with the mesh's blocks spread over processes; Section 2
-- physics updates one block at a time from its guard cells, which the Grid
unit fills.  A step therefore needs, on each rank, only the data of the
blocks it owns and of the blocks those updates read.

The plan here (this design's choice; the paper prints none):

* ``partition``: the leaves, ordered along a Z-order (Morton) curve of their
  lower corners on the finest block lattice, are cut into ``nranks``
  contiguous runs of equal zone counts (every leaf holds the same zones), so
  that each rank owns a compact region.
* ``halo``: the leaves a rank must receive before a step -- every leaf
  within ``rings`` touch-steps (faces, edges, corners, periodic wrap) of one
  it owns.  Three rings are a safe bound: what the update of an owned leaf
  reads is reached by at most three such steps -- its touching leaves, a
  coarser neighbour's limited slopes (which read that neighbour's touching
  leaves), and for flux correction a finer neighbour's face fluxes (whose
  transverse guards may be prolonged from a leaf touching that neighbour).
  In practice one ring suffices for blocks of 8 or more cells: a leaf that
  touches no owned leaf lies at least one block of the next finer level (4
  cells of the owned leaf's level) away, beyond the two-cell stencil and the
  one coarse cell of slope support it could feed.  The CPU tests confirm it
  by brute force (perturbing each block in turn, one step reaches only the
  leaves touching it, and a parent reaches nothing) and find one ring
  bit-identical to the unsharded run on every mesh they step (8-cell blocks,
  two and three levels, periodic and outflow).  That holds per stage: an
  SSP-RK step would exchange its halo before each stage, or take a ring per
  stage.  The default keeps the safe bound.
* ``exchange_lists``: for each ordered pair of ranks, the blocks the first
  owns that lie in the second's halo -- one message per pair and step.  The
  lists name whole blocks, which is what the CPU emulation moves; a GPU
  exchange would pack only the cells the receiver reads, a shell two cells
  deep around its region (plus one coarse cell of slope support at
  coarse-fine faces).  For the 256^3 shear layer on 8 ranks (8^3 blocks of
  16^3 each) that shell is 132^3 - 128^3 cells, 9.7 % of a rank's state,
  against 0.95x for one ring of whole blocks and 4.4x for three.
* dt is the CFL limit of each rank's own data, combined by a MIN reduction
  (the CFL number divided by the largest signal speed is monotone in that
  speed, so the minimum over ranks is the global value bit for bit).

The benchmark's multi-rank runs advance independent replicas (no data-path
exchange); this plan is exercised on CPU ranks (gloo), with the FP64 oracle
doing the arithmetic, against an unsharded run.
"""
from __future__ import annotations

from collections import deque

import numpy as np

__all__ = ["finest_corners", "morton_keys", "partition", "leaf_adjacency", "halo",
           "exchange_lists"]


def finest_corners(mesh):
    """Per block: the lower corner and the side (per axis), in units of
    blocks of the finest level present, of the region the block covers."""
    lmax = int(mesh.level.max())
    lo = np.zeros((mesh.nb, 3), dtype=np.int64)
    side = np.ones(mesh.nb, dtype=np.int64)
    for b in range(mesh.nb):
        s = 1 << (lmax - int(mesh.level[b]))
        side[b] = s
        for d in range(mesh.ndim):
            lo[b, d] = (int(mesh.origin[b, d]) // mesh.nxb) * s
    return lo, side


def morton_keys(mesh):
    """Z-order key of each block's lower corner on the finest block lattice
    (bits of x, y, z interleaved, x lowest)."""
    lo, _ = finest_corners(mesh)
    keys = np.zeros(mesh.nb, dtype=np.int64)
    nbits = int(max(1, int(lo.max()) + 1).bit_length())
    for b in range(mesh.nb):
        k = 0
        for i in range(nbits):
            for d in range(mesh.ndim):
                k |= ((int(lo[b, d]) >> i) & 1) << (mesh.ndim * i + d)
        keys[b] = k
    return keys


def partition(mesh, nranks: int) -> np.ndarray:
    """Owner rank of every block: leaves in contiguous Z-order runs of equal
    size (the first ``nleaves % nranks`` runs one longer); parents -1."""
    if nranks < 1:
        raise ValueError("nranks must be positive")
    leaf = np.flatnonzero(mesh.is_leaf() == 1)
    order = leaf[np.argsort(morton_keys(mesh)[leaf], kind="stable")]
    owner = np.full(mesh.nb, -1, dtype=np.int64)
    cuts = [len(order) * r // nranks for r in range(nranks + 1)]
    for r in range(nranks):
        owner[order[cuts[r]:cuts[r + 1]]] = r
    return owner


def leaf_adjacency(mesh):
    """For each leaf, the sorted leaves that touch it (share a face, an edge
    or a corner; periodic axes wrap); empty for parents.  Paints the finest
    block lattice (one int64 per finest-level block: 32^3 for the 512^3
    uniform workload, 16^3 for the two-level Sedov mesh); deep hierarchies
    would want a hashed lookup like the library's regrid planner."""
    lo, side = finest_corners(mesh)
    n = [int(mesh.nroot[d]) << int(mesh.level.max()) if d < mesh.ndim else 1 for d in range(3)]
    periodic = [mesh.bc[d][0] == 1 for d in range(3)]
    paint = np.full((n[2], n[1], n[0]), -1, dtype=np.int64)
    leaf = mesh.is_leaf() == 1
    for b in np.flatnonzero(leaf):
        x0, y0, z0 = lo[b]
        s = int(side[b])
        sz = s if mesh.ndim == 3 else 1
        paint[z0:z0 + sz, y0:y0 + s, x0:x0 + s] = b
    if np.any(paint < 0):
        raise ValueError("the leaves do not cover the domain")
    out = [np.zeros(0, dtype=np.int64) for _ in range(mesh.nb)]
    for b in np.flatnonzero(leaf):
        s = int(side[b])
        ranges = []
        for d in range(3):
            if d >= mesh.ndim:
                ranges.append(np.zeros(1, dtype=np.int64))
                continue
            r = np.arange(lo[b, d] - 1, lo[b, d] + s + 1)
            if periodic[d]:
                r = r % n[d]
            else:
                r = r[(r >= 0) & (r < n[d])]
            ranges.append(r)
        found = paint[np.ix_(ranges[2], ranges[1], ranges[0])].ravel()
        found = np.unique(found)
        out[b] = found[found != b]
    return out


def halo(mesh, owner, rank: int, rings: int = 3, adjacency=None) -> np.ndarray:
    """Leaves not owned by ``rank`` within ``rings`` touch-steps of one it
    owns (sorted)."""
    adj = adjacency if adjacency is not None else leaf_adjacency(mesh)
    owned = np.flatnonzero(owner == rank)
    dist = {int(b): 0 for b in owned}
    q = deque(int(b) for b in owned)
    while q:
        b = q.popleft()
        if dist[b] == rings:
            continue
        for c in adj[b]:
            c = int(c)
            if c not in dist:
                dist[c] = dist[b] + 1
                q.append(c)
    return np.array(sorted(b for b in dist if owner[b] != rank), dtype=np.int64)


def exchange_lists(mesh, owner, nranks: int, rings: int = 3):
    """``{(src, dst): blocks}``: the blocks ``src`` owns that lie in the
    halo of ``dst`` (sorted), for every ordered pair with something to send."""
    adj = leaf_adjacency(mesh)
    out = {}
    for dst in range(nranks):
        h = halo(mesh, owner, dst, rings, adj)
        for src in range(nranks):
            if src == dst:
                continue
            blocks = h[owner[h] == src]
            if len(blocks):
                out[(src, dst)] = blocks
    return out
