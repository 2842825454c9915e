"""Seeded synthetic inputs: block meshes and primitive initial states.

This module is shared by the CUDA path, the tests and the benchmark.  It holds
mesh bookkeeping (integer block coordinates, levels, parents) and initial
conditions expressed in primitive variables (density, velocity, pressure).  It
performs none of the finite-volume method's arithmetic: no equation of state,
no reconstruction, no fluxes.  Each side converts primitives to conserved
variables with its own equation of state.

Block layout used everywhere: ``W[block][var][z][y][x]`` with ``var`` in
(rho, u, v, w, p), ``P = nxb + 2*ng`` cells per padded axis and a single
z-plane in 2D.  Interior cell ``(i, j, k)`` sits at padded index
``(i + ng, j + ng, k + ng)`` (``k`` is 0 in 2D).

Block origins are lower-corner cell indices in the block's own level lattice
(level ``l`` has ``nroot[d] * nxb * 2**l`` cells along axis ``d``), matching the
octree block organisation of the paper's PARAMESH grid (Section 2).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

OUTFLOW = 0
PERIODIC = 1
REFLECT = 2


@dataclass
class Mesh:
    """A block set: one uniform level or a 2:1-balanced octree of blocks."""

    ndim: int
    nxb: int
    ng: int
    nroot: tuple           # level-0 blocks per axis (3 entries, 1 for unused axes)
    level: np.ndarray      # int32 [nb]
    origin: np.ndarray     # int64 [nb, 3]
    parent: np.ndarray     # int32 [nb], -1 for a root block
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    bc: tuple = ((OUTFLOW, OUTFLOW),) * 3
    name: str = ""
    extra: dict = field(default_factory=dict)
    species: tuple = ()    # multispecies perfect gas: ((gamma_k, A_k), ...)

    @property
    def nb(self) -> int:
        return int(self.level.shape[0])

    @property
    def nspec(self) -> int:
        return len(self.species)

    @property
    def nvar(self) -> int:
        """Variables per cell: rho, rho u, rho v, rho w, E, then rho X_k."""
        return 5 + len(self.species)

    @property
    def P(self) -> int:
        return self.nxb + 2 * self.ng

    @property
    def PZ(self) -> int:
        return self.P if self.ndim == 3 else 1

    @property
    def shape(self) -> tuple:
        """Shape of one state buffer ``[nb, nvar, PZ, P, P]``."""
        return (self.nb, self.nvar, self.PZ, self.P, self.P)

    def is_leaf(self) -> np.ndarray:
        leaf = np.ones(self.nb, dtype=np.int32)
        par = self.parent[self.parent >= 0]
        leaf[par] = 0
        return leaf

    def leaf_zones(self) -> int:
        return int(self.is_leaf().sum()) * self.nxb ** self.ndim

    def cells_per_axis(self, lev: int) -> list:
        return [self.nroot[d] * self.nxb * (2 ** lev) if d < self.ndim else 1
                for d in range(3)]

    def bc_flat(self) -> np.ndarray:
        return np.array([self.bc[d][s] for d in range(3) for s in range(2)], dtype=np.int32)

    def cell_centers(self, b: int):
        """Physical centres of block ``b``'s interior cells as (x, y, z) arrays
        broadcastable to ``[k, j, i]``."""
        lev = int(self.level[b])
        n = self.cells_per_axis(lev)
        out = []
        for d in range(3):
            if d >= self.ndim:
                out.append(np.zeros(1))
                continue
            dx = (self.hi[d] - self.lo[d]) / n[d]
            g = self.origin[b, d] + np.arange(self.nxb)
            out.append(self.lo[d] + (g + 0.5) * dx)
        nz = self.nxb if self.ndim == 3 else 1
        x = out[0].reshape(1, 1, self.nxb)
        y = out[1].reshape(1, self.nxb, 1)
        z = out[2].reshape(nz, 1, 1)
        return x, y, z

    def cell_centers_all(self):
        """``cell_centers`` of every block at once: (x, y, z) broadcastable to
        ``[nb, k, j, i]`` (the same arithmetic per cell)."""
        n = self.nxb
        lev = np.asarray(self.level, dtype=np.int64)
        out = []
        for d in range(3):
            if d >= self.ndim:
                out.append(np.zeros((self.nb, 1)))
                continue
            ncell = np.array([self.cells_per_axis(int(l))[d] for l in range(int(lev.max()) + 1)])
            dx = (self.hi[d] - self.lo[d]) / ncell[lev]
            g = self.origin[:, d][:, None] + np.arange(n)[None, :]
            out.append(self.lo[d] + (g + 0.5) * dx[:, None])
        nz = n if self.ndim == 3 else 1
        return (out[0].reshape(self.nb, 1, 1, n), out[1].reshape(self.nb, 1, n, 1),
                out[2].reshape(self.nb, nz, 1, 1))

    def global_index_all(self):
        """``global_index`` of every block at once, broadcastable to
        ``[nb, k, j, i]``."""
        n = self.nxb
        g = []
        for d in range(3):
            if d >= self.ndim:
                g.append(np.zeros((self.nb, 1), dtype=np.int64))
            else:
                g.append(self.origin[:, d][:, None] + np.arange(n, dtype=np.int64)[None, :])
        nz = n if self.ndim == 3 else 1
        return (g[0].reshape(self.nb, 1, 1, n), g[1].reshape(self.nb, 1, n, 1),
                g[2].reshape(self.nb, nz, 1, 1))

    def global_index(self, b: int):
        """Integer cell indices of block ``b``'s interior in its level lattice."""
        g = []
        for d in range(3):
            if d >= self.ndim:
                g.append(np.zeros(1, dtype=np.int64))
            else:
                g.append(self.origin[b, d] + np.arange(self.nxb, dtype=np.int64))
        nz = self.nxb if self.ndim == 3 else 1
        return (g[0].reshape(1, 1, self.nxb), g[1].reshape(1, self.nxb, 1),
                g[2].reshape(nz, 1, 1))

    def interior(self, arr: np.ndarray) -> np.ndarray:
        """View of the interior cells of a ``[nb, 5, PZ, P, P]`` array."""
        g, n = self.ng, self.nxb
        if self.ndim == 3:
            return arr[:, :, g:g + n, g:g + n, g:g + n]
        return arr[:, :, :, g:g + n, g:g + n]


# ----------------------------------------------------------------------------
# meshes
# ----------------------------------------------------------------------------

def uniform_mesh(ndim: int, nblk: tuple, nxb: int = 16, ng: int = 4,
                 bc: int | tuple = OUTFLOW, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0),
                 name: str = "", species: tuple = ()) -> Mesh:
    """One level of ``nblk[0] x nblk[1] (x nblk[2])`` blocks, x fastest."""
    nb3 = [nblk[d] if d < ndim else 1 for d in range(3)]
    origin = []
    for k in range(nb3[2]):
        for j in range(nb3[1]):
            for i in range(nb3[0]):
                origin.append((i * nxb, j * nxb, k * nxb if ndim == 3 else 0))
    nb = len(origin)
    if isinstance(bc, int):
        bc = ((bc, bc),) * 3
    return Mesh(ndim=ndim, nxb=nxb, ng=ng, nroot=tuple(nb3),
                level=np.zeros(nb, dtype=np.int32),
                origin=np.array(origin, dtype=np.int64).reshape(nb, 3),
                parent=-np.ones(nb, dtype=np.int32), lo=tuple(lo), hi=tuple(hi),
                bc=tuple(tuple(x) for x in bc), name=name, species=tuple(species))


def refine(mesh: Mesh, refine_flags: np.ndarray, name: str = "") -> Mesh:
    """Add one finer level: every flagged leaf gets 2**ndim children.

    Children are appended after all existing blocks, in the order of their
    parents, child octant ``cx + 2*cy + 4*cz``.
    """
    level = list(mesh.level)
    origin = [tuple(o) for o in mesh.origin]
    parent = list(mesh.parent)
    leaf = mesh.is_leaf()
    nchild = 2 ** mesh.ndim
    for b in range(mesh.nb):
        if not refine_flags[b]:
            continue
        if not leaf[b]:
            raise ValueError("only leaves can be refined")
        for c in range(nchild):
            off = [(c >> d) & 1 for d in range(3)]
            o = tuple(2 * int(mesh.origin[b, d]) + off[d] * mesh.nxb if d < mesh.ndim else 0
                      for d in range(3))
            level.append(int(mesh.level[b]) + 1)
            origin.append(o)
            parent.append(b)
    nb = len(level)
    return Mesh(ndim=mesh.ndim, nxb=mesh.nxb, ng=mesh.ng, nroot=mesh.nroot,
                level=np.array(level, dtype=np.int32),
                origin=np.array(origin, dtype=np.int64).reshape(nb, 3),
                parent=np.array(parent, dtype=np.int32), lo=mesh.lo, hi=mesh.hi,
                bc=mesh.bc, name=name or mesh.name, species=mesh.species)


def sedov_refine_flags(nblk: int) -> np.ndarray:
    """Centred, cube-symmetric refined set of a ``nblk^3`` coarse block grid.

    A coarse block ``(i, j, k)`` is refined iff the descending-sorted triple of
    ``o(x) = |x - c| - 1/2`` (``c = (nblk - 1) / 2``) is one of (0,0,0),
    (1,0,0), (1,1,0), (2,0,0), (2,1,0).  For ``nblk = 8`` this refines exactly
    128 blocks.  For smaller grids the same rule refines the centre.
    """
    c = (nblk - 1) / 2.0
    allowed = {(0, 0, 0), (1, 0, 0), (1, 1, 0), (2, 0, 0), (2, 1, 0)}
    flags = []
    for k in range(nblk):
        for j in range(nblk):
            for i in range(nblk):
                o = tuple(sorted((int(round(abs(x - c) - 0.5)) for x in (i, j, k)), reverse=True))
                flags.append(o in allowed)
    return np.array(flags, dtype=bool)


def sedov_mesh(nblk: int = 8, nxb: int = 16, ng: int = 4, bc: int = OUTFLOW) -> Mesh:
    """Two-level octree for the Sedov blast: ``nblk^3`` coarse blocks, the
    centre refined once (512 coarse + 1024 fine blocks at ``nblk = 8``)."""
    base = uniform_mesh(3, (nblk, nblk, nblk), nxb, ng, bc)
    return refine(base, sedov_refine_flags(nblk), name=f"sedov_amr_{nblk}")


# ----------------------------------------------------------------------------
# initial conditions (primitive variables rho, u, v, w, p)
# ----------------------------------------------------------------------------

def _empty(mesh: Mesh) -> np.ndarray:
    return np.zeros(mesh.shape, dtype=np.float64)


def _fill_all(mesh: Mesh, W: np.ndarray, fields) -> None:
    """Interior of every block from fields broadcastable to ``[nb, k, j, i]``."""
    g, n = mesh.ng, mesh.nxb
    nz = n if mesh.ndim == 3 else 1
    for v in range(len(fields)):
        val = np.broadcast_to(fields[v], (mesh.nb, nz, n, n))
        if mesh.ndim == 3:
            W[:, v, g:g + n, g:g + n, g:g + n] = val
        else:
            W[:, v, 0, g:g + n, g:g + n] = val[:, 0]


def _fill(mesh: Mesh, W: np.ndarray, b: int, fields) -> None:
    g, n = mesh.ng, mesh.nxb
    for v in range(len(fields)):
        val = np.broadcast_to(fields[v], (n if mesh.ndim == 3 else 1, n, n))
        if mesh.ndim == 3:
            W[b, v, g:g + n, g:g + n, g:g + n] = val
        else:
            W[b, v, 0, g:g + n, g:g + n] = val


def sod_state(mesh: Mesh, axis: int = 0, mirror: bool = False) -> np.ndarray:
    """Sod shock tube: (rho, p) = (1, 1) for x < 0.5 and (0.125, 0.1) otherwise,
    at rest.  ``mirror`` swaps the two sides."""
    W = _empty(mesh)
    xyz = mesh.cell_centers_all()
    left = xyz[axis] < 0.5
    if mirror:
        left = ~left
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    z = np.zeros(1)
    _fill_all(mesh, W, (rho, z, z, z, p))
    return W


def uniform_state(mesh: Mesh, rho=1.3, vel=(0.3, -0.2, 0.1), p=0.7) -> np.ndarray:
    W = _empty(mesh)
    v = list(vel)
    if mesh.ndim == 2:
        v[2] = 0.0
    _fill_all(mesh, W, (np.array(rho), np.array(v[0]), np.array(v[1]), np.array(v[2]),
                        np.array(p)))
    return W


def kh_state(mesh: Mesh, seed: int = 1234, amp: float = 0.01) -> np.ndarray:
    """Kelvin-Helmholtz shear layer: rho = 2, vx = +0.5 for |y - 0.5| < 0.25,
    else rho = 1, vx = -0.5; p = 2.5; vy = amp * (2r - 1) with one uniform
    draw r per cell of the level-0 lattice (index order [z][y][x], seed
    ``seed``); vz = 0."""
    W = _empty(mesh)
    n = mesh.cells_per_axis(0)
    rng = np.random.default_rng(seed)
    r = rng.random((n[2], n[1], n[0]))
    x, y, z = mesh.cell_centers_all()
    gx, gy, gz = mesh.global_index_all()
    inner = np.abs(y - 0.5) < 0.25
    rho = np.where(inner, 2.0, 1.0)
    vx = np.where(inner, 0.5, -0.5)
    s = (2 ** np.asarray(mesh.level, dtype=np.int64)).reshape(mesh.nb, 1, 1, 1)
    vy = amp * (2.0 * r[gz // s, gy // s, gx // s] - 1.0)
    _fill_all(mesh, W, (rho, vx, vy, np.zeros(1), np.array(2.5)))
    return W


def sedov_state(mesh: Mesh, e_blast: float = 1.0, r_cells: float = 3.5,
                gamma: float = 1.4) -> np.ndarray:
    """Sedov blast: rho = 1, p = 1e-5 at rest; the energy ``e_blast`` spread
    uniformly over the finest-level cells whose centres lie within
    ``r_cells`` finest cell widths of the domain centre.

    The pressure there is ``(gamma - 1) * e_blast / (count * dV)`` with
    ``count`` the number of such cells.  That is the ideal-gas relation between
    internal energy density and pressure; it fixes the input, not the scheme.
    """
    W = _empty(mesh)
    lmax = int(mesh.level.max())
    nf = mesh.cells_per_axis(lmax)
    dxf = [(mesh.hi[d] - mesh.lo[d]) / nf[d] for d in range(3)]
    ctr = [0.5 * (mesh.lo[d] + mesh.hi[d]) for d in range(3)]
    leaf = mesh.is_leaf().astype(bool)
    x, y, z = mesh.cell_centers_all()
    r2 = ((x - ctr[0]) / dxf[0]) ** 2 + ((y - ctr[1]) / dxf[1]) ** 2 + \
         ((z - ctr[2]) / dxf[2]) ** 2
    finest = (np.asarray(mesh.level) == lmax).reshape(mesh.nb, 1, 1, 1)
    inside = (r2 < r_cells ** 2) & finest
    count = int(inside[leaf].sum())
    if count == 0:
        raise ValueError("blast region holds no finest-level cells")
    dv = dxf[0] * dxf[1] * dxf[2]
    p_in = (gamma - 1.0) * e_blast / (count * dv)
    p = np.where(inside, p_in, 1e-5)
    _fill_all(mesh, W, (np.array(1.0), np.zeros(1), np.zeros(1), np.zeros(1), p))
    mesh.extra["sedov_cells"] = count
    mesh.extra["sedov_p"] = p_in
    return W


def advection_modes(seed: int = 2208, nmodes: int = 8, kmax: int = 4):
    """Wave vectors k_m in {-kmax..kmax}^3 with 1 <= |k_m|_inf <= kmax and
    phases in [0, 2 pi), drawn with ``default_rng(seed)``."""
    rng = np.random.default_rng(seed)
    ks = []
    while len(ks) < nmodes:
        k = rng.integers(-kmax, kmax + 1, size=3)
        if 1 <= np.max(np.abs(k)) <= kmax:
            ks.append(k)
    phases = rng.uniform(0.0, 2.0 * np.pi, size=nmodes)
    return np.array(ks, dtype=np.int64), phases


def advection_density(x, y, z, t=0.0, vel=(1.0, 0.5, 0.25), seed=2208, nmodes=8,
                      kmax=4, amp=0.1):
    """rho(x - v t) = 1 + amp * sum_m sin(2 pi k_m . (x - v t) + phi_m)."""
    ks, ph = advection_modes(seed, nmodes, kmax)
    xs = (x - vel[0] * t, y - vel[1] * t, z - vel[2] * t)
    rho = 1.0
    for m in range(len(ks)):
        arg = 2.0 * np.pi * (ks[m, 0] * xs[0] + ks[m, 1] * xs[1] + ks[m, 2] * xs[2]) + ph[m]
        rho = rho + amp * np.sin(arg)
    return rho


def advection_state(mesh: Mesh, vel=(1.0, 0.5, 0.25), seed=2208, nmodes=8, kmax=4,
                    amp=0.1) -> np.ndarray:
    """Smooth advection: p = 1, uniform velocity, Fourier-mode density."""
    W = _empty(mesh)
    x, y, z = mesh.cell_centers_all()
    rho = advection_density(x, y, z, 0.0, vel, seed, nmodes, kmax, amp)
    _fill_all(mesh, W, (rho, np.array(vel[0]), np.array(vel[1]),
                        np.array(vel[2] if mesh.ndim == 3 else 0.0), np.array(1.0)))
    return W


def random_smooth_state(mesh: Mesh, seed: int = 7) -> np.ndarray:
    """Positive, smooth-ish random state for unit and parity tests: a few
    random Fourier modes per field on top of a positive background."""
    rng = np.random.default_rng(seed)
    W = _empty(mesh)
    base = np.array([1.0, 0.2, -0.1, 0.05, 1.0])
    amps = np.array([0.3, 0.4, 0.4, 0.4, 0.3])
    ks = rng.integers(-3, 4, size=(5, 3, 3))
    ph = rng.uniform(0, 2 * np.pi, size=(5, 3))
    for b in range(mesh.nb):
        x, y, z = mesh.cell_centers(b)
        fields = []
        for v in range(5):
            f = base[v]
            for m in range(3):
                f = f + amps[v] / 3 * np.sin(2 * np.pi * (ks[v, m, 0] * x + ks[v, m, 1] * y +
                                                          ks[v, m, 2] * z) + ph[v, m])
            if v == 3 and mesh.ndim == 2:
                f = np.zeros(1)
            fields.append(np.asarray(f))
        _fill(mesh, W, b, fields)
    return W


def random_blocky_state(mesh: Mesh, seed: int = 11) -> np.ndarray:
    """Independent uniform draws per cell (positive rho and p): maximally
    non-smooth data, used to exercise every limiter and Riemann branch."""
    rng = np.random.default_rng(seed)
    W = _empty(mesh)
    g, n = mesh.ng, mesh.nxb
    nz = n if mesh.ndim == 3 else 1
    for b in range(mesh.nb):
        rho = rng.uniform(0.5, 2.0, size=(nz, n, n))
        u = rng.uniform(-1.5, 1.5, size=(nz, n, n))
        v = rng.uniform(-1.5, 1.5, size=(nz, n, n))
        w = rng.uniform(-1.5, 1.5, size=(nz, n, n)) if mesh.ndim == 3 else np.zeros(1)
        p = rng.uniform(0.5, 2.0, size=(nz, n, n))
        _fill(mesh, W, b, (rho, u, v, w, p))
    return W


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

def workload_mesh(name: str, scale: int | None = None) -> Mesh:
    """The mesh of a named workload (see ``workload``), without its state."""
    if name == "sod2d":
        n = scale or 8
        return uniform_mesh(2, (n, n), 16, 4, OUTFLOW, name="sod2d")
    if name == "kh3d":
        n = scale or 16
        return uniform_mesh(3, (n, n, n), 16, 4, PERIODIC, name="kh3d")
    if name == "sedov_amr":
        return sedov_mesh(scale or 8, 16, 4, OUTFLOW)
    if name == "advection3d":
        n = scale or 32
        return uniform_mesh(3, (n, n, n), 16, 4, PERIODIC, name="advection3d")
    raise KeyError(name)


def workload(name: str, scale: int | None = None):
    """Return ``(mesh, W0, gamma, cfl)`` for a named workload.

    * ``sod2d``: [0,1]^2, 8x8 blocks of 16^2 (+4 guard), outflow.
    * ``kh3d``: [0,1]^3, ``scale``^3 blocks of 16^3 (16 -> 256^3), periodic.
    * ``sedov_amr``: 8^3 coarse blocks of 16^3 + 1024 fine blocks, outflow.
    * ``advection3d``: [0,1]^3, ``scale``^3 blocks of 16^3 (32 -> 512^3), periodic.
    """
    gamma, cfl = 1.4, 0.8
    mesh = workload_mesh(name, scale)
    state = {"sod2d": sod_state, "kh3d": kh_state, "advection3d": advection_state,
             "sedov_amr": lambda m: sedov_state(m, gamma=gamma)}[name]
    return mesh, state(mesh), gamma, cfl
