"""The synthetic workloads against their stated recipes, on CPU: the meshes
at full size (block counts, levels, zones, boundaries) and the initial
states at full size where they are small, else at a reduced scale that
keeps the recipe (Sod shock tube, the 3D shear layer, the Sedov deposit,
the Fourier-mode density of the advection test)."""
import itertools
import math

import numpy as np
import pytest

from paper_2208_11630_gb300 import inputs

O_, P_ = inputs.OUTFLOW, inputs.PERIODIC


@pytest.mark.parametrize("name,blocks,leaves,zones,bc,ndim", [
    ("sod2d", 64, 64, 128 ** 2, O_, 2),
    ("kh3d", 4096, 4096, 256 ** 3, P_, 3),
    ("sedov_amr", 1536, 1408, 1408 * 16 ** 3, O_, 3),
    ("advection3d", 32768, 32768, 512 ** 3, P_, 3),
])
def test_full_size_meshes(name, blocks, leaves, zones, bc, ndim):
    m = inputs.workload_mesh(name)
    assert m.ndim == ndim and m.nxb == 16 and m.ng == 4
    assert m.nb == blocks and int(m.is_leaf().sum()) == leaves and m.leaf_zones() == zones
    assert all(m.bc[d] == (bc, bc) for d in range(ndim))


def test_sedov_refined_set_is_128_cube_symmetric_blocks():
    f = inputs.sedov_refine_flags(8).reshape(8, 8, 8)   # [k][j][i]
    assert f.sum() == 128
    for perm in itertools.permutations(range(3)):
        g = f.transpose(perm)
        for flips in itertools.product([False, True], repeat=3):
            h = g
            for ax, fl in enumerate(flips):
                if fl:
                    h = np.flip(h, ax)
            assert np.array_equal(h, f)
    m = inputs.workload_mesh("sedov_amr")
    assert np.bincount(m.level).tolist() == [512, 1024]
    assert (m.is_leaf() == 0).sum() == 128


def test_sod_state_recipe():
    m, W, gamma, cfl = inputs.workload("sod2d")
    assert (gamma, cfl) == (1.4, 0.8)
    I = m.interior(W)
    for b in range(m.nb):
        x = m.cell_centers(b)[0].ravel()
        left = x < 0.5
        assert np.all(I[b, 0, 0][:, left] == 1.0) and np.all(I[b, 4, 0][:, left] == 1.0)
        assert np.all(I[b, 0, 0][:, ~left] == 0.125) and np.all(I[b, 4, 0][:, ~left] == 0.1)
        assert np.all(I[b, 1:4] == 0.0)
    # the interface is a cell face: exactly half the columns on each side
    assert (I[:, 0] == 1.0).sum() == (I[:, 0] == 0.125).sum() == 128 ** 2 // 2


def test_kh_state_recipe():
    m, W, _, _ = inputs.workload("kh3d", scale=4)     # 64^3, the same recipe
    I = m.interior(W)
    r = np.random.default_rng(1234).random((64, 64, 64))  # one draw per cell, [z][y][x]
    for b in range(m.nb):
        x, y, z = m.cell_centers(b)
        gx, gy, gz = m.global_index(b)
        inner = np.broadcast_to(np.abs(y - 0.5) < 0.25, (16, 16, 16))
        assert np.all(I[b, 0][inner] == 2.0) and np.all(I[b, 0][~inner] == 1.0)
        assert np.all(I[b, 1][inner] == 0.5) and np.all(I[b, 1][~inner] == -0.5)
        assert np.array_equal(I[b, 2], 0.01 * (2.0 * r[gz, gy, gx] - 1.0))
        assert np.all(I[b, 3] == 0.0) and np.all(I[b, 4] == 2.5)
    # the band |y - 0.5| < 0.25 holds half the cells (faces at y = 0.25, 0.75)
    assert (I[:, 0] == 2.0).sum() * 2 == 64 ** 3
    vy = I[:, 2]
    assert np.abs(vy).max() < 0.01 and abs(vy.mean()) < 4 * 0.01 / math.sqrt(3 * 64 ** 3)


def test_sedov_deposit_recipe():
    # the deposit covers the finest cells whose centres lie within 3.5 finest
    # widths of the centre: 160 of them, counted here by brute force over
    # half-integer offsets from the (cell-corner) centre
    offs = np.arange(-3.5, 4.0, 1.0)
    a, b, c = np.meshgrid(offs, offs, offs, indexing="ij")
    assert int(((a ** 2 + b ** 2 + c ** 2) < 3.5 ** 2).sum()) == 160
    # at full size: p = (gamma - 1) / (160 dV_fine) with dV = 256^-3
    assert 0.4 / (160 * 256.0 ** -3) == pytest.approx(41943.04, rel=1e-15)
    # a reduced two-level mesh keeps the recipe: 160 cells, total energy 1
    m = inputs.sedov_mesh(4, 16, 4)
    W = inputs.sedov_state(m, gamma=1.4)
    dvf = 128.0 ** -3
    assert m.extra["sedov_cells"] == 160
    assert m.extra["sedov_p"] == pytest.approx(0.4 / (160 * dvf), rel=1e-15)
    I = m.interior(W)
    leaf = m.is_leaf() == 1
    hot = I[leaf, 4] > 1.0
    assert hot.sum() == 160
    e_int = (I[leaf, 4][hot] / 0.4).sum() * dvf
    assert e_int == pytest.approx(1.0, rel=1e-13)
    assert np.all(I[leaf, 4][~hot] == 1e-5) and np.all(I[:, 0] == 1.0) and np.all(I[:, 1:4] == 0.0)


def test_advection_state_recipe():
    ks, ph = inputs.advection_modes()
    assert ks.shape == (8, 3) and np.all(np.abs(ks).max(axis=1) >= 1)
    assert np.all(np.abs(ks).max(axis=1) <= 4) and np.all((ph >= 0) & (ph < 2 * np.pi))
    m, W, _, _ = inputs.workload("advection3d", scale=2)   # 32^3
    I = m.interior(W)
    assert np.all(I[:, 1] == 1.0) and np.all(I[:, 2] == 0.5) and np.all(I[:, 3] == 0.25)
    assert np.all(I[:, 4] == 1.0)
    rho = I[:, 0]
    assert rho.min() >= 0.2 and rho.max() <= 1.8
    # integer wave vectors resolved by the grid: each mode sums to zero over
    # the cell centres, so the mean density is 1
    assert abs(rho.mean() - 1.0) < 1e-13
    # rho(x - v t) is the initial profile again at t = 4, when every axis has
    # been crossed a whole number of times (4, 2 and 1); at t = 1 only x has
    x, y, z = m.cell_centers(0)
    assert np.allclose(inputs.advection_density(x, y, z, t=4.0), rho[0], rtol=0, atol=1e-12)
    assert not np.allclose(inputs.advection_density(x, y, z, t=1.0), rho[0], rtol=0, atol=1e-6)
