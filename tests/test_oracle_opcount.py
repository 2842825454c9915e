"""The op-counting build of the oracle (oracle/opcount.cpp) that gives the
benchmark its flops per zone update.

Pins: the counting build computes exactly what the normal build computes
(bit for bit, so the operations counted are the oracle's own), and the
counts of the steps whose arithmetic does not depend on the data equal the
counts read off their definitions by hand:
* primitives of a cell: u_d = m_d / rho (3 divisions) and
  p = (gamma - 1)(E - 0.5 |m|^2 / rho): 3 mul + 2 add for |m|^2, 1 mul by
  0.5, 1 division, 1 sub, 1 sub for gamma - 1, 1 mul -- 2 add, 2 sub, 5 mul,
  4 div;
* conservative update of a cell, per variable and direction (F- - F+) / dx
  summed, then U + dt * sum: 5 x (3 sub, 3 div, 3 add, 1 mul, 1 add);
* CFL signal speed of a cell (sum form, 3D): the primitives, c = sqrt(gamma p
  / rho) (1 mul, 1 div, 1 sqrt), per direction (|u_d| + c) / dx_d added to
  the sum (2 add, 1 div); and the step's one division dt = cfl / max.
"""
import pytest

opcount = pytest.importorskip("oracle.opcount")


@pytest.fixture(scope="module")
def kh():
    return opcount.count_step("kh3d", scale=2, warm=3)


def test_counting_build_computes_what_the_oracle_computes(orc, kh):
    assert kh["same_as_oracle"]
    r = opcount.count_step("sedov_amr", scale=2, warm=2)   # AMR: reflux, prolongation
    assert r["same_as_oracle"]


def test_data_independent_counts_match_the_definitions(kh):
    u = kh["per_unit"]
    prim = u[opcount.STEPS[0]]
    assert (prim["add"], prim["sub"], prim["mul"], prim["div"], prim["sqrt"]) == (2, 2, 5, 4, 0)
    upd = u[opcount.STEPS[3]]
    assert (upd["add"], upd["sub"], upd["mul"], upd["div"], upd["sqrt"]) == (20, 15, 5, 15, 0)
    sig = u[opcount.STEPS[5]]
    assert (sig["add"], sig["sub"], sig["mul"], sig["sqrt"]) == (2 + 6, 2, 5 + 1, 1)
    # 4 + 1 + 3 divisions per cell, plus the one dt = cfl / max of the step
    assert sig["div"] * sig["units"] == (4 + 1 + 3) * sig["units"] + 1


def test_units_follow_the_block_loops(kh):
    """Units opened per step equal the oracle's loop extents: primitives on
    every padded cell, the predictor on the interior grown by one, the faces
    of the interior (n + 1 per row per direction), the interior cells."""
    n, g, nb = 16, 4, 8
    u = kh["per_unit"]
    assert u[opcount.STEPS[0]]["units"] == nb * (n + 2 * g) ** 3
    assert u[opcount.STEPS[1]]["units"] == nb * (n + 2) ** 3
    assert u[opcount.STEPS[2]]["units"] == nb * 3 * (n + 1) * n * n
    assert u[opcount.STEPS[3]]["units"] == nb * n ** 3
    assert u[opcount.STEPS[5]]["units"] == nb * n ** 3
    # the algorithmic count per zone: within the range a hand count of the
    # scheme gives (HLLC about 100 flops per face, predictor about 220)
    assert 550 < kh["algorithmic_per_zone"] < 700


@pytest.mark.parametrize("name,scale", [("kh3d", 4), ("sedov_amr", 4), ("advection3d", 4),
                                        ("sod2d", 0)])
def test_bench_flops_per_zone_are_the_counted_ones(name, scale):
    """The benchmark's algorithmic flops per zone update (its FP64 roofline
    numerator) are this build's counts for the documented commands
    (`python -m oracle.opcount <workload> <scale> 10`), to the printed digit."""
    import bench
    r = opcount.count_step(name, scale=scale, warm=10)
    assert round(r["algorithmic_per_zone"], 1) == bench.ALGO_FLOPS_PER_ZONE[name]
