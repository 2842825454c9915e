"""Host side of the serving stream on CPU: the request generator follows the
serving workload's recipe (Poisson arrivals; blocks log-uniform over
8..4096; nxb uniform over {8, 16, 32}; k uniform over 1..20; the four
setups and the two precisions equally likely), block counts factor into
balanced root grids, and every request's problem is a valid mesh with a
physical initial state.  The serving loop itself needs the GPU."""
import math

import numpy as np
import pytest

from paper_2208_11630_gb300 import fx
from paper_2208_11630_gb300 import serve as sv

N = 2000


@pytest.fixture(scope="module")
def stream():
    return sv.make_stream(N, rate=50.0)


def test_stream_is_seeded_and_deterministic(stream):
    again = sv.make_stream(N, rate=50.0)
    assert [(r.setup, r.nblocks, r.nxb, r.precision, r.k, r.arrival) for r in stream] == \
           [(r.setup, r.nblocks, r.nxb, r.precision, r.k, r.arrival) for r in again]
    other = sv.make_stream(N, rate=50.0, seed=1)
    assert [r.nblocks for r in other] != [r.nblocks for r in stream]


def test_arrivals_are_poisson(stream):
    t = np.array([r.arrival for r in stream])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps >= 0)
    # exponential gaps: mean 1/rate, coefficient of variation 1 (4 sigma)
    assert abs(gaps.mean() * 50.0 - 1.0) < 4 / math.sqrt(N)
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1
    burst = sv.make_stream(20, rate=float("inf"))
    assert all(r.arrival == 0.0 for r in burst)


def test_request_mix_follows_the_recipe(stream):
    nb = np.array([r.nblocks for r in stream])
    assert nb.min() >= 8 and nb.max() <= 4096
    # log-uniform: ln(nb) uniform on [ln 8, ln 4096] (mean and spread, 4 sigma)
    u = (np.log(nb) - math.log(8)) / (math.log(4096) - math.log(8))
    sd = 1 / math.sqrt(12)
    assert abs(u.mean() - 0.5) < 4 * sd / math.sqrt(N)
    assert abs(u.std() - sd) < 0.02
    k = np.array([r.k for r in stream])
    assert set(k.tolist()) == set(range(1, 21))
    assert abs(k.mean() - 10.5) < 4 * math.sqrt((20 ** 2 - 1) / 12) / math.sqrt(N)

    def share(values, expected):
        values = list(values)
        for v in expected:
            p = values.count(v) / len(values)
            q = 1 / len(expected)
            assert abs(p - q) < 4 * math.sqrt(q * (1 - q) / len(values)), (v, p)

    share((r.nxb for r in stream), (8, 16, 32))
    share((r.setup for r in stream), sv.SETUPS)
    share((r.precision for r in stream), (fx.FX_F64, fx.FX_F32BULK))


def test_new_arrivals_keep_the_requests(stream):
    later = sv.with_arrivals(stream[:200], rate=5.0)
    assert [(r.rid, r.nblocks, r.k) for r in later] == [(r.rid, r.nblocks, r.k) for r in stream[:200]]
    t = np.array([r.arrival for r in later])
    assert np.all(np.diff(t) >= 0) and abs(t[-1] / 200 * 5.0 - 1.0) < 0.3


@pytest.mark.parametrize("nb", [8, 12, 30, 64, 97, 360, 1024, 4096, 4095])
@pytest.mark.parametrize("parts", [2, 3])
def test_factor_is_a_balanced_exact_product(nb, parts):
    dims = sv._factor(nb, parts)
    assert len(dims) == parts and math.prod(dims) == nb
    assert list(dims) == sorted(dims, reverse=True)
    # balanced: no part exceeds another by more than the largest prime factor
    p, rest, largest = 2, nb, 1
    while p * p <= rest:
        while rest % p == 0:
            largest, rest = max(largest, p), rest // p
        p += 1
    largest = max(largest, rest)
    assert dims[0] <= max(dims[-1], 1) * largest


@pytest.mark.parametrize("setup", sv.SETUPS)
@pytest.mark.parametrize("nblocks,nxb", [(8, 8), (27, 16), (40, 8)])
def test_request_problem_is_valid(setup, nblocks, nxb):
    req = sv.Request(0, setup, nblocks, nxb, fx.FX_F64, 3, 0.0)
    mesh, W = sv.request_problem(req)
    assert mesh.nxb == nxb and mesh.ndim == (2 if setup == "sod" else 3)
    if setup == "sedov":
        # coarse c^3 blocks with the central (c/2)^3 refined: about 2 c^3 blocks
        c = mesh.nroot[0]
        assert mesh.nroot == (c, c, c) and c % 2 == 0 and mesh.level.max() == 1
        assert (mesh.is_leaf() == 0).sum() == (c // 2) ** 3
        assert mesh.nb == c ** 3 + 8 * (c // 2) ** 3
        assert 0.25 * nblocks <= mesh.nb <= 4 * nblocks
    else:
        assert mesh.nb == nblocks and mesh.level.max() == 0
    assert W.shape[0] == mesh.nb and np.all(np.isfinite(W))
    assert np.all(mesh.interior(W)[:, 0] > 0) and np.all(mesh.interior(W)[:, 4] > 0)
    assert sv.state_bytes(mesh, fx.FX_F64) == 2 * mesh.nb * mesh.nvar * mesh.PZ * mesh.P ** 2 * 8
    assert sv.state_bytes(mesh, fx.FX_F32BULK) * 2 == sv.state_bytes(mesh, fx.FX_F64)
