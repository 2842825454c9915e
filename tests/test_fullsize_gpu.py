"""GPU parity on the benchmark configurations themselves, at full size.

The 3D Kelvin-Helmholtz shear layer (256^3 as 4096 blocks of 16^3, periodic)
and the 3D Sedov blast on its two-level octree (8^3 coarse blocks of 16^3, 128
of them refined into 1024 fine blocks; 1408 leaves) are each advanced 100
steps by the CUDA path -- the same fx_step sequence, launch configuration and
block size the benchmark times -- and by the FP64 CPU oracle from the same
seeded primitive state.  Every leaf cell (and every parent of the AMR mesh) is
compared with the stated tolerance for 100 steps, 1e-10 relative
(|a - b| / max(|b|, max|b_var|)); the time reached (the sum of the 100 dt)
must agree to 1e-12.

The oracle needs about two minutes on 16 host cores for both.
"""
import numpy as np
import pytest

from paper_2208_11630_gb300 import inputs
from tests.helpers import max_rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.fullsize]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_11630_gb300 import fx as _fx
    _fx.load()
    return _fx


def _run_both(orc, fx, name, nsteps):
    mesh, W, gamma, cfl = inputs.workload(name)
    om = orc.OracleMesh(mesh, gamma)
    U = om.prim_to_cons(W)
    bs = fx.BlockSet(mesh, gamma)
    bs.set_conserved(U)
    del W
    t_gpu = 0.0
    for _ in range(nsteps):
        bs.step(cfl)
        t_gpu += float(bs.dt.item())
    assert bs.status() == 0
    G = bs.state()
    bs.close()
    torch.cuda.empty_cache()
    Uo, t, n = om.run(U, nsteps=nsteps, cfl=cfl)
    del U
    assert n == nsteps
    return mesh, G, Uo, t_gpu, t


@pytest.mark.parametrize("name", ["kh3d", "sedov_amr"])
def test_full_size_100_steps(orc, fx, name):
    mesh, G, Uo, t_gpu, t = _run_both(orc, fx, name, 100)
    assert t_gpu == pytest.approx(t, rel=1e-12)
    err = max_rel_err(mesh, G, Uo)
    assert err <= 1e-10, err
    par = ~mesh.is_leaf().astype(bool)
    if par.any():   # restricted parents follow their children
        a, b = mesh.interior(G)[par], mesh.interior(Uo)[par]
        s = np.maximum(np.abs(b).max(axis=(0, 2, 3, 4), keepdims=True), 1e-300)
        assert (np.abs(a - b) / np.maximum(np.abs(b), s)).max() <= 1e-10
