"""The sharding plan (paper_2208_11630_gb300/shard.py) on CPU ranks.

Plan checks: balanced Z-order partitions, symmetric touch adjacency with
periodic wrap, halos disjoint from what a rank owns, exchange lists that
send only owned blocks into the receiver's halo.

Sharded steps (gloo, world size 2): each rank keeps only the blocks it owns
and poisons every other block with a quiet state, receives its halo from
the owners, takes the global dt by a MIN reduction of its own CFL limit,
and steps its array with the FP64 oracle.  After several steps, the leaves
it owns must equal, bit for bit, those of an unsharded run, on uniform,
two-level and three-level meshes, periodic and outflow -- with the plan's
default halo of three rings and with one ring alike; with no halo the
result differs (the poisoning is effective).
"""
import os
import socket

import numpy as np
import pytest

from paper_2208_11630_gb300 import inputs, shard

torch = pytest.importorskip("torch")

O_, P_ = inputs.OUTFLOW, inputs.PERIODIC


def _amr(ndim, nblk, bc, seed):
    base = inputs.uniform_mesh(ndim, (nblk,) * ndim, 8, 4, bc)
    lo, hi = nblk // 4, nblk // 4 + nblk // 2
    flags = [all(lo <= base.origin[b, d] // 8 < hi for d in range(ndim)) for b in range(base.nb)]
    mesh = inputs.refine(base, np.array(flags))
    return mesh, inputs.random_smooth_state(mesh, seed)


def _three_levels():
    """2D, 8 x 8 level-0 blocks, outflow: the central 4 x 4 refined, and the
    central 4 x 4 of the resulting 8 x 8 level-1 blocks refined again."""
    base = inputs.uniform_mesh(2, (8, 8), 8, 4, O_)
    f1 = [all(2 <= base.origin[b, d] // 8 < 6 for d in range(2)) for b in range(base.nb)]
    m1 = inputs.refine(base, np.array(f1))
    f2 = [int(m1.level[b]) == 1 and all(6 <= m1.origin[b, d] // 8 < 10 for d in range(2))
          for b in range(m1.nb)]
    mesh = inputs.refine(m1, np.array(f2))
    return mesh, inputs.random_smooth_state(mesh, 8)


CASES = {
    "uniform3d_periodic": lambda: (lambda m: (m, inputs.kh_state(m)))(
        inputs.uniform_mesh(3, (4, 4, 4), 8, 4, P_)),
    "amr3d_periodic": lambda: _amr(3, 4, P_, 3),
    "amr2d_outflow": lambda: _amr(2, 8, O_, 5),
    "amr2d_three_levels": _three_levels,
}


def test_partition_is_balanced_and_follows_the_curve():
    mesh, _ = CASES["amr3d_periodic"]()
    leaf = np.flatnonzero(mesh.is_leaf() == 1)
    keys = shard.morton_keys(mesh)
    assert len(np.unique(keys[leaf])) == len(leaf)
    for n in (1, 2, 3, 5):
        owner = shard.partition(mesh, n)
        assert np.all(owner[mesh.is_leaf() == 0] == -1)
        counts = np.bincount(owner[leaf], minlength=n)
        assert counts.sum() == len(leaf) and counts.max() - counts.min() <= 1
        # each rank owns one contiguous run of the curve
        order = leaf[np.argsort(keys[leaf])]
        assert np.all(np.diff(owner[order]) >= 0)


@pytest.mark.parametrize("ndim,bc,expect", [(3, P_, 26), (2, P_, 8), (3, O_, None)])
def test_adjacency_on_uniform_meshes(ndim, bc, expect):
    mesh = inputs.uniform_mesh(ndim, (4,) * ndim, 8, 4, bc)
    adj = shard.leaf_adjacency(mesh)
    for b in range(mesh.nb):
        for c in adj[b]:
            assert b in adj[c]
        idx = mesh.origin[b, :ndim] // 8
        if expect is not None:
            assert len(adj[b]) == expect
        else:   # outflow: 3^k - 1 neighbours with k axes away from both walls
            inner = sum(1 for d in range(ndim) if 0 < idx[d] < 3)
            assert len(adj[b]) == 3 ** inner * 2 ** (ndim - inner) - 1


def test_adjacency_across_levels():
    mesh, _ = CASES["amr2d_outflow"]()
    adj = shard.leaf_adjacency(mesh)
    lo, side = shard.finest_corners(mesh)
    leaf = np.flatnonzero(mesh.is_leaf() == 1)
    # brute force: closed boxes on the finest block lattice intersect
    for b in leaf:
        want = []
        for c in leaf:
            if c == b:
                continue
            if all(lo[b, d] <= lo[c, d] + side[c] and lo[c, d] <= lo[b, d] + side[b]
                   for d in range(2)):
                want.append(c)
        assert adj[b].tolist() == sorted(want)
        assert np.all(np.abs(mesh.level[adj[b]] - mesh.level[b]) <= 1)


def test_halo_and_exchange_lists():
    mesh, _ = CASES["amr3d_periodic"]()
    owner = shard.partition(mesh, 3)
    lists = shard.exchange_lists(mesh, owner, 3)
    for r in range(3):
        h1, h3 = shard.halo(mesh, owner, r, 1), shard.halo(mesh, owner, r, 3)
        assert not np.any(owner[h3] == r) and np.all(owner[h3] >= 0)
        assert set(h1) <= set(h3)
        got = np.sort(np.concatenate([lists.get((s, r), np.zeros(0, np.int64))
                                      for s in range(3) if s != r]))
        assert np.array_equal(got, h3)
    for (s, d), blocks in lists.items():
        assert np.all(owner[blocks] == s)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _exchange(dist, U, lists, rank, ws):
    reqs, inbox = [], []
    for peer in range(ws):
        if peer == rank:
            continue
        out = lists.get((rank, peer))
        if out is not None:
            reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(U[out])), dst=peer))
        into = lists.get((peer, rank))
        if into is not None:
            buf = torch.empty((len(into),) + U.shape[1:], dtype=torch.float64)
            reqs.append(dist.irecv(buf, src=peer))
            inbox.append((into, buf))
    for q in reqs:
        q.wait()
    for into, buf in inbox:
        U[into] = buf.numpy()


def _worker(rank, ws, port, case, rings, steps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import oracle
        oracle.set_threads(2)
        mesh, W = CASES[case]()
        om = oracle.OracleMesh(mesh)
        U0 = om.prim_to_cons(W)
        owner = shard.partition(mesh, ws)
        lists = shard.exchange_lists(mesh, owner, ws, rings)
        mine = owner == rank
        # a quiet state (at rest, pressure 1e-30): physical, with a negligible
        # signal speed, and different from every block of the real state
        Wq = np.zeros((1,) + W.shape[1:])
        Wq[:, 0] = 1.0
        Wq[:, 4] = 1e-30
        poison = om.prim_to_cons(np.broadcast_to(Wq, W.shape).copy())[0]
        U, Uref = U0.copy(), U0.copy()
        same_dt = True
        for _ in range(steps):
            U[~mine] = poison
            _exchange(dist, U, lists, rank, ws)
            t = torch.tensor([om.compute_dt(U)], dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MIN)
            dt = float(t.item())
            Ug = U.copy()
            om.guardcell_fill(Ug)
            U, _, _ = om.hydro_advance(Ug, dt)   # status of poisoned blocks ignored
            Uref, dref = om.step(Uref)
            same_dt = same_dt and dt == dref
        a, b = mesh.interior(U)[mine], mesh.interior(Uref)[mine]
        out[rank] = (bool(np.array_equal(a, b)), float(np.max(np.abs(a - b))), same_dt,
                     int(mine.sum()))
    finally:
        dist.destroy_process_group()


def _run(case, rings, steps=3, ws=2):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, ws, port, case, rings, steps, out))
                 for r in range(ws)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        return [out[r] for r in range(ws)]


@pytest.mark.parametrize("rings", [3, 1])
@pytest.mark.parametrize("case", sorted(CASES))
def test_sharded_steps_equal_the_unsharded_run(case, rings):
    res = _run(case, rings=rings)
    for equal, diff, same_dt, nown in res:
        assert nown > 0 and same_dt
        assert equal, diff


def test_without_a_halo_the_result_differs():
    """The poisoning is real: with no halo received, the owned leaves next
    to the other rank's region come out different."""
    res = _run("amr3d_periodic", rings=0)
    assert not any(r[0] for r in res)


@pytest.mark.parametrize("case", ["amr3d_periodic", "amr2d_outflow", "amr2d_three_levels"])
def test_one_step_reads_only_touching_leaves(orc, case):
    """Brute-force dependency check with the oracle: perturb one block at a
    time, take one step at a fixed dt, and record which leaves change.  Every
    leaf a perturbation reaches is the perturbed leaf or touches it -- one
    touch-step, so one ring of halo suffices on these meshes -- and a parent
    reaches nothing (the step restricts it from its children first)."""
    mesh, W = CASES[case]()
    om = orc.OracleMesh(mesh)
    U0 = om.prim_to_cons(W)
    dt = om.compute_dt(U0)
    I0 = mesh.interior(om.step(U0, dt=dt)[0]).reshape(mesh.nb, -1)
    adj = shard.leaf_adjacency(mesh)
    leaf = mesh.is_leaf() == 1
    reach = 0
    for b in range(mesh.nb):
        U = U0.copy()
        I = mesh.interior(U)
        I[b, 0] *= 1.001
        I[b, 4] *= 1.001
        changed = np.flatnonzero(np.any(
            mesh.interior(om.step(U, dt=dt)[0]).reshape(mesh.nb, -1) != I0, axis=1))
        changed = changed[leaf[changed]]
        if not leaf[b]:
            assert len(changed) == 0, (b, changed)
            continue
        assert b in changed
        outside = [int(c) for c in changed if c != b and c not in set(adj[b].tolist())]
        assert not outside, (b, outside)
        reach = max(reach, len(changed))
    assert reach > 1   # perturbations do cross block boundaries
