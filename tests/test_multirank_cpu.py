"""Multi-rank bookkeeping of the benchmark on CPU (gloo, world size 2).

On GPUs every rank advances an independent replica (replicas of independent
block sets; no data-path collective).  What crosses ranks is only the
reduction of the measurement: zones are summed, the time is the slowest
rank's.  This is checked here with two CPU ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    zones = 1000.0 * (rank + 1)
    secs = 0.5 + rank
    z, t = bench.aggregate(zones, secs)
    out[rank] = (z, t, bench.dist_env())
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_ranks():
    ws = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()   # no fork of a multi-threaded process
    out = mgr.dict()
    mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
    for r in range(ws):
        z, t, env = out[r]
        assert z == 3000.0          # zones summed over ranks
        assert t == 1.5             # slowest rank's time
        assert env == (ws, r, r)
