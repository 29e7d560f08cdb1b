"""The benchmark's multi-rank path on CPU (gloo, world size 2): every rank
gets its own meshes (weak scaling, no data exchange) and the timings are
max-reduced, the unit counts summed."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    d = bench.Dist(backend="gloo")
    try:
        seeds = bench.rank_mesh_seeds(8, d.rank)
        t_max = d.max(1.0 + rank)
        units = d.sum(100 * (rank + 1))
        d.barrier()
        out[rank] = (seeds, t_max, units)
    finally:
        d.close()


def test_two_rank_gloo_sharding_and_reductions():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    s0, s1 = set(res[0][0]), set(res[1][0])
    assert len(s0) == 8 and len(s1) == 8 and not (s0 & s1)
    assert res[0][1] == res[1][1] == 2.0
    assert res[0][2] == res[1][2] == 300.0
