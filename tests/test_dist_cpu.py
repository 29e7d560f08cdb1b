"""The benchmark's multi-rank path on CPU (gloo, world size 2): one batch split
between the ranks by whole meshes, balanced by vertex count
(lms_partition_meshes); no data exchange during the sweeps; timings
max-reduced, unit counts summed.  Each rank smooths its share (here with the
oracle on the CPU, standing in for the GPU path) and the per-mesh results are
gathered and checked against the one-rank run."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

COUNT, LO, HI, SWEEPS = 14, 10, 40, 6


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
    import oracle
    d = bench.Dist(backend="gloo")
    try:
        meshes, mine, load = bench.rank_batch(COUNT, d.rank, d.world, lo=LO, hi=HI)
        res = [oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], SWEEPS)[0] for m in meshes]
        gathered = [None] * world
        d.pg.all_gather_object(gathered, (mine, res))
        t_max = d.max(1.0 + rank)
        units = d.sum(100 * (rank + 1))
        d.barrier()
        out[rank] = (mine, load, gathered, t_max, units)
    finally:
        d.close()


def test_two_rank_gloo_batch_split_and_reductions():
    import bench
    import oracle
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    meshes = bench.batch_meshes(COUNT, LO, HI)
    sizes = [m["n"] for m in meshes]
    mine0, mine1 = res[0][0], res[1][0]
    assert sorted(mine0 + mine1) == list(range(COUNT))  # every mesh on exactly one rank
    load = res[0][1]
    assert load == res[1][1] and sum(load) == sum(sizes)
    assert load == [sum(sizes[i] for i in mine0), sum(sizes[i] for i in mine1)]
    assert max(load) - min(load) <= max(sizes)
    # per-mesh results gathered from both ranks equal the one-rank run
    got = {}
    for idx, xs in res[0][2]:
        for i, x in zip(idx, xs):
            got[i] = x
    assert sorted(got) == list(range(COUNT))
    for i, m in enumerate(meshes):
        want, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], SWEEPS)
        assert np.array_equal(got[i], want)
    assert res[0][3] == res[1][3] == 2.0
    assert res[0][4] == res[1][4] == 300.0
