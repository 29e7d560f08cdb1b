"""Pins of the oracle's block RDR ordering (a data-parallel variant of Algorithm 2, not in the paper).

Block RDR cuts the BFS order into blocks of consecutive positions and applies Algorithm 2 to each
block's own subgraph.  Its two limits reduce to pinned orderings - one block is Algorithm 2, blocks
of one vertex are the BFS order - and a hand-derived trace on a path checks the in-block walk.
"""
import numpy as np
import pytest

import meshgen
import oracle


def path6():
    # path 0-1-2-3-4-5, ends fixed
    rp = np.array([0, 1, 3, 5, 7, 9, 10], np.int32)
    ci = np.array([1, 0, 2, 1, 3, 2, 4, 3, 5, 4], np.int32)
    bnd = np.array([1, 0, 0, 0, 0, 1], np.uint8)
    q = np.array([0.9, 0.5, 0.3, 0.2, 0.8, 0.9])
    return rp, ci, bnd, q


def test_hand_derived_path():
    rp, ci, bnd, q = path6()
    # Algorithm 2: seeds 3, 2, 1, 4; walk 3 -> l = [2, 4] -> from 2: l = [1] -> from 1: l = [0]; seed 4:
    # l = [5]
    assert oracle.order_rdr(rp, ci, bnd, q).tolist() == [3, 2, 4, 1, 0, 5]
    # blocks of 3 BFS positions: {0, 1, 2} with seeds 2, 1 (walk 2 -> 1 -> 0; 3 lies outside), then
    # {3, 4, 5} with seeds 3, 4 (walk 3 -> 4 -> 5)
    assert oracle.order_brdr(rp, ci, bnd, q, block=3).tolist() == [2, 1, 0, 3, 4, 5]
    # blocks of 4: {0, 1, 2, 3} (seeds 3, 2, 1: walk 3 -> 2 -> 1 -> 0), then {4, 5} (seed 4: 4 -> 5)
    assert oracle.order_brdr(rp, ci, bnd, q, block=4).tolist() == [3, 2, 1, 0, 4, 5]


@pytest.mark.parametrize("side", [9, 23, 40])
def test_limits_are_rdr_and_bfs(side):
    m = meshgen.workload(1, side=side)
    q = oracle.vertex_quality(m["n"], m["tri"], m["xy"])
    args = (m["row_ptr"], m["col_idx"], m["is_boundary"], q)
    assert np.array_equal(oracle.order_brdr(*args, block=m["n"]), oracle.order_rdr(*args))
    assert np.array_equal(oracle.order_brdr(*args, block=10 * m["n"]), oracle.order_rdr(*args))
    assert np.array_equal(oracle.order_brdr(*args, block=1), oracle.order_bfs(m["row_ptr"], m["col_idx"]))


@pytest.mark.parametrize("block", [7, 64, 500])
def test_blocks_keep_the_bfs_vertex_sets(block):
    m = meshgen.workload(1, side=30)
    q = oracle.vertex_quality(m["n"], m["tri"], m["xy"])
    p = oracle.order_brdr(m["row_ptr"], m["col_idx"], m["is_boundary"], q, block=block)
    bfs = oracle.order_bfs(m["row_ptr"], m["col_idx"])
    assert sorted(p.tolist()) == list(range(m["n"]))
    for s in range(0, m["n"], block):
        members = bfs[s:s + block]
        assert set(p[s:s + block].tolist()) == set(members.tolist())
        inner = [v for v in members.tolist() if not m["is_boundary"][v]]
        if inner:  # every block starts with its worst interior vertex (ties by id)
            assert p[s] == min(inner, key=lambda v: (q[v], v))


def test_block_rdr_shortens_reuse_like_bfs_and_rdr():
    m = meshgen.workload(1, side=64)
    q = oracle.vertex_quality(m["n"], m["tri"], m["xy"])
    res = {}
    for name, p in (("bfs", oracle.order_bfs(m["row_ptr"], m["col_idx"])),
                    ("rdr", oracle.order_rdr(m["row_ptr"], m["col_idx"], m["is_boundary"], q)),
                    ("brdr", oracle.order_brdr(m["row_ptr"], m["col_idx"], m["is_boundary"], q, block=512))):
        t = oracle.access_trace(m["row_ptr"], m["col_idx"], m["is_boundary"], p)
        d = oracle.reuse_distances(t, m["n"], oracle.DISTINCT)
        res[name] = (oracle.quantile(d, 0.75), oracle.quantile(d, 1.0))
    assert res["brdr"][0] < res["bfs"][0]       # RDR's short reuse inside blocks
    assert res["brdr"][1] < res["rdr"][1]       # no reuse spans the mesh
