"""Device breadth-first orderings (k_bfs) against the oracle's sequential search.

lms_reorder(LMS_BFS / LMS_RBFS) and lms_batch_create with a breadth-first
ordering run the level-synchronous search on the device; the permutation must
equal the oracle's BFS (reversed for RBFS) position for position, on graphs
with several components, rows in any order, rows longer than the register
fast path, single-CTA searches (small meshes) and cluster searches (large
ones).
"""
import numpy as np
import pytest

import meshgen
import oracle
import paper_1606_00803_gb300 as lms
from test_bfs_levels import disjoint_union, shuffled_rows, star_with_hubs

pytestmark = pytest.mark.gpu


def csr_mesh(rp, ci, seed=0):
    n = len(rp) - 1
    rng = np.random.default_rng(seed)
    bnd = np.zeros(n, np.uint8)
    bnd[:: 7] = 1
    return dict(n=n, row_ptr=rp, col_idx=ci, xy=rng.random((n, 2)), is_boundary=bnd)


def device_order(m, ordering):
    with lms.Mesh.from_dict(m, lms.FP32) as g:
        g.reorder(ordering)
        return g.permutation()


@pytest.mark.parametrize("ordering", [lms.BFS, lms.RBFS])
def test_device_bfs_on_components_with_shuffled_rows(ordering):
    rp, ci = disjoint_union(meshgen.workload(1, side=30), meshgen.workload(0, side=9), meshgen.workload(1, side=3))
    ci = shuffled_rows(rp, ci, 4)
    want = oracle.order_bfs(rp, ci)
    got = device_order(csr_mesh(rp, ci), ordering)
    assert np.array_equal(got, want if ordering == lms.BFS else want[::-1])


def test_device_bfs_rows_longer_than_fast_path():
    rp, ci = star_with_hubs(3000, 5)  # hubs of degree 600
    assert np.diff(rp).max() > 16
    assert np.array_equal(device_order(csr_mesh(rp, ci), lms.BFS), oracle.order_bfs(rp, ci))


def test_device_bfs_cluster_search_on_large_mesh():
    # more than 65,536 vertices: the search runs on a cluster of CTAs
    m = meshgen.workload(1, side=400)
    ci = shuffled_rows(m["row_ptr"], m["col_idx"], 8)
    m2 = dict(m, col_idx=ci)
    assert np.array_equal(device_order(m2, lms.BFS), oracle.order_bfs(m["row_ptr"], ci))
    rp, cc = disjoint_union(meshgen.workload(1, side=300), meshgen.workload(1, side=200))
    assert np.array_equal(device_order(csr_mesh(rp, cc), lms.RBFS), oracle.order_bfs(rp, cc)[::-1])


def test_device_bfs_batch_of_many_meshes():
    meshes = [meshgen.generate(s, jitter=0.3, flip_frac=0.1, split_frac=0.05, seed=500 + s)
              for s in (3, 4, 9, 17, 40, 64, 100, 5, 200)]
    with lms.Batch(meshes, ordering=lms.BFS) as b:
        for i, m in enumerate(meshes):
            assert np.array_equal(b.permutation(i), oracle.order_bfs(m["row_ptr"], m["col_idx"]))


def test_reorder_times_are_reported():
    m = meshgen.workload(1, side=50)
    with lms.Mesh.from_dict(m, lms.FP64) as g:
        assert all(np.isnan(t) for t in g.last_reorder_ms())
        for o in (lms.BFS, lms.RDR, lms.RANDOM, lms.ORI, lms.RBFS):
            g.reorder(o)
            order_ms, layout_ms = g.last_reorder_ms()
            assert 0.0 <= order_ms < 60e3 and 0.0 <= layout_ms < 60e3


def brdr_want(m, rp=None, ci=None):
    rp = m["row_ptr"] if rp is None else rp
    ci = m["col_idx"] if ci is None else ci
    q = oracle.vertex_quality(m["n"], m["tri"], m["xy"])
    return oracle.order_brdr(rp, ci, m["is_boundary"], q, block=lms.BRDR_BLOCK)


@pytest.mark.parametrize("side", [5, 60, 100, 400])
def test_device_block_rdr_single_mesh(side):
    m = meshgen.workload(1, side=side)
    with lms.Mesh.from_dict(m, lms.FP64) as g:
        g.reorder(lms.BRDR)
        assert np.array_equal(g.permutation(), brdr_want(m))


def test_device_block_rdr_shuffled_rows_and_components():
    a, b = meshgen.workload(1, side=90), meshgen.workload(0, side=40)
    rp, ci = disjoint_union(a, b)
    ci = shuffled_rows(rp, ci, 3)
    m = dict(n=a["n"] + b["n"], row_ptr=rp, col_idx=ci, is_boundary=np.concatenate([a["is_boundary"], b["is_boundary"]]),
             tri=np.concatenate([a["tri"], b["tri"] + a["n"]]), xy=np.concatenate([a["xy"], b["xy"] + 2.0]))
    with lms.Mesh.from_dict(m, lms.FP32) as g:
        g.reorder(lms.BRDR)
        assert np.array_equal(g.permutation(), brdr_want(m))


def test_device_block_rdr_batch():
    meshes = [meshgen.generate(s, jitter=0.3, flip_frac=0.1, split_frac=0.05, seed=900 + s)
              for s in (3, 7, 30, 64, 120, 200)]
    with lms.Batch(meshes, ordering=lms.BRDR) as b:
        for i, m in enumerate(meshes):
            assert np.array_equal(b.permutation(i), brdr_want(m))
