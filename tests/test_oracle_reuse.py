"""Pins of the oracle's reuse-distance analyser and reversed-BFS ordering.

Paper: Aupy, Park & Raghavan, "Locality-Aware Laplacian Mesh Smoothing".
  Section 2.2 / Fig. 1 - reuse distance: distinct elements accessed between two
                         consecutive accesses to one element
  Fig. 3               - the access pattern of one smoothing step: the vertex,
                         then its neighbours
  Table 2              - quantiles of the reuse distances of the first sweep
  Section 2            - reversed breadth-first order (Munson and Hovland)

The checks are a hand-derived trace, Mattson's stack property (a fully
associative LRU cache of C elements misses exactly on the first accesses and on
the reuses whose distinct-element distance is at least C), telescoping sums,
numpy's inverted-CDF quantile, and BFS level structure.
"""
from collections import OrderedDict

import numpy as np
import pytest

import meshgen
import oracle


def path5():
    """Path 0-1-2-3-4, ends fixed."""
    rp = np.array([0, 1, 3, 5, 7, 8], np.int32)
    ci = np.array([1, 0, 2, 1, 3, 2, 4, 3], np.int32)
    bnd = np.array([1, 0, 0, 0, 1], np.uint8)
    return rp, ci, bnd


def test_hand_derived_path_trace():
    rp, ci, bnd = path5()
    # interior 1, 2, 3 in order; each vertex, then its row
    t = oracle.access_trace(rp, ci, bnd, np.arange(5), with_vertex=True)
    assert t.tolist() == [1, 0, 2, 2, 1, 3, 3, 2, 4]
    # reuses: 2 at t=3 (previous t=2, nothing between), 1 at t=4 (between: 0 2 2), 3 at t=6
    # (nothing between), 2 at t=7 (between: 1 3 3)
    assert oracle.reuse_distances(t, 5, oracle.DISTINCT).tolist() == [0, 2, 0, 2]
    assert oracle.reuse_distances(t, 5, oracle.ACCESSES).tolist() == [0, 3, 0, 3]
    t = oracle.access_trace(rp, ci, bnd, np.arange(5), with_vertex=False)
    assert t.tolist() == [0, 2, 1, 3, 2, 4]
    assert oracle.reuse_distances(t, 5, oracle.DISTINCT).tolist() == [2]
    # visiting order 3, 2, 1 (boundary vertices in the sequence are skipped)
    t = oracle.access_trace(rp, ci, bnd, np.array([4, 3, 2, 1, 0]), with_vertex=False)
    assert t.tolist() == [2, 4, 1, 3, 0, 2]
    assert oracle.reuse_distances(t, 5, oracle.DISTINCT).tolist() == [4]


def lru_misses(trace, capacity):
    cache = OrderedDict()
    misses = 0
    for x in trace.tolist():
        if x in cache:
            cache.move_to_end(x)
            continue
        misses += 1
        cache[x] = None
        if len(cache) > capacity:
            cache.popitem(last=False)
    return misses


@pytest.mark.parametrize("ordering", [oracle.ORI, oracle.RANDOM, oracle.BFS, oracle.RDR])
def test_distinct_distance_predicts_lru_misses(ordering):
    m = meshgen.workload(1, side=24)
    p = oracle.order(m, ordering, seed=7)
    t = oracle.access_trace(m["row_ptr"], m["col_idx"], m["is_boundary"], p)
    d = oracle.reuse_distances(t, m["n"], oracle.DISTINCT)
    cold = len(np.unique(t))
    assert cold + len(d) == len(t)
    for cap in (1, 2, 7, 16, 64, 300):
        assert lru_misses(t, cap) == cold + int((d >= cap).sum())


def test_access_distance_telescopes():
    m = meshgen.workload(1, side=20)
    for ordering in (oracle.ORI, oracle.RANDOM):
        p = oracle.order(m, ordering, seed=3)
        t = oracle.access_trace(m["row_ptr"], m["col_idx"], m["is_boundary"], p)
        d_acc = oracle.reuse_distances(t, m["n"], oracle.ACCESSES)
        d_dis = oracle.reuse_distances(t, m["n"], oracle.DISTINCT)
        # sum over reuses of (gap + 1) = sum over elements of (last time - first time)
        first, last = {}, {}
        for i, x in enumerate(t.tolist()):
            first.setdefault(x, i)
            last[x] = i
        assert int((d_acc + 1).sum()) == sum(last[x] - first[x] for x in first)
        assert (d_dis <= d_acc).all() and (d_dis <= m["n"] - 1).all()


def test_trace_length_closed_form():
    m = meshgen.workload(1, side=30)
    deg = np.diff(m["row_ptr"])
    inner = m["is_boundary"] == 0
    p = oracle.order(m, oracle.BFS)
    assert len(oracle.access_trace(m["row_ptr"], m["col_idx"], m["is_boundary"], p)) == int((deg[inner] + 1).sum())
    assert len(oracle.access_trace(m["row_ptr"], m["col_idx"], m["is_boundary"], p, False)) == int(deg[inner].sum())


def test_quantile_definition():
    v = np.array([5, 1, 3, 2, 4])
    assert [oracle.quantile(v, x) for x in (0.0, 0.2, 0.5, 0.9, 1.0)] == [1, 1, 3, 5, 5]
    rng = np.random.default_rng(11)
    for m in (1, 2, 7, 100, 1001):
        v = rng.integers(0, 50, size=m)
        for x in (0.01, 0.25, 0.5, 0.75, 0.9, 0.99, 1.0):
            assert oracle.quantile(v, x) == int(np.quantile(v, x, method="inverted_cdf"))


def test_orderings_shrink_reuse_distance_like_table_2():
    # Table 2's pattern on a synthetic mesh: a random order has by far the largest distances, and
    # RDR has the smallest 75% quantile (most reuses come within a few accesses)
    m = meshgen.workload(1, side=48)
    q = {}
    for o in (oracle.ORI, oracle.RANDOM, oracle.BFS, oracle.RDR):
        t = oracle.access_trace(m["row_ptr"], m["col_idx"], m["is_boundary"], oracle.order(m, o, seed=5))
        d = oracle.reuse_distances(t, m["n"], oracle.DISTINCT)
        q[o] = [oracle.quantile(d, x) for x in (0.5, 0.75, 0.9)]
    others = [q[o] for o in (oracle.ORI, oracle.BFS, oracle.RDR)]
    assert q[oracle.RANDOM][0] > 10 * max(x[0] for x in others)
    assert q[oracle.RANDOM][2] > max(x[2] for x in others)
    assert q[oracle.RDR][1] < min(q[oracle.ORI][1], q[oracle.BFS][1])


def test_reversed_bfs():
    m = meshgen.workload(1, side=25)
    p = oracle.order(m, oracle.RBFS)
    assert sorted(p.tolist()) == list(range(m["n"]))
    # BFS levels from vertex 0 (plain level-synchronous search): non-increasing along the order,
    # vertex 0 last
    level = np.full(m["n"], -1)
    level[0] = 0
    frontier = [0]
    while frontier:
        nxt = []
        for v in frontier:
            for u in m["col_idx"][m["row_ptr"][v]:m["row_ptr"][v + 1]]:
                if level[u] < 0:
                    level[u] = level[v] + 1
                    nxt.append(u)
        frontier = nxt
    assert (np.diff(level[p]) <= 0).all() and p[-1] == 0


def test_plausible_mistakes_fail_the_reuse_pins():
    # an analyser that counted accesses instead of distinct elements, or that forgot to skip
    # boundary vertices, would fail the LRU and closed-form pins: check on mutated data
    m = meshgen.workload(1, side=16)
    t = oracle.access_trace(m["row_ptr"], m["col_idx"], m["is_boundary"], oracle.order(m, oracle.ORI))
    d_acc = oracle.reuse_distances(t, m["n"], oracle.ACCESSES)
    cold = len(np.unique(t))
    assert any(lru_misses(t, c) != cold + int((d_acc >= c).sum()) for c in (2, 7, 16, 64))
    all_b = np.zeros_like(m["is_boundary"])
    t2 = oracle.access_trace(m["row_ptr"], m["col_idx"], all_b, np.arange(m["n"]))
    deg = np.diff(m["row_ptr"])
    assert len(t2) != int((deg[m["is_boundary"] == 0] + 1).sum())
