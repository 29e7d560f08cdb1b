"""The identity the device BFS ordering is built on, checked on the CPU.

A sequential breadth-first search (from vertex 0, neighbours appended in
ascending id, restart at the smallest unvisited id) appends level L+1 in the
order of (queue position of the first level-L vertex adjacent to it, vertex
id).  This file restates the search in that level-synchronous form, written
with numpy, and compares it with the oracle's sequential search on meshes
with several components, shuffled rows and high-degree vertices.
"""
import numpy as np
import pytest

import meshgen
import oracle


def level_synchronous_bfs(row_ptr, col_idx):
    n = len(row_ptr) - 1
    pos = np.full(n, -1, np.int64)
    out = []
    while len(out) < n:
        root = int(np.flatnonzero(pos < 0)[0])
        pos[root] = len(out)
        out.append(root)
        fa, fb = len(out) - 1, len(out)
        while fa < fb:
            parent = {}
            for i in range(fa, fb):
                w = out[i]
                for u in col_idx[row_ptr[w]:row_ptr[w + 1]].tolist():
                    if pos[u] < 0:
                        parent[u] = min(parent.get(u, i), i)
            for u in sorted(parent, key=lambda u: (parent[u], u)):
                pos[u] = len(out)
                out.append(u)
            fa, fb = fb, len(out)
    return np.array(out, np.int32)


def disjoint_union(*meshes):
    rps, cis, off, eoff = [], [], 0, 0
    for m in meshes:
        rps.append(m["row_ptr"][(1 if rps else 0):] + eoff)
        cis.append(m["col_idx"] + off)
        off += m["n"]
        eoff += m["row_ptr"][-1]
    return np.concatenate(rps).astype(np.int32), np.concatenate(cis).astype(np.int32)


def shuffled_rows(row_ptr, col_idx, seed):
    rng = np.random.default_rng(seed)
    ci = col_idx.copy()
    for v in range(len(row_ptr) - 1):
        rng.shuffle(ci[row_ptr[v]:row_ptr[v + 1]])
    return ci


def star_with_hubs(n_leaves, hubs):
    # hub h is joined to every leaf with index = h mod hubs (degree ~ n_leaves / hubs); leaves form a path
    n = hubs + n_leaves
    adj = [set() for _ in range(n)]
    for k in range(n_leaves):
        v = hubs + k
        adj[v].add(k % hubs)
        adj[k % hubs].add(v)
        if k:
            adj[v].add(v - 1)
            adj[v - 1].add(v)
    rp = np.zeros(n + 1, np.int32)
    ci = []
    for v in range(n):
        ci += sorted(adj[v])
        rp[v + 1] = len(ci)
    return rp, np.array(ci, np.int32)


@pytest.mark.parametrize("side", [5, 16, 33])
def test_level_synchronous_form_equals_sequential_bfs(side):
    m = meshgen.workload(1, side=side)
    want = oracle.order_bfs(m["row_ptr"], m["col_idx"])
    assert np.array_equal(level_synchronous_bfs(m["row_ptr"], m["col_idx"]), want)
    ci = shuffled_rows(m["row_ptr"], m["col_idx"], side)
    assert np.array_equal(level_synchronous_bfs(m["row_ptr"], ci), oracle.order_bfs(m["row_ptr"], ci))


def test_level_synchronous_form_on_components_and_hubs():
    rp, ci = disjoint_union(meshgen.workload(1, side=9), meshgen.workload(0, side=6), meshgen.workload(1, side=4))
    assert np.array_equal(level_synchronous_bfs(rp, ci), oracle.order_bfs(rp, ci))
    rp, ci = star_with_hubs(200, 3)
    assert np.array_equal(level_synchronous_bfs(rp, ci), oracle.order_bfs(rp, ci))
