"""Pins of the oracle's block order for the in-place sweep (or_block_sequence): tiles of consecutive
storage positions, first-fit tile colours, visits by (tile colour, tile, vertex colour, position).

The order is not in the paper; it is the sequential form of a block Gauss-Seidel whose tiles of one
colour (and vertices of one colour inside a tile) run at the same time.  What pins it: a hand-derived
trace, the two limits that reduce it to the coloured Gauss-Seidel order, a proper tile colouring, and
the independence that makes the parallel form equal the sequential one."""
import numpy as np
import pytest

import meshgen
import oracle


def path(n):
    rp, ci = [0], []
    for v in range(n):
        ci += [u for u in (v - 1, v + 1) if 0 <= u < n]
        rp.append(len(ci))
    bnd = np.zeros(n, np.uint8)
    bnd[0] = bnd[n - 1] = 1
    return np.array(rp, np.int32), np.array(ci, np.int32), bnd


def test_hand_trace_on_a_path():
    # path 0..9 with fixed ends, identity storage order, tiles of 3 positions: {0,1,2} {3,4,5} {6,7,8} {9}.
    # First-fit vertex colours alternate 0,1 from vertex 1.  Interior edges 2-3 and 5-6 join tiles 0-1
    # and 1-2; tile 3 holds only a boundary vertex.  Tile colours 0,1,0,0.  Visits: colour-0 tiles in
    # order - tile 0: colour 0 [1], colour 1 [2]; tile 2: colour 0 [7], colour 1 [6, 8] - then tile 1:
    # colour 0 [3, 5], colour 1 [4].
    rp, ci, bnd = path(10)
    p = np.arange(10, dtype=np.int32)
    colour, nc = oracle.color_greedy(rp, ci, bnd, p)
    seq, tc, nt = oracle.block_sequence(rp, ci, bnd, p, colour, nc, 3)
    assert list(tc) == [0, 1, 0, 0] and nt == 2
    assert list(seq) == [1, 2, 7, 6, 8, 3, 5, 4]


@pytest.fixture(scope="module")
def mesh():
    return meshgen.workload(1, side=24)


@pytest.mark.parametrize("ordering", [oracle.ORI, oracle.BFS, oracle.RDR, oracle.RANDOM])
def test_limits_reduce_to_the_coloured_order(mesh, ordering):
    m = mesh
    p = oracle.order(m, ordering, seed=5)
    colour, nc = oracle.color_greedy(m["row_ptr"], m["col_idx"], m["is_boundary"], p)
    want = oracle.color_sequence(m["is_boundary"], p, colour, nc)
    for tile in (1, m["n"], m["n"] + 17):  # one position per tile (tile colours = vertex colours), one tile
        seq, _, _ = oracle.block_sequence(m["row_ptr"], m["col_idx"], m["is_boundary"], p, colour, nc, tile)
        assert np.array_equal(seq, want)


@pytest.mark.parametrize("tile", [2, 7, 64, 100])
def test_permutation_and_proper_tile_colouring(mesh, tile):
    m = mesh
    p = oracle.order(m, oracle.RDR)
    colour, nc = oracle.color_greedy(m["row_ptr"], m["col_idx"], m["is_boundary"], p)
    seq, tc, nt = oracle.block_sequence(m["row_ptr"], m["col_idx"], m["is_boundary"], p, colour, nc, tile)
    interior = np.nonzero(m["is_boundary"] == 0)[0]
    assert np.array_equal(np.sort(seq), interior)
    pos = np.empty(m["n"], np.int64)
    pos[p] = np.arange(m["n"])
    rp, ci, bnd = m["row_ptr"], m["col_idx"], m["is_boundary"]
    for v in interior:
        for u in ci[rp[v]:rp[v + 1]]:
            if not bnd[u] and pos[u] // tile != pos[v] // tile:
                assert tc[pos[u] // tile] != tc[pos[v] // tile]
    assert 1 <= nt <= int(tc.max()) + 1


def group_reversed(seq, p, colour, tc, tile):
    """The same visits with the tiles of each tile colour, and the vertices of each (tile, colour) group,
    taken in reverse order."""
    pos = np.empty(len(p), np.int64)
    pos[p] = np.arange(len(p))
    t = pos[seq] // tile
    keys = list(zip(tc[t], t, colour[seq]))
    out, groups = [], {}
    for v, k in zip(seq, keys):
        groups.setdefault(k, []).append(v)
    for c in sorted({k[0] for k in keys}):
        tiles = sorted({k[1] for k in keys if k[0] == c}, reverse=True)
        for ti in tiles:
            for k in sorted(k for k in groups if k[0] == c and k[1] == ti):
                out += groups[k][::-1]
    return np.array(out, np.int32)


@pytest.mark.parametrize("tile", [5, 48])
def test_order_inside_a_tile_colour_does_not_matter(mesh, tile):
    # the independence that lets tiles of one colour, and one colour's vertices in a tile, run at once
    m = mesh
    p = oracle.order(m, oracle.BFS)
    colour, nc = oracle.color_greedy(m["row_ptr"], m["col_idx"], m["is_boundary"], p)
    seq, tc, _ = oracle.block_sequence(m["row_ptr"], m["col_idx"], m["is_boundary"], p, colour, nc, tile)
    alt = group_reversed(seq, p, colour, tc, tile)
    assert not np.array_equal(alt, seq)
    a, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 4, mode=oracle.INPLACE, seq=seq)
    b, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 4, mode=oracle.INPLACE, seq=alt)
    assert np.array_equal(a, b)
    # control: with every tile given one colour the reversed order reads neighbours at other times
    flat = np.zeros_like(tc)
    alt_flat = group_reversed(seq, p, colour, flat, tile)
    c, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 4, mode=oracle.INPLACE,
                            seq=alt_flat)
    assert not np.array_equal(a, c)


def test_block_gauss_seidel_reaches_the_harmonic_limit():
    # every in-place order converges to the discrete harmonic embedding (dense Dirichlet solve)
    m = meshgen.generate(9, jitter=0.3, flip_frac=0.1, split_frac=0.05, seed=77)
    rp, ci, bnd, xy = m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"]
    n = m["n"]
    L = np.zeros((n, n))
    for v in range(n):
        for u in ci[rp[v]:rp[v + 1]]:
            L[v, u] -= 1.0
        L[v, v] = rp[v + 1] - rp[v]
    I, B = np.nonzero(bnd == 0)[0], np.nonzero(bnd == 1)[0]
    want = xy.copy()
    want[I] = np.linalg.solve(L[np.ix_(I, I)], -L[np.ix_(I, B)] @ xy[B])
    p = oracle.order(m, oracle.RDR)
    got, _, _ = oracle.block_gs_smooth(m, p, 7, 3000)
    assert np.abs(got - want).max() <= 1e-10
