"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself through a retyped formula: each
check is a closed form, a dense-matrix restatement solved by numpy, a
hand-derived trace of Algorithm 2, or an invariant of the method.

Paper: Aupy, Park & Raghavan, "Locality-Aware Laplacian Mesh Smoothing".
  Eq. 1          - the Laplacian update (mean of the neighbours)
  Algorithm 1    - in-place sweep over the interior vertices, global quality
  Section 3.2    - edge-length ratio quality, vertex and mesh means
  Section 5.1    - stopping criterion on the quality improvement
  Algorithm 2    - RDR ordering; Theorem 1 (every vertex ordered once)
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import meshgen
import oracle
from conftest import GOLDEN


def grid_mesh(s, h=None, jitter=0.0, seed=1):
    """s x s grid with every cell split along the same diagonal (i,j)-(i+1,j+1)."""
    h = 1.0 / (s - 1) if h is None else h
    xy = np.array([[i * h, j * h] for j in range(s) for i in range(s)], np.float64)
    bnd = np.array([1 if (i in (0, s - 1) or j in (0, s - 1)) else 0 for j in range(s) for i in range(s)], np.uint8)
    tri = []
    for j in range(s - 1):
        for i in range(s - 1):
            v00, v10, v01, v11 = j * s + i, j * s + i + 1, (j + 1) * s + i, (j + 1) * s + i + 1
            tri += [(v00, v10, v11), (v00, v11, v01)]
    if jitter:
        rng = np.random.default_rng(seed)
        inner = bnd == 0
        xy[inner] += rng.uniform(-jitter * h, jitter * h, size=(inner.sum(), 2))
    return mesh_from_triangles(len(xy), np.array(tri, np.int32), xy, bnd)


def mesh_from_triangles(n, tri, xy, bnd):
    adj = [set() for _ in range(n)]
    for a, b, c in tri:
        for p, q in ((a, b), (b, c), (c, a)):
            adj[p].add(q)
            adj[q].add(p)
    row_ptr = np.zeros(n + 1, np.int32)
    col = []
    for v in range(n):
        col += sorted(adj[v])
        row_ptr[v + 1] = len(col)
    return dict(n=n, xy=xy, tri=tri, is_boundary=bnd, row_ptr=row_ptr, col_idx=np.array(col, np.int32))


def dense_adjacency(m):
    n = m["n"]
    A = np.zeros((n, n))
    for v in range(n):
        for e in range(m["row_ptr"][v], m["row_ptr"][v + 1]):
            A[v, m["col_idx"][e]] = 1.0
    return A


def path_mesh(m_len, a, b, y_fn):
    """Path 0..m with both ends fixed, as a CSR graph (no triangles)."""
    n = m_len + 1
    row_ptr = [0]
    col = []
    for v in range(n):
        nb = [u for u in (v - 1, v + 1) if 0 <= u < n]
        col += nb
        row_ptr.append(len(col))
    bnd = np.zeros(n, np.uint8)
    bnd[0] = bnd[-1] = 1
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, n)
    x[0], x[-1] = a, b
    xy = np.stack([x, y_fn(np.arange(n))], axis=1).astype(np.float64)
    return dict(n=n, row_ptr=np.array(row_ptr, np.int32), col_idx=np.array(col, np.int32), is_boundary=bnd, xy=xy)


def small_meshes():
    """Tiny generated meshes with flips and splits (degree 3..12)."""
    return [meshgen.workload(1, side=s) for s in (5, 7, 9)] + [meshgen.workload(2, side=8), meshgen.workload(0, side=6)]


# ------------------------------------------------------------------ Eq. 1


def test_uniform_grid_is_exact_fixed_point():
    # every interior vertex of a same-diagonal grid has centrally symmetric neighbours
    # (+-x, +-y, +-(1,1)): Eq. 1 returns it exactly (dyadic spacing, all sums exact)
    m = grid_mesh(17)
    x1 = oracle.jacobi_sweep(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"])
    assert np.array_equal(x1, m["xy"])
    x2 = oracle.inplace_sweep(m["row_ptr"], m["col_idx"], m["is_boundary"], np.arange(m["n"]), m["xy"])
    assert np.array_equal(x2, m["xy"])
    xs, k, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 25)
    assert k == 25 and np.array_equal(xs, m["xy"])


def test_random_diagonal_grid_is_not_fixed_point():
    # with random diagonals the neighbourhoods are no longer symmetric: the sweep must move vertices
    m = meshgen.generate(17, jitter=0.0, seed=11)
    x1 = oracle.jacobi_sweep(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"])
    assert np.abs(x1 - m["xy"]).max() > 1e-3


@pytest.mark.parametrize("mode", [oracle.JACOBI, oracle.INPLACE])
def test_boundary_never_moves(mode):
    m = meshgen.workload(1, side=24)
    seq = oracle.order(m, oracle.RDR)
    x, k, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 40, mode=mode, seq=seq)
    b = m["is_boundary"] == 1
    assert np.array_equal(x[b], m["xy"][b])
    assert np.abs(x[~b] - m["xy"][~b]).max() > 1e-4


def test_path_jacobi_matches_sine_series_closed_form():
    # path 0..m, ends fixed at a, b: the error e = x - (a + (b-a) j/m) evolves as
    # e^k_j = sum_s c_s cos^k(s pi/m) sin(s pi j/m), c_s the discrete sine coefficients of e^0
    mlen, a, b = 24, 0.25, 1.75
    m = path_mesh(mlen, a, b, lambda j: np.sin(0.3 * j))
    j = np.arange(mlen + 1)
    lines = [m["xy"][0] + (m["xy"][-1] - m["xy"][0]) * j[:, None] / mlen]
    e0 = m["xy"] - lines[0]
    sidx = np.arange(1, mlen)
    S = np.sin(np.pi * np.outer(sidx, j) / mlen)           # [s, j]
    c = (2.0 / mlen) * S @ e0                                # [s, 2]
    for k in (1, 3, 17, 200):
        x, done, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], k)
        ek = (S.T * np.cos(np.pi * sidx / mlen) ** k) @ c
        assert done == k
        np.testing.assert_allclose(x, lines[0] + ek, rtol=0, atol=1e-13)
    x, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 20000)
    np.testing.assert_allclose(x, lines[0], rtol=0, atol=1e-12)


def test_path_gauss_seidel_rate_is_square_of_jacobi_rate():
    # in-place sweep over a 2-colouring (red-black) of a path: the slowest error mode decays
    # by cos^2(pi/m) per sweep, against cos(pi/m) for Jacobi
    mlen = 20
    m = path_mesh(mlen, 0.0, 1.0, lambda j: 0.0 * j)
    line = np.linspace(0.0, 1.0, mlen + 1)
    perm = np.arange(mlen + 1, dtype=np.int32)
    colour, nc = oracle.color_greedy(m["row_ptr"], m["col_idx"], m["is_boundary"], perm)
    assert nc == 2
    seq = oracle.color_sequence(m["is_boundary"], perm, colour, nc)

    def err_after(k, mode):
        x, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], k, mode=mode, seq=seq)
        return np.abs(x[:, 0] - line).max()

    # modes s=1 and s=m-1 both decay by |cos(pi/m)| for Jacobi (the second alternates in sign),
    # so measure the rate over an even number of sweeps
    # (late enough that the s=2 mode, decaying by cos(2 pi/m), no longer shows)
    rj = (err_after(1200, oracle.JACOBI) / err_after(1000, oracle.JACOBI)) ** (1.0 / 200)
    assert abs(rj - math.cos(math.pi / mlen)) < 1e-6
    rg = (err_after(600, oracle.INPLACE) / err_after(400, oracle.INPLACE)) ** (1.0 / 200)
    assert abs(rg - math.cos(math.pi / mlen) ** 2) < 1e-6


@pytest.mark.parametrize("idx", range(5))
def test_jacobi_equals_dense_matrix_iteration(idx):
    # x^{k+1}_I = D^-1 A x^k on interior rows, boundary rows unchanged
    m = small_meshes()[idx]
    A = dense_adjacency(m)
    D = A.sum(axis=1)
    inner = m["is_boundary"] == 0
    x = m["xy"].copy()
    for _ in range(7):
        nx = x.copy()
        nx[inner] = (A[inner] @ x) / D[inner, None]
        x = nx
    got, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 7)
    np.testing.assert_allclose(got, x, rtol=0, atol=1e-14)


@pytest.mark.parametrize("idx", range(5))
def test_inplace_sweep_equals_forward_substitution(idx):
    # Algorithm 1's in-place sweep in order sigma is one step of (D - L_sigma) x' = U_sigma x + B x_B
    m = small_meshes()[idx]
    A = dense_adjacency(m)
    n = m["n"]
    for ordering in (oracle.ORI, oracle.RANDOM, oracle.RDR):
        sigma = oracle.order(m, ordering, seed=5)
        inner_seq = [v for v in sigma if not m["is_boundary"][v]]
        pos = {v: i for i, v in enumerate(inner_seq)}
        ni = len(inner_seq)
        bidx = [v for v in range(n) if m["is_boundary"][v]]
        x = m["xy"].copy()
        for _ in range(3):
            M = np.zeros((ni, ni))
            rhs = np.zeros((ni, 2))
            for v in inner_seq:
                r = pos[v]
                M[r, r] = A[v].sum()
                for u in np.nonzero(A[v])[0]:
                    if m["is_boundary"][u]:
                        rhs[r] += x[u]
                    elif pos[u] < r:
                        M[r, pos[u]] = -1.0
                    else:
                        rhs[r] += x[u]
            sol = np.linalg.solve(M, rhs)
            nx = x.copy()
            nx[inner_seq] = sol
            nx[bidx] = x[bidx]
            x = nx
        got, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 3, mode=oracle.INPLACE,
                                  seq=sigma)
        np.testing.assert_allclose(got, x, rtol=0, atol=1e-13)


def test_all_modes_converge_to_discrete_harmonic_solution():
    # the common limit of every sweep and ordering solves L_II x_I = -L_IB x_B (Tutte embedding)
    m = meshgen.workload(1, side=12)
    A = dense_adjacency(m)
    L = np.diag(A.sum(axis=1)) - A
    inner = np.nonzero(m["is_boundary"] == 0)[0]
    bd = np.nonzero(m["is_boundary"] == 1)[0]
    xI = np.linalg.solve(L[np.ix_(inner, inner)], -L[np.ix_(inner, bd)] @ m["xy"][bd])
    for ordering in (oracle.ORI, oracle.RANDOM, oracle.BFS, oracle.RDR):
        p = oracle.order(m, ordering, seed=9)
        xj, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 4000)
        np.testing.assert_allclose(xj[inner], xI, rtol=0, atol=1e-12)
        xg, _, _ = oracle.gs_smooth(m, p, 2000)
        np.testing.assert_allclose(xg[inner], xI, rtol=0, atol=1e-12)
        xs, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 2000, mode=oracle.INPLACE,
                                 seq=p)
        np.testing.assert_allclose(xs[inner], xI, rtol=0, atol=1e-12)


@pytest.mark.parametrize("ordering", [oracle.RANDOM, oracle.BFS, oracle.RDR])
def test_jacobi_is_bit_invariant_under_relabelling(ordering):
    # rows keep their entry order under relabelling, so every neighbour sum adds the same
    # numbers in the same order: Jacobi commutes with the permutation exactly
    m = meshgen.workload(1, side=33)
    p = oracle.order(m, ordering, seed=21)
    rp, ci = oracle.relabel(m["row_ptr"], m["col_idx"], p)
    x_ref, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 15)
    x_p, _, _ = oracle.smooth(rp, ci, m["is_boundary"][p], m["xy"][p], 15)
    back = np.empty_like(x_p)
    back[p] = x_p
    assert np.array_equal(back, x_ref)


# --------------------------------------------------------------- quality


def test_quality_closed_forms():
    g = json.load(open(os.path.join(GOLDEN, "quality_closed_forms.json")))
    for t in g["triangles"]:
        xy = np.array(t["xy"], np.float64)
        for corners in ([0, 1, 2], [1, 2, 0], [2, 0, 1], [0, 2, 1]):
            q = oracle.triangle_quality(np.array([corners], np.int32), xy)[0]
            assert q == t["q_num"] / t["q_den"], t["name"]
    mm = g["two_triangle_mesh"]
    xy, tri = np.array(mm["xy"], np.float64), np.array(mm["tri"], np.int32)
    qv = oracle.vertex_quality(4, tri, xy)
    for got, (a, b) in zip(qv, mm["q_v_num_den"]):
        assert abs(got - a / b) <= 2 * np.spacing(a / b)
    Q = oracle.mesh_quality(4, tri, xy)
    a, b = mm["Q_num_den"]
    assert abs(Q - a / b) <= 4 * np.spacing(a / b)


def test_quality_right_isosceles_and_equilateral():
    m = grid_mesh(9)
    q = oracle.triangle_quality(m["tri"], m["xy"])
    assert np.abs(q - 1 / math.sqrt(2)).max() <= np.spacing(1 / math.sqrt(2))
    Q = oracle.mesh_quality(m["n"], m["tri"], m["xy"])
    assert abs(Q - 1 / math.sqrt(2)) <= 8 * np.spacing(1 / math.sqrt(2))
    eq = np.array([[0.0, 0.0], [1.0, 0.0], [0.5, math.sqrt(3) / 2]])
    qe = oracle.triangle_quality(np.array([[0, 1, 2]], np.int32), eq)[0]
    assert abs(qe - 1.0) < 1e-15 and qe <= 1.0


def test_quality_range_and_isolated_vertex():
    m = meshgen.workload(1, side=20)
    q_t = oracle.triangle_quality(m["tri"], m["xy"])
    assert (q_t > 0).all() and (q_t <= 1).all()
    # a vertex that belongs to no triangle has quality 0 and still counts in |V|
    xy = np.vstack([m["xy"], [[5.0, 5.0]]])
    qv = oracle.vertex_quality(m["n"] + 1, m["tri"], xy)
    assert qv[-1] == 0.0
    Q1 = oracle.mesh_quality(m["n"] + 1, m["tri"], xy)
    Q0 = oracle.mesh_quality(m["n"], m["tri"], m["xy"])
    assert abs(Q1 - Q0 * m["n"] / (m["n"] + 1)) < 1e-15


def test_quality_is_similarity_invariant():
    # the edge-length ratio does not change under translation, rotation and uniform scaling
    m = meshgen.workload(1, side=15)
    c, s = math.cos(0.7), math.sin(0.7)
    R = np.array([[c, -s], [s, c]])
    xy2 = (m["xy"] @ R.T) * 3.5 + np.array([10.0, -4.0])
    np.testing.assert_allclose(oracle.triangle_quality(m["tri"], xy2), oracle.triangle_quality(m["tri"], m["xy"]),
                               rtol=1e-13)


# --------------------------------------------------------- stopping rule


def test_stopping_rule_on_fixed_point_stops_after_one_sweep():
    m = grid_mesh(9)
    x, k, hist = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 50, tri=m["tri"], tol=5e-6)
    assert k == 1 and hist[1] - hist[0] == 0.0


def test_stopping_rule_sequence():
    # the loop stops at the first sweep whose improvement is below tol, never earlier;
    # each recorded Q_k is the quality of the mesh after exactly k fixed sweeps
    m = meshgen.workload(1, side=30)
    for tol in (5e-6, 1e-4, 1e-3):
        x, k, hist = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 500, tri=m["tri"], tol=tol)
        d = np.diff(hist)
        assert k < 500
        assert (d[:-1] >= tol).all() and d[-1] < tol
        xk, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], k)
        assert np.array_equal(xk, x)
        assert oracle.mesh_quality(m["n"], m["tri"], xk) == hist[-1]
    # goal reached after the first sweep
    Q0 = oracle.mesh_quality(m["n"], m["tri"], m["xy"])
    _, k, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 100, tri=m["tri"], tol=0.0,
                            goal=Q0)
    assert k == 1


def test_smoothing_improves_quality_of_jittered_mesh():
    # the purpose of LMS (Section 3.2): mean quality rises on a jittered mesh
    m = meshgen.workload(1, side=40)
    Q0 = oracle.mesh_quality(m["n"], m["tri"], m["xy"])
    x, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 20)
    assert oracle.mesh_quality(m["n"], m["tri"], x) > Q0 + 0.05


# -------------------------------------------------------------- orderings


def _is_perm(p, n):
    return len(p) == n and np.array_equal(np.sort(p), np.arange(n))


def test_rdr_golden_4x4():
    """Algorithm 2 by hand on the 4x4 grid of orderings_4x4.json (keys q_v given).

    interior by key: 9 (.2), 6 (.3), 5 (.4), 10 (.45)
    i=9: order 9; l = {13,5,10,4,8,14} -> order all; go to 13
      l(13) = [8,14,12] -> order 12; go to 8;  l(8) = [4,12]; go to 4
      l(4) = [5,0] -> order 0; go to 5;  l(5) = [6,10,1,0] -> order 6,1; go to 6
      l(6) = [10,1,11,2,7] -> order 11,2,7; go to 10;  l(10) = [11,14,15] -> order 15; go to 11
      l(11) = [7,15]; go to 7;  l(7) = [2,3] -> order 3; go to 2;  l(2) = [1,3]; go to 1
      l(1) = [0]; go to 0;  l(0) = [] -> stop.   6, 5, 10 are already processed.
    """
    g = json.load(open(os.path.join(GOLDEN, "orderings_4x4.json")))
    rp, ci, bnd, q = (np.array(g[k]) for k in ("row_ptr", "col_idx", "is_boundary", "q_v"))
    p = oracle.order_rdr(rp, ci, bnd, q)
    assert p.tolist() == g["rdr_new_to_old"]
    assert oracle.order_bfs(rp, ci).tolist() == g["bfs_new_to_old"]
    colour, nc = oracle.color_greedy(rp, ci, bnd, p)
    assert colour.tolist() == g["rdr_colour"] and nc == g["rdr_ncolours"]
    assert oracle.color_sequence(bnd, p, colour, nc).tolist() == g["rdr_gs_sequence"]


def test_rdr_golden_path_and_star():
    """Path: i=2 orders 2, l=[3,1] -> order 3,1; go to 3: l=[4] -> order 4; go to 4: l=[] -> stop.
    i=1 (ordered, not processed): l=[0] -> order 0; go to 0: l=[] -> stop.  5, 6 never reached: appended.
    Star: centre 0, l = [3, 1, 2, 4] (keys .1 then three ties at .7 ordered by id)."""
    g = json.load(open(os.path.join(GOLDEN, "rdr_small.json")))
    for case in g["cases"]:
        p = oracle.order_rdr(np.array(case["row_ptr"]), np.array(case["col_idx"]), np.array(case["is_boundary"]),
                             np.array(case["q_v"]))
        assert p.tolist() == case["rdr_new_to_old"], case["name"]


@pytest.mark.parametrize("side", [6, 17, 40])
def test_orderings_are_permutations(side):
    # Theorem 1: every vertex ordered exactly once
    m = meshgen.workload(1, side=side)
    for ordering in (oracle.ORI, oracle.RANDOM, oracle.BFS, oracle.RDR):
        assert _is_perm(oracle.order(m, ordering, seed=side), m["n"])


def test_rdr_structure_on_generated_mesh():
    # the first entry is the worst interior vertex; the next entries are its neighbours by
    # increasing (quality, id); every walk step continues from the worst unprocessed neighbour
    m = meshgen.workload(1, side=30)
    q = oracle.vertex_quality(m["n"], m["tri"], m["xy"])
    p = oracle.order_rdr(m["row_ptr"], m["col_idx"], m["is_boundary"], q)
    inner = np.nonzero(m["is_boundary"] == 0)[0]
    first = min(inner, key=lambda v: (q[v], v))
    assert p[0] == first
    nb = m["col_idx"][m["row_ptr"][first]:m["row_ptr"][first + 1]]
    expect = sorted(nb, key=lambda v: (q[v], v))
    assert p[1:1 + len(nb)].tolist() == [int(v) for v in expect]
    # positions grow along the order of first appearance; neighbours of any ordered interior
    # vertex appear within the list (no vertex missing)
    assert _is_perm(p, m["n"])


def test_bfs_levels_non_decreasing():
    m = meshgen.workload(1, side=25)
    p = oracle.order_bfs(m["row_ptr"], m["col_idx"])
    assert p[0] == 0
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
    assert (np.diff(level[p]) >= 0).all()


def test_random_ordering_matches_splitmix64_known_answers():
    # splitmix64 from state 0 (Steele, Lea & Flood 2014; reference outputs of Vigna's splitmix64.c):
    # 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F.  Fisher-Yates on n=4 draws
    # j = out0 % 4, out1 % 3, out2 % 2 for i = 3, 2, 1.
    outs = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    p = [0, 1, 2, 3]
    for i, o in zip((3, 2, 1), outs):
        j = o % (i + 1)
        p[i], p[j] = p[j], p[i]
    assert oracle.order_random(4, 0).tolist() == p
    assert not np.array_equal(oracle.order_random(1000, 1), oracle.order_random(1000, 2))


def test_relabel_round_trip_and_row_order():
    m = meshgen.workload(1, side=20)
    p = oracle.order(m, oracle.RDR)
    rp, ci = oracle.relabel(m["row_ptr"], m["col_idx"], p)
    inv = np.empty_like(p)
    inv[p] = np.arange(len(p), dtype=np.int32)
    for k in range(0, m["n"], 7):
        old = m["col_idx"][m["row_ptr"][p[k]]:m["row_ptr"][p[k] + 1]]
        assert ci[rp[k]:rp[k + 1]].tolist() == inv[old].tolist()
    rp2, ci2 = oracle.relabel(rp, ci, inv)
    assert np.array_equal(rp2, m["row_ptr"]) and np.array_equal(ci2, m["col_idx"])


# -------------------------------------------------------------- colouring


@pytest.mark.parametrize("ordering", [oracle.ORI, oracle.RANDOM, oracle.BFS, oracle.RDR])
def test_colouring_is_proper_and_first_fit(ordering):
    m = meshgen.workload(1, side=35)
    p = oracle.order(m, ordering, seed=4)
    colour, nc = oracle.color_greedy(m["row_ptr"], m["col_idx"], m["is_boundary"], p)
    pos = np.empty(m["n"], np.int64)
    pos[p] = np.arange(m["n"])
    assert (colour[m["is_boundary"] == 1] == -1).all()
    for v in range(m["n"]):
        if m["is_boundary"][v]:
            continue
        nb = m["col_idx"][m["row_ptr"][v]:m["row_ptr"][v + 1]]
        nb_int = [u for u in nb if not m["is_boundary"][u]]
        assert all(colour[u] != colour[v] for u in nb_int)
        earlier = {colour[u] for u in nb_int if pos[u] < pos[v]}
        assert all(c in earlier for c in range(colour[v]))
    assert nc == colour.max() + 1 and nc <= 13


def test_coloured_gs_independent_of_order_inside_colour():
    # vertices of one colour share no edge, so their in-place updates commute exactly
    m = meshgen.workload(1, side=25)
    p = oracle.order(m, oracle.RDR)
    colour, nc = oracle.color_greedy(m["row_ptr"], m["col_idx"], m["is_boundary"], p)
    seq = oracle.color_sequence(m["is_boundary"], p, colour, nc)
    rng = np.random.default_rng(0)
    shuffled = np.concatenate([rng.permutation(seq[colour[seq] == c]) for c in range(nc)])
    a, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 9, mode=oracle.INPLACE, seq=seq)
    b, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 9, mode=oracle.INPLACE,
                            seq=shuffled)
    assert np.array_equal(a, b)


def test_plausible_mistakes_fail_the_pins():
    # the dense-matrix pin would catch a dropped neighbour, and the closed-form quality pin a
    # swapped min/max: check the pins' sensitivity on a mutated copy of the data, on the CPU
    m = small_meshes()[0]
    A = dense_adjacency(m)
    inner = m["is_boundary"] == 0
    x = m["xy"].copy()
    ref = x.copy()
    ref[inner] = (A[inner] @ x) / A.sum(axis=1)[inner, None]
    bad = m["col_idx"].copy()
    v = int(np.nonzero(inner)[0][0])
    bad[m["row_ptr"][v]] = bad[m["row_ptr"][v] + 1]        # one neighbour read twice, another dropped
    got = oracle.jacobi_sweep(m["row_ptr"], bad, m["is_boundary"], x)
    assert np.abs(got - ref).max() > 1e-6
    q = oracle.triangle_quality(np.array([[0, 1, 2]], np.int32), np.array([[0, 0], [4, 0], [0, 3]], np.float64))
    assert q[0] != 5 / 3


def test_openmp_timing_baseline_equals_oracle_jacobi():
    """The all-core timing baseline (OpenMP static schedule over vertices) runs the oracle's Eq. 1
    arithmetic per vertex, so its Jacobi result equals the single-thread oracle bit for bit at any thread
    count."""
    m = meshgen.generate(37, jitter=0.3, flip_frac=0.10, split_frac=0.05, seed=77)
    want, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 13)
    for threads in (1, 3, 0):
        got, used = oracle.jacobi_omp(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 13, threads)
        assert used >= 1 and (threads == 0 or used == threads)
        assert np.array_equal(got, want)
