"""Block Gauss-Seidel sweeps (LMS_BLOCK_GS) through the C ABI against the oracle's in-place sweep in block
order: FP64 bit-exact, FP32 within 2e-6 x bounding-box diagonal."""
import math

import numpy as np
import pytest

import meshgen
import oracle
import paper_1606_00803_gb300 as lms

pytestmark = pytest.mark.gpu

TOL32 = 2e-6


def diag(m):
    return math.hypot(np.ptp(m["xy"][:, 0]), np.ptp(m["xy"][:, 1]))


@pytest.fixture(scope="module")
def mesh():
    return meshgen.workload(1, side=70)  # ~5k vertices: many tiles, a ragged last tile


@pytest.mark.parametrize("staged", [True, False])
@pytest.mark.parametrize("ordering", [lms.ORI, lms.BFS, lms.RDR, lms.RANDOM])
@pytest.mark.parametrize("tile", [32, 96, 1000])
def test_fp64_block_gs_bit_exact(mesh, ordering, tile, staged):
    """Both forms of the sweep - tile and halo staged in shared memory, or read from global memory - are
    the oracle's in-place sweep in block order, bit for bit."""
    m = mesh
    p = oracle.order(m, ordering, seed=3)
    want, _, _ = oracle.block_gs_smooth(m, p, tile, 12)
    with lms.Mesh.from_dict(m, lms.FP64) as g:
        g.reorder(ordering, seed=3)
        g.set_block_tile(tile)
        g.set_block_staging(staged)
        assert g.block_tile() == tile
        g.smooth(12, mode=lms.BLOCK_GS)
        got = g.coords()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("staged", [True, False])
@pytest.mark.parametrize("tile", [64, 512])
def test_fp32_block_gs_within_tolerance(mesh, tile, staged):
    m = mesh
    p = oracle.order(m, oracle.RDR)
    want, _, _ = oracle.block_gs_smooth(m, p, tile, 100)
    with lms.Mesh.from_dict(m, lms.FP32) as g:
        g.reorder(lms.RDR)
        g.set_block_tile(tile)
        g.set_block_staging(staged)
        g.smooth(100, mode=lms.BLOCK_GS)
        got = g.coords()
    assert np.abs(got - want).max() <= TOL32 * diag(m)


def test_block_gs_tile_too_large_for_shared_memory_falls_back():
    """A tile whose halo does not fit in one CTA's shared memory (a random order scatters the neighbours of
    a 40,000-position tile over the whole mesh) runs from global memory with the same result."""
    m = meshgen.workload(1, side=260)
    p = oracle.order(m, oracle.RANDOM, seed=5)
    want, _, _ = oracle.block_gs_smooth(m, p, 40000, 3)
    with lms.Mesh.from_dict(m, lms.FP64) as g:
        g.reorder(lms.RANDOM, seed=5)
        g.set_block_tile(40000)
        g.set_block_staging(1)
        g.smooth(3, mode=lms.BLOCK_GS)
        got = g.coords()
    assert np.array_equal(got, want)


def test_block_staging_rejects_bad_values():
    m = meshgen.workload(0)
    with lms.Mesh.from_dict(m, lms.FP64) as g:
        for bad in (-1, 2):
            with pytest.raises(lms.LmsError):
                g.set_block_staging(bad)


def test_block_gs_mixed_with_other_modes_and_automatic_tile():
    m = meshgen.workload(2, side=40)
    with lms.Mesh.from_dict(m, lms.FP64) as g:
        g.reorder(lms.BFS)
        tile = g.block_tile()  # chosen by mesh size
        assert 128 <= tile <= 1024
        g.smooth(3, mode=lms.COLORED_GS)  # colour-major layout, then back to the ordering's
        g.smooth(4, mode=lms.BLOCK_GS)
        g.smooth(2)
        got = g.coords()
        st = g.last_stats()
    p = oracle.order(m, oracle.BFS)
    x, _, _ = oracle.gs_smooth(m, p, 3)
    m2 = dict(m)
    m2["xy"] = x
    x, _, _ = oracle.block_gs_smooth(m2, p, tile, 4)
    want, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], x, 2)
    assert np.array_equal(got, want)
    assert st["max_disp"] > 0


def test_block_gs_stopping_rule_and_displacement():
    m = meshgen.workload(2, side=45)
    tol = 5e-6
    p = oracle.order(m, oracle.RDR)
    with lms.Mesh.from_dict(m, lms.FP64) as g:
        g.reorder(lms.RDR)
        g.set_block_tile(200)
        k = g.smooth(200, mode=lms.BLOCK_GS, tol=tol)
        got = g.coords()
        st = g.last_stats()
        g.smooth(1, mode=lms.BLOCK_GS)
        x1 = g.coords()
        disp = g.last_stats()["max_disp"]
    _, k_or, hist = oracle.block_gs_smooth(m, p, 200, 200, tol=tol)
    assert k == k_or or abs(np.diff(hist) - tol)[min(k, k_or) - 1] < 1e-9
    want, _, _ = oracle.block_gs_smooth(m, p, 200, k)
    assert np.array_equal(got, want)
    assert abs(st["q_first"] - hist[0]) < 1e-13
    assert abs(disp - np.sqrt(((x1 - got) ** 2).sum(axis=1)).max()) <= 1e-15 * diag(m) + 1e-12 * disp


def test_block_tile_rejects_negative():
    m = meshgen.workload(0)
    with lms.Mesh.from_dict(m, lms.FP64) as g:
        with pytest.raises(lms.LmsError):
            g.set_block_tile(-1)


RANGE_TILE = 65536  # tiles from this size up run on the block-range layout


@pytest.fixture(scope="module")
def mesh_big():
    return meshgen.workload(1, side=420)  # ~195k vertices: two 65,536-position tiles and a ragged third


@pytest.mark.parametrize("ordering", [lms.ORI, lms.BFS, lms.RDR, lms.RANDOM])
def test_fp64_block_gs_range_form_bit_exact(mesh_big, ordering):
    """Large tiles run as one range per (tile colour, vertex colour) on a layout sorted that way; that is
    the oracle's in-place sweep in block order, bit for bit."""
    m = mesh_big
    assert m["n"] > 2 * RANGE_TILE
    p = oracle.order(m, ordering, seed=3)
    want, _, _ = oracle.block_gs_smooth(m, p, RANGE_TILE, 6)
    with lms.Mesh.from_dict(m, lms.FP64) as g:
        g.reorder(ordering, seed=3)
        g.set_block_tile(RANGE_TILE)
        assert g.block_tile() == RANGE_TILE
        g.smooth(6, mode=lms.BLOCK_GS)
        got = g.coords()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("sweeps", [1, 2, 40])
@pytest.mark.parametrize("tile", [RANGE_TILE, 100000])
def test_fp32_block_gs_range_form_within_tolerance(mesh_big, sweeps, tile):
    """FP32 on the block-range layout: one in-place launch per range.  A range reading positions one sweep
    old would show as an error of the order of one sweep's displacement (about 1e-3 of the diagonal on this
    jittered mesh), far above the bound after the first sweeps."""
    m = mesh_big
    p = oracle.order(m, oracle.RDR)
    want, _, _ = oracle.block_gs_smooth(m, p, tile, sweeps)
    with lms.Mesh.from_dict(m, lms.FP32) as g:
        g.reorder(lms.RDR)
        g.set_block_tile(tile)
        g.smooth(sweeps, mode=lms.BLOCK_GS)
        got = g.coords()
    assert np.abs(got - want).max() <= TOL32 * diag(m)


@pytest.mark.parametrize("sweeps", [1, 2])
@pytest.mark.parametrize("ordering", [lms.BFS, lms.RDR, lms.RANDOM])
def test_fp32_coloured_gs_first_sweeps(mesh_big, ordering, sweeps):
    """Coloured GS in FP32 after one or two sweeps of a ~195k-vertex mesh: a colour pass that read a
    neighbour one sweep old would show as an error near one sweep's displacement."""
    m = mesh_big
    p = oracle.order(m, ordering, seed=9)
    want, _, _ = oracle.gs_smooth(m, p, sweeps)
    x0 = m["xy"]
    with lms.Mesh.from_dict(m, lms.FP32) as g:
        g.reorder(ordering, seed=9)
        g.smooth(sweeps, mode=lms.COLORED_GS)
        got = g.coords()
    assert np.abs(want - x0).max() > 100 * TOL32 * diag(m)  # the sweeps move vertices far beyond the bound
    assert np.abs(got - want).max() <= TOL32 * diag(m)


@pytest.mark.parametrize("precision", [lms.FP64, lms.FP32])
def test_block_gs_with_one_tile_is_coloured_gs(mesh_big, precision):
    """A tile covering the whole mesh has one tile colour, so its block order is the colour order and the
    block Gauss-Seidel sweeps the same ranges as coloured GS, with the same results."""
    m = mesh_big
    with lms.Mesh.from_dict(m, precision) as g:
        g.reorder(lms.RDR)
        g.smooth(5, mode=lms.COLORED_GS)
        a = g.coords()
        g.set_coords(m["xy"])
        g.set_block_tile(1 << 20)
        g.smooth(5, mode=lms.BLOCK_GS)
        b = g.coords()
    assert np.array_equal(a, b)
    if precision == lms.FP64:
        want, _, _ = oracle.gs_smooth(m, oracle.order(m, oracle.RDR), 5)
        assert np.array_equal(b, want)


def test_block_gs_range_form_stopping_rule_and_mixed_modes():
    m = meshgen.workload(2, side=300)
    tol = 2e-5  # the rule fires after about 30 sweeps
    p = oracle.order(m, oracle.BFS)
    with lms.Mesh.from_dict(m, lms.FP64) as g:
        g.reorder(lms.BFS)
        g.set_block_tile(RANGE_TILE)
        k = g.smooth(300, mode=lms.BLOCK_GS, tol=tol)
        got = g.coords()
        st = g.last_stats()
        # then: coloured GS, the range form with another tile, the small-tile form, Jacobi
        g.smooth(2, mode=lms.COLORED_GS)
        g.set_block_tile(70000)
        g.smooth(3, mode=lms.BLOCK_GS)
        g.set_block_tile(500)
        g.smooth(2, mode=lms.BLOCK_GS)
        g.smooth(1)
        chained = g.coords()
    _, k_or, hist = oracle.block_gs_smooth(m, p, RANGE_TILE, 300, tol=tol)
    assert k == k_or or abs(np.diff(hist) - tol)[min(k, k_or) - 1] < 1e-9
    want, _, _ = oracle.block_gs_smooth(m, p, RANGE_TILE, k)
    assert np.array_equal(got, want)
    assert abs(st["q_first"] - hist[0]) < 1e-13
    m2 = dict(m)
    m2["xy"], _, _ = oracle.gs_smooth(dict(m, xy=want), p, 2)
    m2["xy"], _, _ = oracle.block_gs_smooth(m2, p, 70000, 3)
    m2["xy"], _, _ = oracle.block_gs_smooth(m2, p, 500, 2)
    x, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m2["xy"], 1)
    assert np.array_equal(chained, x)


@pytest.mark.parametrize("precision", [lms.FP64, lms.FP32])
def test_block_gs_range_form_with_the_staged_kernel(mesh_big, precision):
    """The staged kernel (TMA tiles of rows and ids) sweeps the block-range layout's ranges too: FP64
    bit-exact, FP32 within tolerance."""
    m = mesh_big
    p = oracle.order(m, oracle.RDR)
    want, _, _ = oracle.block_gs_smooth(m, p, RANGE_TILE, 4)
    with lms.Mesh.from_dict(m, precision) as g:
        g.reorder(lms.RDR)
        g.set_launch(lms.KERNEL_STAGED, 256, 256)
        g.set_block_tile(RANGE_TILE)
        g.smooth(4, mode=lms.BLOCK_GS)
        got = g.coords()
    if precision == lms.FP64:
        assert np.array_equal(got, want)
    else:
        assert np.abs(got - want).max() <= TOL32 * diag(m)
