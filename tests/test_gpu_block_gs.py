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
