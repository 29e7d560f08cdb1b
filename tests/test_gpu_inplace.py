"""The paper's parallel in-place sweep (LMS_INPLACE_STATIC) against the oracle.

With one GPU thread the mode is the sequential Algorithm 1 in storage order and must equal the
oracle's in-place sweep bit for bit in FP64.  With many threads (the paper's static split of the
vertices between threads, racing on block borders) results depend on timing, so they are checked
against what holds for every interleaving: boundary vertices never move, every position stays a
convex combination of the old ones (inside the bounding box), the iteration converges to the same
discrete harmonic limit as the sequential sweep, and the stopping rule fires no later than Jacobi's.
"""
import math

import numpy as np
import pytest

import meshgen
import oracle
import paper_1606_00803_gb300 as lms

pytestmark = pytest.mark.gpu

ORDERINGS = [lms.ORI, lms.RANDOM, lms.BFS, lms.RDR, lms.RBFS]


def diag(m):
    return math.hypot(np.ptp(m["xy"][:, 0]), np.ptp(m["xy"][:, 1]))


@pytest.fixture(scope="module")
def mesh():
    return meshgen.workload(1, side=33)


@pytest.mark.parametrize("ordering", ORDERINGS)
def test_one_thread_is_sequential_algorithm_1_bit_exact(mesh, ordering):
    m = mesh
    p = oracle.order(m, ordering, seed=3)
    want, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 12, mode=oracle.INPLACE, seq=p)
    with lms.Mesh.from_dict(m, lms.FP64) as g:
        g.reorder(ordering, seed=3)
        g.set_inplace_split(1)
        assert g.smooth(12, mode=lms.INPLACE_STATIC) == 12
        got = g.coords()
    assert np.array_equal(got, want)


def test_one_thread_fp32_within_tolerance(mesh):
    m = mesh
    p = oracle.order(m, oracle.RDR)
    want, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 100, mode=oracle.INPLACE, seq=p)
    with lms.Mesh.from_dict(m, lms.FP32) as g:
        g.reorder(lms.RDR)
        g.set_inplace_split(1)
        g.smooth(100, mode=lms.INPLACE_STATIC)
        got = g.coords()
    assert np.abs(got - want).max() <= 2e-6 * diag(m)


def test_back_from_the_coloured_layout(mesh):
    m = mesh
    p = oracle.order(m, oracle.BFS)
    mid, _, _ = oracle.gs_smooth(m, p, 5)
    want, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], mid, 4, mode=oracle.INPLACE, seq=p)
    with lms.Mesh.from_dict(m, lms.FP64) as g:
        g.reorder(lms.BFS)
        g.smooth(5, mode=lms.COLORED_GS)
        g.set_inplace_split(1)
        g.smooth(4, mode=lms.INPLACE_STATIC)
        assert np.array_equal(g.coords(), want)


@pytest.mark.parametrize("threads", [0, 32, 7, 100000])
@pytest.mark.parametrize("precision", [lms.FP64, lms.FP32])
def test_many_threads_keep_the_invariants(mesh, threads, precision):
    m = mesh
    bd = m["is_boundary"] == 1
    lo, hi = m["xy"].min(axis=0), m["xy"].max(axis=0)
    with lms.Mesh.from_dict(m, precision) as g:
        g.reorder(lms.RDR)
        g.set_inplace_split(threads)
        g.smooth(30, mode=lms.INPLACE_STATIC)
        got = g.coords()
        disp = g.last_stats()["max_disp"]
    assert np.isfinite(got).all() and np.array_equal(got[bd], m["xy"][bd])
    margin = (1e-12 if precision == lms.FP64 else 1e-6) * diag(m)  # FP32: rounding of the normalised form
    assert (got >= lo - margin).all() and (got <= hi + margin).all()
    assert math.isfinite(disp) and disp >= 0.0


@pytest.mark.parametrize("threads", [0, 32])
def test_many_threads_converge_to_the_harmonic_limit(threads):
    m = meshgen.workload(1, side=14)
    p = oracle.order(m, oracle.ORI)
    want, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 3000, mode=oracle.INPLACE, seq=p)
    with lms.Mesh.from_dict(m, lms.FP64) as g:
        g.set_inplace_split(threads)
        g.smooth(3000, mode=lms.INPLACE_STATIC)
        got = g.coords()
    assert np.abs(got - want).max() <= 1e-10 * diag(m)


def test_stopping_rule_fires_no_later_than_jacobi():
    m = meshgen.workload(1, side=60)
    with lms.Mesh.from_dict(m, lms.FP64) as g:
        g.reorder(lms.RDR)
        k_jacobi = g.smooth(400, mode=lms.JACOBI, tol=5e-6)
        g.set_coords(m["xy"])
        k_inplace = g.smooth(400, mode=lms.INPLACE_STATIC, tol=5e-6)
    assert 1 <= k_inplace <= k_jacobi < 400


def test_split_rejects_negative_thread_counts(mesh):
    with lms.Mesh.from_dict(mesh, lms.FP64) as g:
        with pytest.raises(lms.LmsError):
            g.set_inplace_split(-1)
