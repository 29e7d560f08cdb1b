"""The per-sweep mesh quality Q_k that drives the Section 5.1 stopping rule, against the oracle's Section 3.2
definition: FP64 positions within 1e-13, FP32 positions within 1e-6, across the ranges where the FP64
kernel takes its fast root (FP32 seed + Newton steps) and where it falls back to sqrt(min / max)."""
import numpy as np
import pytest

import meshgen
import oracle
import paper_1606_00803_gb300 as lms

pytestmark = pytest.mark.gpu


def q_first(m, precision):
    """Q_0 as the stopping rule computes it: one sweep under a tolerance that stops after it."""
    with lms.Mesh.from_dict(m, precision) as g:
        g.smooth(1, tol=1e9)
        return g.last_stats()["q_first"]


def scaled(m, s, shift=(0.0, 0.0)):
    m = dict(m)
    m["xy"] = m["xy"] * s + np.array(shift)
    return m


@pytest.fixture(scope="module")
def base():
    return meshgen.workload(2, side=50)  # graded: edge ratios well spread


@pytest.mark.parametrize("scale,shift", [(1.0, (0.0, 0.0)), (1.0, (-0.4, -0.6)), (1e-150, (0.0, 0.0)),
                                         (1e150, (0.0, 0.0)), (3e-300, (0.0, 0.0)), (1e-5, (7.0, -3.0))])
def test_fp64_sweep_quality_matches_definition(base, scale, shift):
    m = scaled(base, scale, shift)
    want = oracle.mesh_quality(m["n"], m["tri"], m["xy"])
    assert abs(q_first(m, lms.FP64) - want) <= 1e-13


def test_fp64_sweep_quality_degenerate_and_needle_triangles(base):
    m = scaled(base, 1.0)
    xy = m["xy"].copy()
    tri = m["tri"].reshape(-1, 3)
    rng = np.random.default_rng(5)
    # zero-length edges (two corners on one point), needles (shortest edge 1e-20 of the longest) and
    # whole triangles collapsed to a point
    for t in rng.choice(len(tri), 40, replace=False):
        xy[tri[t, 1]] = xy[tri[t, 0]]
    for t in rng.choice(len(tri), 40, replace=False):
        xy[tri[t, 2]] = xy[tri[t, 1]] + np.array([1e-20, 0.0])
    for t in rng.choice(len(tri), 10, replace=False):
        xy[tri[t, 1]] = xy[tri[t, 2]] = xy[tri[t, 0]]
    m["xy"] = xy
    want = oracle.mesh_quality(m["n"], m["tri"], m["xy"])
    assert abs(q_first(m, lms.FP64) - want) <= 1e-13


@pytest.mark.parametrize("scale,shift", [(1.0, (0.0, 0.0)), (1e-30, (5.0, 5.0)), (1e30, (0.0, 0.0))])
def test_fp32_sweep_quality_matches_definition(base, scale, shift):
    m = scaled(base, scale, shift)
    want = oracle.mesh_quality(m["n"], m["tri"], m["xy"])
    assert abs(q_first(m, lms.FP32) - want) <= 1e-6


def test_fp32_sweep_quality_large_mesh():
    # 4.6M vertices: per-thread FP32 sums over ~35 triangles each, Kahan-compensated
    m = meshgen.workload(2)
    want = oracle.mesh_quality(m["n"], m["tri"], m["xy"])
    assert abs(q_first(m, lms.FP32) - want) <= 1e-6
    assert abs(q_first(m, lms.FP64) - want) <= 1e-13
