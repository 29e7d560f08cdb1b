"""FP64 sweeps with their arithmetic on the integer pipes (LMS_FP64_ARITH_INT_ADDS / _INT) and on the FP64
unit: the device addition and division against IEEE arithmetic, and every mode bit-identical to the
oracle."""
import numpy as np
import pytest

import meshgen
import oracle
import paper_1606_00803_gb300 as lms
from test_fp64_int_host import from_parts

pytestmark = pytest.mark.gpu

MODES = [lms.FP64_ARITH_FPU, lms.FP64_ARITH_INT_ADDS, lms.FP64_ARITH_INT, lms.FP64_ARITH_MIXED2,
         lms.FP64_ARITH_MIXED3]


def check_device_add(a, b):
    got = lms.selftest_add64(a, b)
    assert np.array_equal(got.view(np.uint64), (a + b).view(np.uint64))


def test_device_addition_matches_ieee():
    rng = np.random.default_rng(11)
    n = 1_000_000
    ea = rng.integers(900, 1150, n)
    a = from_parts(rng.integers(0, 2, n), ea, rng.integers(0, 1 << 52, n, dtype=np.uint64))
    b = from_parts(rng.integers(0, 2, n), np.clip(ea + rng.integers(-70, 71, n), 1, 2045),
                   rng.integers(0, 1 << 52, n, dtype=np.uint64))
    check_device_add(a, b)
    # ties and exact sums (few significant bits), cancellations, carries with a sticky bit
    top = rng.integers(0, 16, n, dtype=np.uint64) << np.uint64(48)
    a = from_parts(rng.integers(0, 2, n), ea, top)
    b = from_parts(rng.integers(0, 2, n), ea - rng.integers(0, 66, n),
                   rng.integers(0, 16, n, dtype=np.uint64) << np.uint64(48))
    check_device_add(a, b)
    x = rng.uniform(-4, 4, n)
    check_device_add(x, -x * (1 + rng.uniform(-1e-6, 1e-6, n)))
    near2 = np.uint64((1 << 52) - 1) - rng.integers(0, 1 << 30, n, dtype=np.uint64)
    check_device_add(from_parts(np.zeros(n, np.int64), ea, near2),
                     from_parts(np.zeros(n, np.int64), ea - rng.integers(11, 21, n),
                                rng.integers(0, 1 << 52, n, dtype=np.uint64)))
    tiny, big = np.finfo(np.float64).tiny, np.finfo(np.float64).max
    v = np.array([0.0, -0.0, tiny, -tiny, 5e-324, 1.5 * tiny, -1.25 * tiny, big / 2, 2.0 ** 1023, 1.0, -0.3])
    p, q = np.meshgrid(v, v)
    with np.errstate(over="ignore"):
        check_device_add(p.ravel(), q.ravel())


def test_device_division_matches_ieee():
    rng = np.random.default_rng(12)
    n = 1_280_000
    d = np.tile(np.arange(1, 65, dtype=np.int32), n // 64)
    s = from_parts(rng.integers(0, 2, n), rng.integers(1, 2047, n), rng.integers(0, 1 << 52, n, dtype=np.uint64))
    assert np.array_equal(lms.selftest_divint64(s, d).view(np.uint64), (s / d).view(np.uint64))
    m = rng.integers(1, 1 << 46, n).astype(np.float64) * d
    for x in (m, np.nextafter(m, np.inf), np.nextafter(m, -np.inf), rng.uniform(-0.5, 0.5, n) * d):
        assert np.array_equal(lms.selftest_divint64(x, d).view(np.uint64), (x / d).view(np.uint64))
    tiny = np.finfo(np.float64).tiny
    v = np.array([0.0, -0.0, 5e-324, tiny / 2, tiny, 3 * tiny, 64 * tiny, 1e-307, np.finfo(np.float64).max])
    x, dd = np.meshgrid(v, np.arange(1, 70, dtype=np.int32))  # 65..69 take the FP64 division
    x, dd = x.ravel(), dd.ravel()
    assert np.array_equal(lms.selftest_divint64(x, dd).view(np.uint64), (x / dd).view(np.uint64))


def straddling(m):
    """The mesh moved so that its box straddles the origin: sums mix signs and cancel."""
    m = dict(m)
    m["xy"] = m["xy"] - np.array([0.4375, 0.53125])
    return m


@pytest.fixture(scope="module", params=["unit_square", "straddling_origin"])
def mesh(request):
    m = meshgen.workload(1, side=90)  # ~8.5k vertices: many blocks, a ragged tail
    return m if request.param == "unit_square" else straddling(m)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("ordering", [lms.ORI, lms.RDR])
def test_jacobi_every_add_mode_bit_exact(mesh, mode, ordering):
    m = mesh
    want, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 30)
    with lms.Mesh.from_dict(m, lms.FP64) as g:
        g.reorder(ordering)
        g.set_fp64_arith(mode)
        g.smooth(30)
        got = g.coords()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("mode", MODES)
def test_coloured_gs_every_add_mode_bit_exact(mesh, mode):
    m = mesh
    p = oracle.order(m, oracle.BFS)
    want, _, _ = oracle.gs_smooth(m, p, 12)
    with lms.Mesh.from_dict(m, lms.FP64) as g:
        g.reorder(lms.BFS)
        g.set_fp64_arith(mode)
        g.smooth(12, mode=lms.COLORED_GS)
        got = g.coords()
    assert np.array_equal(got, want)


def test_switching_modes_between_sweeps_and_stopping_rule():
    m = straddling(meshgen.workload(2, side=60))
    tol = 5e-6
    _, k_or, hist = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 200, tri=m["tri"], tol=tol)
    with lms.Mesh.from_dict(m, lms.FP64) as g:
        g.reorder(lms.RDR)
        g.set_fp64_arith(lms.FP64_ARITH_INT)
        k = g.smooth(200, tol=tol)
        # the stop may differ only where the oracle's quality change is within 1e-9 of tol
        assert k == k_or or abs(np.diff(hist) - tol)[min(k, k_or) - 1] < 1e-9
        want, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], k)
        assert np.array_equal(g.coords(), want)
        # the same sweeps split across modes
        g.set_coords(m["xy"])
        g.set_fp64_arith(lms.FP64_ARITH_FPU)
        g.smooth(7)
        g.set_fp64_arith(lms.FP64_ARITH_INT_ADDS)
        g.smooth(6)
        g.set_fp64_arith(lms.FP64_ARITH_INT)
        g.smooth(4)
        g.set_fp64_arith(lms.FP64_ARITH_MIXED2)
        g.smooth(3)
        got = g.coords()
    want20, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 20)
    assert np.array_equal(got, want20)


def test_rejects_unknown_mode():
    m = meshgen.workload(0)
    with lms.Mesh.from_dict(m, lms.FP64) as g:
        with pytest.raises(lms.LmsError):
            g.set_fp64_arith(5)
