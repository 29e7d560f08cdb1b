"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances: FP64 max |dx| <= 1e-12 x bounding-box diagonal (and bit-exact
where the design promises it: Jacobi and coloured GS keep the oracle's
summation order and use a correctly rounded division); FP32 with normalised
coordinates and Kahan sums <= 2e-6 x diagonal after up to 200 sweeps;
permutations, colourings and relabelled CSR bit-exact.
"""
import math

import numpy as np
import pytest

import meshgen
import oracle
import paper_1606_00803_gb300 as lms

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-6
ORDERINGS = [lms.ORI, lms.RANDOM, lms.BFS, lms.RDR, lms.RBFS, lms.BRDR]


def diag(m):
    xy = m["xy"]
    return math.hypot(xy[:, 0].max() - xy[:, 0].min(), xy[:, 1].max() - xy[:, 1].min())


def err(a, b, m):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / diag(m)


@pytest.fixture(scope="module")
def mesh_mid():
    # ~10.5k vertices: many 256-thread blocks and a ragged last block
    return meshgen.workload(1, side=100)


@pytest.fixture(scope="module")
def mesh_graded():
    return meshgen.workload(2, side=70)


def test_division_selftest_matches_ieee():
    rng = np.random.default_rng(0)
    d = rng.integers(1, 80, size=2_000_000).astype(np.int32)
    s = rng.uniform(-8, 8, size=d.size) * np.exp2(rng.integers(-30, 30, size=d.size))
    # neighbour sums of positions: also exact multiples and values near them
    s[:1000] = np.arange(1000) * 3.0
    s[1000:2000] = np.nextafter(np.arange(1000) * 7.0, np.inf)
    s[2000:3000] = 0.0
    # sums whose quotients are subnormal or near it (IEEE division below biased exponent 64)
    s[3000:13000] = rng.uniform(-1, 1, 10000) * np.exp2(rng.integers(-1074, -900, 10000).astype(np.float64))
    q = lms.selftest_div64(s, d)
    assert np.array_equal(q.view(np.uint64), (s / d).view(np.uint64))


def test_fp32_mean_selftest_matches_ieee():
    """The FP32 sweeps' mean (rounded reciprocal, product, one fused correction) is the IEEE quotient bit
    for bit on 4M cases across the exponent range of FP32 neighbour sums, exact multiples and their
    neighbours, signed zeros and values near the largest finite one; for sums below 2^-100 (subnormal
    quotients, which no normalised mesh produces) it is within one ulp."""
    rng = np.random.default_rng(1)
    n = 4_000_000
    d = rng.integers(1, 65, size=n).astype(np.int32)
    e = rng.integers(-40, 20, size=n)
    s = (rng.uniform(-2, 2, size=n) * np.exp2(e)).astype(np.float32)
    k = np.arange(2000, dtype=np.float32)
    s[:2000] = k * d[:2000].astype(np.float32) * np.float32(0.125)           # exact quotients
    s[2000:4000] = np.nextafter(s[:2000], np.float32(np.inf))                 # their neighbours
    s[4000:5000] = 0.0
    s[5000:6000] = -0.0
    tiny = rng.uniform(-1, 1, 10000) * np.exp2(rng.integers(-149, -60, 10000).astype(np.float64))
    s[6000:16000] = tiny.astype(np.float32)
    s[16000:17000] = np.float32(3.0e38) * rng.uniform(-1, 1, 1000).astype(np.float32)
    q = lms.selftest_div32(s, d)
    want = (s / d.astype(np.float32)).astype(np.float32)
    exact = (np.abs(s) >= np.float32(2.0 ** -100)) | (s == 0)
    assert np.array_equal(q[exact].view(np.uint32), want[exact].view(np.uint32))
    # below 2^-100 (subnormal quotients): within one ulp, same sign
    qi, wi = q[~exact].view(np.int32).astype(np.int64), want[~exact].view(np.int32).astype(np.int64)
    assert np.all(np.abs(qi - wi) <= 1)


def test_config0_fp64_jacobi_bit_exact():
    m = meshgen.workload(0)
    want, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 10)
    with lms.Mesh.from_dict(m, lms.FP64) as g:
        assert g.smooth(10) == 10
        got = g.coords()
    assert err(got, want, m) <= TOL64
    assert np.array_equal(got, want)


@pytest.mark.parametrize("ordering", ORDERINGS)
def test_fp64_jacobi_all_orderings(mesh_mid, ordering):
    m = mesh_mid
    want, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 37)
    with lms.Mesh.from_dict(m, lms.FP64) as g:
        g.reorder(ordering, seed=77)
        assert np.array_equal(g.permutation(), oracle.order(m, ordering, seed=77))
        g.smooth(37)
        got = g.coords()
    assert err(got, want, m) <= TOL64
    assert np.array_equal(got, want)


@pytest.mark.parametrize("ordering", ORDERINGS)
def test_fp32_jacobi_all_orderings(mesh_mid, ordering):
    m = mesh_mid
    want, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 100)
    with lms.Mesh.from_dict(m, lms.FP32) as g:
        g.reorder(ordering, seed=5)
        g.smooth(100)
        got = g.coords()
    assert err(got, want, m) <= TOL32


@pytest.mark.parametrize("precision", [lms.FP64, lms.FP32])
@pytest.mark.parametrize("ordering", ORDERINGS)
def test_coloured_gs_equals_inplace_sweep_in_colour_order(mesh_mid, precision, ordering):
    m = mesh_mid
    p = oracle.order(m, ordering, seed=11)
    want, _, _ = oracle.gs_smooth(m, p, 25)
    with lms.Mesh.from_dict(m, precision) as g:
        g.reorder(ordering, seed=11)
        g.smooth(25, mode=lms.COLORED_GS)
        got = g.coords()
        colour, nc = g.colors()
    c_want, nc_want = oracle.color_greedy(m["row_ptr"], m["col_idx"], m["is_boundary"], p)
    assert nc == nc_want and np.array_equal(colour, c_want)
    if precision == lms.FP64:
        assert err(got, want, m) <= TOL64
        assert np.array_equal(got, want)
    else:
        assert err(got, want, m) <= TOL32


@pytest.mark.parametrize("ordering", ORDERINGS)
def test_relabelled_csr_matches_oracle(mesh_graded, ordering):
    m = mesh_graded
    with lms.Mesh.from_dict(m, lms.FP64) as g:
        g.reorder(ordering, seed=2)
        rp, ci, storage = g.csr()
        p = g.permutation()
    assert np.array_equal(p, oracle.order(m, ordering, seed=2))
    assert np.array_equal(storage, p)
    rp_w, ci_w = oracle.relabel(m["row_ptr"], m["col_idx"], p)
    assert np.array_equal(rp, rp_w) and np.array_equal(ci, ci_w)


def test_coloured_layout_csr(mesh_graded):
    m = mesh_graded
    with lms.Mesh.from_dict(m, lms.FP32) as g:
        g.reorder(lms.RDR)
        g.smooth(1, mode=lms.COLORED_GS)
        rp, ci, storage = g.csr()
        colour, nc = g.colors()
        p = g.permutation()
    seq = oracle.color_sequence(m["is_boundary"], p, colour, nc)
    assert np.array_equal(storage[: len(seq)], seq)
    rp_w, ci_w = oracle.relabel(m["row_ptr"], m["col_idx"], storage)
    assert np.array_equal(rp, rp_w) and np.array_equal(ci, ci_w)


@pytest.mark.parametrize("precision", [lms.FP64, lms.FP32])
def test_quality_matches_oracle(mesh_graded, precision):
    m = mesh_graded
    with lms.Mesh.from_dict(m, precision) as g:
        g.reorder(lms.RDR)
        q0 = g.quality()
        g.smooth(20)
        q1 = g.quality()
        x = g.coords()
    w0 = oracle.mesh_quality(m["n"], m["tri"], m["xy"])
    w1 = oracle.mesh_quality(m["n"], m["tri"], x)
    tol = 1e-13 if precision == lms.FP64 else 1e-6
    assert abs(q0 - w0) <= tol and abs(q1 - w1) <= tol
    assert q1 > q0


@pytest.mark.parametrize("mode", [lms.JACOBI, lms.COLORED_GS])
@pytest.mark.parametrize("precision", [lms.FP64, lms.FP32])
def test_stopping_rule_matches_oracle(mesh_graded, mode, precision):
    m = mesh_graded
    tol = 5e-6
    p = oracle.order(m, oracle.RDR)
    if mode == lms.JACOBI:
        _, k_or, hist = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 200, tri=m["tri"], tol=tol)
    else:
        _, k_or, hist = oracle.gs_smooth(m, p, 200, tol=tol)
    with lms.Mesh.from_dict(m, precision) as g:
        g.reorder(lms.RDR)
        k = g.smooth(200, mode=mode, tol=tol)
        got = g.coords()
        st = g.last_stats()
    assert 1 <= k <= 200
    if precision == lms.FP64:
        near = np.abs(np.diff(hist) - tol) < 1e-9
        assert k == k_or or near[min(k, k_or) - 1]
    # compare positions with the oracle run for the GPU's sweep count
    if mode == lms.JACOBI:
        want, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], k)
    else:
        want, _, _ = oracle.gs_smooth(m, p, k)
    assert err(got, want, m) <= (TOL64 if precision == lms.FP64 else TOL32)
    assert abs(st["q_first"] - hist[0]) < (1e-13 if precision == lms.FP64 else 1e-6)


@pytest.mark.parametrize("precision", [lms.FP64, lms.FP32])
def test_boundary_fixed_and_displacement(mesh_mid, precision):
    m = mesh_mid
    b = m["is_boundary"] == 1
    with lms.Mesh.from_dict(m, precision) as g:
        g.reorder(lms.BFS)
        g.smooth(30)
        x30 = g.coords()
        g.smooth(1)
        x31 = g.coords()
        st = g.last_stats()
        assert g.last_error_stats() == (st["max_disp"], st["ms"])  # the boundary's lms_last_error_stats
    assert np.array_equal(x31[b], m["xy"][b])  # FP32 returns the stored FP64 boundary values
    want = np.sqrt(((x31 - x30) ** 2).sum(axis=1)).max()
    assert abs(st["max_disp"] - want) <= (1e-15 if precision == lms.FP64 else 1e-6) * diag(m) + 1e-12 * want
    assert st["ms"] > 0


@pytest.mark.parametrize("precision", [lms.FP64, lms.FP32])
def test_checkpoint_resume_is_exact(mesh_mid, precision):
    # 40 + 40 sweeps through get/set of FP64 positions equals 80 sweeps (FP64 exactly; FP32 within
    # one normalisation round trip per checkpoint)
    m = mesh_mid
    with lms.Mesh.from_dict(m, precision) as g:
        g.reorder(lms.RDR)
        g.smooth(80)
        full = g.coords()
    with lms.Mesh.from_dict(m, precision) as g:
        g.reorder(lms.RDR)
        g.smooth(40)
        mid = g.coords()
        g.set_coords(mid)
        g.smooth(40)
        resumed = g.coords()
    if precision == lms.FP64:
        assert np.array_equal(full, resumed)
    else:
        assert err(full, resumed, m) <= TOL32


def test_fp32_error_report_after_200_sweeps(mesh_graded):
    m = mesh_graded
    want, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 200)
    with lms.Mesh.from_dict(m, lms.FP32) as g:
        g.reorder(lms.RDR)
        g.smooth(200)
        got = g.coords()
    assert err(got, want, m) <= TOL32


def test_uniform_grid_fixed_point_on_gpu():
    s = 33
    h = 1.0 / 32
    xy = np.array([[i * h, j * h] for j in range(s) for i in range(s)])
    bnd = np.array([1 if (i in (0, s - 1) or j in (0, s - 1)) else 0 for j in range(s) for i in range(s)], np.uint8)
    adj = [set() for _ in range(s * s)]
    for j in range(s):
        for i in range(s):
            v = j * s + i
            for di, dj in ((1, 0), (0, 1), (1, 1)):
                if i + di < s and j + dj < s:
                    u = (j + dj) * s + i + di
                    adj[v].add(u)
                    adj[u].add(v)
    rp = np.cumsum([0] + [len(a) for a in adj]).astype(np.int32)
    ci = np.concatenate([sorted(a) for a in adj]).astype(np.int32)
    for precision in (lms.FP64, lms.FP32):
        with lms.Mesh(rp, ci, xy, bnd, precision=precision) as g:
            g.reorder(lms.RANDOM, seed=1)
            g.smooth(10)
            got = g.coords()
            g.smooth(3, mode=lms.COLORED_GS)
            got2 = g.coords()
        assert np.array_equal(got, xy) and np.array_equal(got2, xy)


def test_api_errors():
    m = meshgen.workload(0, side=10)
    with pytest.raises(lms.LmsError) as e:
        lms.Mesh(m["row_ptr"], m["col_idx"][::-1].copy(), m["xy"], m["is_boundary"], m["tri"])
    assert e.value.status == -2
    with lms.Mesh(m["row_ptr"], m["col_idx"], m["xy"], m["is_boundary"], None) as g:
        with pytest.raises(lms.LmsError) as e:
            g.reorder(lms.RDR)
        assert e.value.status == -4
        with pytest.raises(lms.LmsError) as e:
            g.smooth(5, tol=1e-6)
        assert e.value.status == -4
        with pytest.raises(lms.LmsError) as e:
            g.smooth(5, mode=9)
        assert e.value.status == -1
        g.smooth(0)
        assert np.array_equal(g.coords(), m["xy"])
    bad = m["xy"].copy()
    bad[3, 0] = np.nan
    with pytest.raises(lms.LmsError):
        lms.Mesh(m["row_ptr"], m["col_idx"], bad, m["is_boundary"], m["tri"])


# ------------------------------------------------------------------- batched


def small_batch(count=10):
    sides = [12, 13, 17, 20, 25, 31, 40, 47, 55, 64][:count]
    return [meshgen.generate(s, jitter=0.3, flip_frac=0.10, split_frac=0.05, seed=1000 + i)
            for i, s in enumerate(sides)]


@pytest.mark.parametrize("config", [(lms.KERNEL_STAGED, 256, 1, 256), (lms.KERNEL_STAGED, 128, 1, 512),
                                    (lms.KERNEL_STAGED, 256, 1, 2048), (lms.KERNEL_STAGED, 128, 1, 128),
                                    (lms.KERNEL_DIRECT, 256, 1, 256), (lms.KERNEL_DIRECT, 512, 2, 1024),
                                    (lms.KERNEL_DIRECT, 128, 4, 512), (lms.KERNEL_DIRECT, 256, 8, 4096),
                                    (lms.KERNEL_DIRECT, 128, 4, 128), (lms.KERNEL_DIRECT, 128, 3, 512),
                                    (lms.KERNEL_DIRECT, 256, 5, 256), (lms.KERNEL_DIRECT, 128, 6, 512),
                                    (lms.KERNEL_SELL, 128, 1, 256),
                                    (lms.KERNEL_SELL, 256, 4, 1024), (lms.KERNEL_SELL, 512, 8, 2048),
                                    (lms.KERNEL_SELL, 128, 4, 128),
                                    (lms.KERNEL_PACKED, 128, 4, 512), (lms.KERNEL_PACKED, 256, 2, 256),
                                    (lms.KERNEL_PACKED, 512, 6, 1024), (lms.KERNEL_PACKED, 128, 4, 128)])
def test_batched_fp32_matches_oracle(config):
    meshes = small_batch()
    with lms.Batch(meshes, ordering=lms.RDR) as b:
        b.set_config(*config)
        b.smooth(50)
        for i, m in enumerate(meshes):
            assert np.array_equal(b.permutation(i), oracle.order(m, oracle.RDR))
            want, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 50)
            assert err(b.coords(i), want, m) <= TOL32
        allc = b.all_coords()
        assert np.array_equal(allc[b.offsets[3]:b.offsets[4]], b.coords(3))


@pytest.mark.parametrize("ordering", [lms.ORI, lms.BFS, lms.RBFS])
def test_batched_orderings(ordering):
    meshes = small_batch(5)
    with lms.Batch(meshes, ordering=ordering) as b:
        b.set_config(lms.KERNEL_DIRECT, 128, 4, 512)
        b.smooth(30)
        for i, m in enumerate(meshes):
            assert np.array_equal(b.permutation(i), oracle.order(m, ordering))
            want, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 30)
            assert err(b.coords(i), want, m) <= TOL32


def test_batched_autotune_keeps_positions():
    meshes = small_batch(6)
    with lms.Batch(meshes, ordering=lms.BFS) as b:
        before = b.all_coords()
        cfg = b.autotune()
        assert cfg["kernel"] in (lms.KERNEL_DIRECT, lms.KERNEL_STAGED, lms.KERNEL_SELL, lms.KERNEL_PACKED)
        assert cfg["block"] in (128, 256, 512) and cfg["chunk"] in (1, 2, 3, 4, 5, 6, 8)
        assert np.array_equal(b.all_coords(), before)
        b.smooth(7)
        b.smooth(8)
        got = b.all_coords()
    for i, m in enumerate(meshes):
        want, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 15)
        assert err(got[sum(len(x["xy"]) for x in meshes[:i]):][: m["n"]], want, m) <= TOL32


def test_batched_kernels_agree_bit_for_bit():
    """Every batched kernel reads the same rows in the same entry order and sums them the same way, so the
    FP32 results of the direct, packed, staged and SELL kernels are identical."""
    meshes = small_batch()
    with lms.Batch(meshes, ordering=lms.RDR) as b:
        xy = np.concatenate([m["xy"] for m in meshes])
        ref = None
        for cfg in ((lms.KERNEL_DIRECT, 128, 5, 512), (lms.KERNEL_PACKED, 128, 4, 512),
                    (lms.KERNEL_PACKED, 256, 6, 256), (lms.KERNEL_PACKED, 512, 2, 1024), (lms.KERNEL_STAGED, 128, 1, 256),
                    (lms.KERNEL_SELL, 128, 4, 512)):
            b.set_config(*cfg)
            b.set_all_coords(xy)
            b.smooth(17)
            got = b.all_coords()
            if ref is None:
                ref = got
            assert np.array_equal(got, ref), cfg


def test_sweep_chains_do_not_change_results():
    """lms_batch_set_chains only changes how the sweeps of the meshes are grouped into parallel launch chains."""
    meshes = small_batch()
    xy = np.concatenate([m["xy"] for m in meshes])
    with lms.Batch(meshes, ordering=lms.RDR) as b:
        b.set_config(lms.KERNEL_PACKED, 128, 4, 256)
        ref = None
        for c in (1, 2, 3, 4, 8):
            b.set_chains(c)
            assert b.chains() == c
            b.set_all_coords(xy)
            b.smooth(13)
            got = b.all_coords()
            if ref is None:
                ref = got
            assert np.array_equal(got, ref), c
        for bad in (0, 9, -1):
            with pytest.raises(lms.LmsError):
                b.set_chains(bad)
        before = b.all_coords()
        cfg = b.autotune()
        assert 1 <= cfg["chains"] <= 4
        assert np.array_equal(b.all_coords(), before)  # the chain timing leaves the coordinates in place


def test_packed_kernel_unavailable_for_a_mesh_of_2_22_id_pairs():
    """The packed row word holds a row's offset within its mesh in 22 bits (in id pairs): a batch holding a
    mesh of 2^22 id pairs or more refuses the packed kernel, and the autotuner never picks it; the other
    kernels still run and match the oracle."""
    big = meshgen.generate(1200, jitter=0.3, flip_frac=0.10, split_frac=0.05, seed=77)
    deg = np.diff(big["row_ptr"])
    assert int(((deg + 1) // 2)[big["is_boundary"] == 0].sum()) >= 2 ** 22  # id pairs of its interior rows
    meshes = [big] + small_batch(3)
    with lms.Batch(meshes, ordering=lms.BFS) as b:
        with pytest.raises(lms.LmsError):
            b.set_config(lms.KERNEL_PACKED, 128, 4, 512)
        b.set_config(lms.KERNEL_DIRECT, 128, 5, 512)
        b.smooth(5)
        for i, m in enumerate(meshes):
            want, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 5)
            assert err(b.coords(i), want, m) <= TOL32
        assert b.autotune()["kernel"] != lms.KERNEL_PACKED


def wheel_mesh(spokes=80):
    """A hub joined to a ring of `spokes` interior vertices inside a fixed outer ring (a fan of triangles
    around the hub, a triangulated annulus around the fan): the hub's row has `spokes` entries."""
    t = 2 * np.pi * np.arange(spokes) / spokes
    xy = np.concatenate([[[0.05, -0.03]], 0.5 * np.c_[np.cos(t), np.sin(t)], np.c_[np.cos(t + 0.1), np.sin(t + 0.1)]])
    inner, outer = 1 + np.arange(spokes), 1 + spokes + np.arange(spokes)
    nxt = np.roll(np.arange(spokes), -1)
    tri = np.concatenate([np.c_[np.zeros(spokes, int), inner, inner[nxt]], np.c_[inner, outer, outer[nxt]],
                          np.c_[inner, outer[nxt], inner[nxt]]]).astype(np.int32)
    n = 1 + 2 * spokes
    adj = [set() for _ in range(n)]
    for a, b, c in tri:
        for u, v in ((a, b), (b, c), (c, a)):
            adj[u].add(int(v))
            adj[v].add(int(u))
    row_ptr = np.zeros(n + 1, np.int32)
    row_ptr[1:] = np.cumsum([len(r) for r in adj])
    col_idx = np.concatenate([sorted(r) for r in adj]).astype(np.int32)
    is_boundary = np.zeros(n, np.int8)
    is_boundary[outer] = 1
    return dict(n=n, row_ptr=row_ptr, col_idx=col_idx, xy=xy.astype(np.float64), is_boundary=is_boundary, tri=tri)


@pytest.mark.parametrize("ordering", [lms.ORI, lms.RDR])
def test_fp32_jacobi_with_a_row_of_more_than_63_entries(ordering):
    """The packed single-mesh Jacobi holds a row's length in 6 bits: a mesh with a longer row runs on the
    row-offset kernel instead, with the same results against the oracle, stop rule included."""
    m = wheel_mesh(80)
    assert np.diff(m["row_ptr"]).max() == 80
    want, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 40)
    with lms.Mesh.from_dict(m, lms.FP32) as g:
        g.reorder(ordering, seed=3)
        g.smooth(40)
        assert err(g.coords(), want, m) <= TOL32
    _, want_done, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 500, tri=m["tri"],
                                    tol=1e-4)
    assert 0 < want_done < 500
    with lms.Mesh.from_dict(m, lms.FP32) as g:
        g.reorder(ordering, seed=3)
        assert abs(g.smooth(500, lms.JACOBI, 1e-4) - want_done) <= 1


def test_fp32_jacobi_across_packed_blocks_and_layouts(mesh_mid):
    """Packed row words are relative to blocks of 4,096 storage positions (mesh_mid spans three, the last
    ragged); re-laying the mesh out rebuilds them, and every layout gives the oracle's result."""
    m = mesh_mid
    assert m["n"] > 2 * 4096
    want, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 30)
    with lms.Mesh.from_dict(m, lms.FP32) as g:
        for ordering in (lms.RDR, lms.RANDOM, lms.ORI, lms.BRDR):
            g.set_coords(m["xy"])
            g.reorder(ordering, seed=11)
            g.smooth(30)
            assert err(g.coords(), want, m) <= TOL32, ordering


def test_batched_config_rejects_unsupported_chunks():
    with lms.Batch(small_batch(2), ordering=lms.ORI) as b:
        for chunk in (0, 7, 9, -1):
            with pytest.raises(lms.LmsError):
                b.set_config(lms.KERNEL_DIRECT, 128, chunk, 512)
        for chunk in (1, 3, 5, 8):
            with pytest.raises(lms.LmsError):
                b.set_config(lms.KERNEL_PACKED, 128, chunk, 512)
        with pytest.raises(lms.LmsError):
            b.set_config(lms.KERNEL_SELL, 128, 3, 512)


def test_batched_set_coords_round_trip():
    meshes = small_batch(4)
    with lms.Batch(meshes, ordering=lms.RANDOM, seed=3) as b:
        xy = np.concatenate([m["xy"] for m in meshes])
        b.smooth(20)
        b.set_all_coords(xy)
        b.smooth(20)
        got = b.all_coords()
    for i, m in enumerate(meshes):
        want, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 20)
        o = sum(x["n"] for x in meshes[:i])
        assert err(got[o:o + m["n"]], want, m) <= TOL32


@pytest.mark.parametrize("launch", [(lms.KERNEL_DIRECT, 128, 0), (lms.KERNEL_STAGED, 128, 64),
                                    (lms.KERNEL_STAGED, 256, 256), (lms.KERNEL_STAGED, 256, 1024),
                                    (lms.KERNEL_STAGED, 128, 1024)])
def test_sweep_kernels_agree_with_oracle(mesh_mid, launch):
    # every launch configuration gives the oracle's result: FP64 bit-exact, FP32 within tolerance
    m = mesh_mid
    kernel, block, tile = launch
    p = oracle.order(m, oracle.RDR)
    want_j, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 21)
    want_g, _, _ = oracle.gs_smooth(m, p, 9)
    for precision in (lms.FP64, lms.FP32):
        with lms.Mesh.from_dict(m, precision) as g:
            g.reorder(lms.RDR)
            g.set_launch(kernel, block, max(tile, 32))
            g.smooth(21)
            got_j = g.coords()
            g.set_coords(m["xy"])
            g.smooth(9, mode=lms.COLORED_GS)
            got_g = g.coords()
            st = g.last_stats()
        if precision == lms.FP64:
            assert np.array_equal(got_j, want_j) and np.array_equal(got_g, want_g)
        else:
            assert err(got_j, want_j, m) <= TOL32 and err(got_g, want_g, m) <= TOL32
        assert st["max_disp"] > 0


def test_batched_rejects_non_finite_coordinates_on_next_read():
    meshes = small_batch(3)
    with lms.Batch(meshes, ordering=lms.ORI) as b:
        xy = np.concatenate([m["xy"] for m in meshes])
        xy[5, 1] = np.inf
        b.set_all_coords(xy)
        with pytest.raises(lms.LmsError) as e:
            b.all_coords()
        assert e.value.status == -1
        xy[5, 1] = 0.5
        b.set_all_coords(xy)
        b.smooth(3)
        assert np.isfinite(b.all_coords()).all()


@pytest.mark.parametrize("groups", [1, 3, 10])
def test_batched_run_equals_set_smooth_get(groups):
    meshes = small_batch(10)
    xy = np.concatenate([m["xy"] for m in meshes])
    with lms.Batch(meshes, ordering=lms.RDR) as b:
        b.set_config(lms.KERNEL_DIRECT, 128, 4, 256)
        b.set_all_coords(xy)
        b.smooth(17)
        want = b.all_coords()
        b.smooth(3)  # move away, then start over from xy
        got = b.run(xy, 17, groups=groups)
        assert np.array_equal(got, want)
        assert np.array_equal(b.all_coords(), want)  # the batch holds the result afterwards
        assert np.array_equal(b.run(xy, 0, groups=groups), b.run(xy, 0, groups=1))
    for i, m in enumerate(meshes):
        o = sum(x["n"] for x in meshes[:i])
        w, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 17)
        assert err(got[o:o + m["n"]], w, m) <= TOL32


def test_batched_run_rejects_bad_input():
    meshes = small_batch(3)
    xy = np.concatenate([m["xy"] for m in meshes])
    with lms.Batch(meshes, ordering=lms.BFS) as b:
        with pytest.raises(lms.LmsError):
            b.run(xy, 5, groups=4)  # more groups than meshes
        bad = xy.copy()
        bad[7, 1] = np.nan
        with pytest.raises(lms.LmsError):
            b.run(bad, 5, groups=2)
        assert np.isfinite(b.run(xy, 5, groups=2)).all()
