"""C ABI of liblms without a GPU: the library loads, exports every entry point
that include/lms.h declares, and its host logic (validation, the four orderings
and the colouring) matches the FP64 oracle bit for bit."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import meshgen
import oracle
import paper_1606_00803_gb300 as lms
from conftest import ROOT


def declared_entry_points():
    text = open(os.path.join(ROOT, "include", "lms.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lms_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = lms._lib()
    names = declared_entry_points()
    assert len(names) >= 30
    nm = subprocess.run(["nm", "-D", "--defined-only", lms.library_path()], stdout=subprocess.PIPE, check=True)
    exported = set(re.findall(r" T (lms_[a-z0-9_]+)", nm.stdout.decode()))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)


def test_error_strings():
    lib = lms._lib()
    for code in [0, -1, -2, -3, -4, -5, -6, -7, -8, -99]:
        s = lib.lms_error_string(code).decode()
        assert s and isinstance(s, str)


def _tiny():
    return meshgen.workload(1, side=9)


def test_validate_accepts_generated_meshes():
    for side in (5, 16, 33):
        m = meshgen.workload(1, side=side)
        assert lms.validate(m["row_ptr"], m["col_idx"], m["is_boundary"], m["tri"]) == 0


def test_validate_rejects_bad_meshes():
    m = _tiny()
    rp, ci, b, t = m["row_ptr"].copy(), m["col_idx"].copy(), m["is_boundary"].copy(), m["tri"].copy()
    v = int(np.nonzero(b == 0)[0][0])
    # out-of-range id
    c2 = ci.copy(); c2[0] = len(rp) + 5
    assert lms.validate(rp, c2, b, t) == -2
    # self-loop
    c2 = ci.copy(); c2[rp[v]] = v
    assert lms.validate(rp, c2, b, t) == -2
    # duplicate entry in a row
    c2 = ci.copy(); c2[rp[v] + 1] = c2[rp[v]]
    assert lms.validate(rp, c2, b, t) == -2
    # asymmetric: replace one neighbour by a non-adjacent vertex
    c2 = ci.copy()
    row = set(ci[rp[v]:rp[v + 1]].tolist()) | {v}
    far = next(u for u in range(len(rp) - 1) if u not in row)
    c2[rp[v]] = far
    assert lms.validate(rp, c2, b, t) == -2
    # non-monotone offsets
    r2 = rp.copy(); r2[3] = r2[4] + 1
    assert lms.validate(r2, ci, b, t) == -2
    # isolated interior vertex: a vertex with an empty row that is not on the boundary
    n = len(rp) - 1
    r3 = np.concatenate([rp, [rp[-1]]]).astype(np.int32)
    b3 = np.concatenate([b, [0]]).astype(np.uint8)
    assert lms.validate(r3, ci, b3, t) == -3
    b3[-1] = 1   # a fixed vertex may be isolated
    assert lms.validate(r3, ci, b3, t) == 0
    # triangle with a repeated or out-of-range corner
    t2 = t.copy(); t2[0, 1] = t2[0, 0]
    assert lms.validate(rp, ci, b, t2) == -1
    t2 = t.copy(); t2[0, 1] = n + 3
    assert lms.validate(rp, ci, b, t2) == -1


@pytest.mark.parametrize("side", [6, 20, 57, 130])
@pytest.mark.parametrize("ordering", [lms.ORI, lms.RANDOM, lms.BFS, lms.RDR, lms.RBFS, lms.BRDR])
def test_host_ordering_matches_oracle(side, ordering):
    m = meshgen.workload(1, side=side)
    q = oracle.vertex_quality(m["n"], m["tri"], m["xy"])
    want = oracle.order(m, ordering, seed=1234 + side, q_v=q)
    got = lms.order_host(m["row_ptr"], m["col_idx"], m["is_boundary"], ordering, seed=1234 + side, q_v=q)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("ordering", [lms.RDR, lms.BRDR])
def test_host_rdr_on_several_threads_matches_oracle(ordering):
    """From 131,072 vertices up the host RDR sorts the keys, ranks the vertices and orders the rows on
    several threads; the walk is the same."""
    m = meshgen.workload(1, side=400)
    assert m["n"] > 2 * 65536
    q = oracle.vertex_quality(m["n"], m["tri"], m["xy"])
    assert np.array_equal(lms.order_host(m["row_ptr"], m["col_idx"], m["is_boundary"], ordering, q_v=q),
                          oracle.order(m, ordering, q_v=q))


def test_host_rdr_with_negative_keys_matches_oracle():
    """Keys below zero take the comparison sort instead of the radix sort of the bit patterns."""
    m = meshgen.workload(1, side=60)
    q = np.random.default_rng(4).uniform(-1.0, 1.0, m["n"])
    q[::7] = -0.0
    assert np.array_equal(lms.order_host(m["row_ptr"], m["col_idx"], m["is_boundary"], lms.RDR, q_v=q),
                          oracle.order_rdr(m["row_ptr"], m["col_idx"], m["is_boundary"], q))


def test_host_rdr_handles_ties_and_unreached_vertices():
    import json
    from conftest import GOLDEN
    g = json.load(open(os.path.join(GOLDEN, "rdr_small.json")))
    for case in g["cases"]:
        got = lms.order_host(case["row_ptr"], case["col_idx"], case["is_boundary"], lms.RDR, q_v=case["q_v"])
        assert got.tolist() == case["rdr_new_to_old"]
    # all keys equal: ties fall back to vertex id in both implementations
    m = meshgen.workload(1, side=15)
    q = np.full(m["n"], 0.5)
    assert np.array_equal(lms.order_host(m["row_ptr"], m["col_idx"], m["is_boundary"], lms.RDR, q_v=q),
                          oracle.order_rdr(m["row_ptr"], m["col_idx"], m["is_boundary"], q))


@pytest.mark.parametrize("ordering", [lms.ORI, lms.RANDOM, lms.BFS, lms.RDR])
def test_host_colouring_matches_oracle(ordering):
    m = meshgen.workload(1, side=45)
    p = oracle.order(m, ordering, seed=3)
    c_want, n_want = oracle.color_greedy(m["row_ptr"], m["col_idx"], m["is_boundary"], p)
    c_got, n_got = lms.color_host(m["row_ptr"], m["col_idx"], m["is_boundary"], p)
    assert n_got == n_want and np.array_equal(c_got, c_want)


def test_host_orderings_on_a_disconnected_mesh():
    a, b = meshgen.workload(1, side=7), meshgen.workload(0, side=5)
    n = a["n"] + b["n"]
    rp = np.concatenate([a["row_ptr"], b["row_ptr"][1:] + a["row_ptr"][-1]]).astype(np.int32)
    ci = np.concatenate([a["col_idx"], b["col_idx"] + a["n"]]).astype(np.int32)
    bnd = np.concatenate([a["is_boundary"], b["is_boundary"]])
    tri = np.concatenate([a["tri"], b["tri"] + a["n"]])
    xy = np.concatenate([a["xy"], b["xy"] + 3.0])
    m = dict(n=n, row_ptr=rp, col_idx=ci, is_boundary=bnd, tri=tri, xy=xy)
    q = oracle.vertex_quality(n, tri, xy)
    for ordering in (lms.BFS, lms.RDR, lms.RANDOM, lms.BRDR):
        assert np.array_equal(lms.order_host(rp, ci, bnd, ordering, seed=9, q_v=q), oracle.order(m, ordering, 9, q))


def test_host_entry_points_reject_bad_arguments():
    m = _tiny()
    with pytest.raises(lms.LmsError):
        lms.order_host(m["row_ptr"], m["col_idx"], m["is_boundary"], 7)
    with pytest.raises(lms.LmsError):
        lms.order_host(m["row_ptr"], m["col_idx"], m["is_boundary"], lms.RDR, q_v=None)


QS = (0.0, 0.01, 0.5, 0.75, 0.9, 0.99, 1.0)


@pytest.mark.parametrize("ordering", [lms.ORI, lms.RANDOM, lms.BFS, lms.RDR, lms.RBFS])
@pytest.mark.parametrize("with_vertex", [True, False])
@pytest.mark.parametrize("measure", [lms.REUSE_DISTINCT, lms.REUSE_ACCESSES])
def test_reuse_profile_matches_oracle(ordering, with_vertex, measure):
    m = meshgen.workload(1, side=37)
    p = oracle.order(m, ordering, seed=21)
    t = oracle.access_trace(m["row_ptr"], m["col_idx"], m["is_boundary"], p, with_vertex)
    d = oracle.reuse_distances(t, m["n"], measure)
    r = lms.reuse_profile(m["row_ptr"], m["col_idx"], m["is_boundary"], p, with_vertex, measure, QS)
    assert [r["quantiles"][x] for x in QS] == [oracle.quantile(d, x) for x in QS]
    assert r["accesses"] == len(t) and r["reuses"] == len(d)
    assert r["mean"] == int(d.sum()) / len(d)
    hist = np.zeros(33, np.int64)
    np.add.at(hist, [0 if x == 0 else int(x).bit_length() for x in d.tolist()], 1)
    assert np.array_equal(r["hist"], hist)


def test_reuse_profile_identity_default_and_edge_cases():
    m = meshgen.workload(1, side=12)
    a = lms.reuse_profile(m["row_ptr"], m["col_idx"], m["is_boundary"])
    b = lms.reuse_profile(m["row_ptr"], m["col_idx"], m["is_boundary"], np.arange(m["n"]))
    assert a["quantiles"] == b["quantiles"] and a["mean"] == b["mean"]
    # every vertex on the boundary: empty trace, no reuses
    r = lms.reuse_profile(m["row_ptr"], m["col_idx"], np.ones(m["n"], np.uint8))
    assert r["accesses"] == 0 and r["reuses"] == 0 and set(r["quantiles"].values()) == {-1}
    # one interior vertex: its row has no repeated element, the vertex itself is not in its row
    r = lms.reuse_profile(m["row_ptr"], m["col_idx"], (np.arange(m["n"]) != 13).astype(np.uint8))
    assert r["reuses"] == 0


def test_reuse_profile_rejects_bad_arguments():
    m = meshgen.workload(1, side=10)
    args = (m["row_ptr"], m["col_idx"], m["is_boundary"])
    bad_perm = np.arange(m["n"])
    bad_perm[3] = 4
    for kw in ({"new_to_old": bad_perm}, {"measure": 2}, {"quantiles": (1.5,)}, {"quantiles": (-0.1,)}):
        with pytest.raises(lms.LmsError) as e:
            lms.reuse_profile(*args, **kw)
        assert e.value.status == -1
    ci = m["col_idx"].copy()
    ci[0] = m["n"]
    with pytest.raises(lms.LmsError) as e:
        lms.reuse_profile(m["row_ptr"], ci, m["is_boundary"])
    assert e.value.status == -2


def test_host_block_rdr_on_many_blocks_matches_oracle():
    # 1024 x 1024 mesh: 282 blocks, spread over host threads
    m = meshgen.workload(1)
    q = oracle.vertex_quality(m["n"], m["tri"], m["xy"])
    got = lms.order_host(m["row_ptr"], m["col_idx"], m["is_boundary"], lms.BRDR, q_v=q)
    assert np.array_equal(got, oracle.order_brdr(m["row_ptr"], m["col_idx"], m["is_boundary"], q, block=lms.BRDR_BLOCK))


def test_timeout_selftest_rejects_bad_bounds_without_device_work():
    assert lms.selftest_timeout(0) == -1
    assert lms.selftest_timeout(3_000_000) == -1


def test_release_build_reports_no_bounds_checks():
    enabled, violations = lms.debug_checks()
    assert enabled is False and violations == 0


def test_binding_declares_a_signature_for_every_entry_point():
    # an entry point without argtypes would pass 64-bit pointers as 32-bit ints
    missing = [n for n in declared_entry_points() if n not in lms._SIGS]
    assert not missing, missing


@pytest.mark.parametrize("ordering", [oracle.ORI, oracle.BFS, oracle.RDR, oracle.RANDOM])
def test_block_order_host_equals_oracle(ordering):
    # library (stamp-array tile colouring, counting sorts) against the oracle's plain loops
    for m in (meshgen.workload(1, side=33), meshgen.workload(2, side=21)):
        p = oracle.order(m, ordering, seed=9)
        colour, nc = oracle.color_greedy(m["row_ptr"], m["col_idx"], m["is_boundary"], p)
        for tile in (1, 2, 5, 128, 700, m["n"], m["n"] + 3):
            want, tcw, ntw = oracle.block_sequence(m["row_ptr"], m["col_idx"], m["is_boundary"], p, colour, nc, tile)
            got, tcg, ntg = lms.block_order(m["row_ptr"], m["col_idx"], m["is_boundary"], p, tile)
            assert np.array_equal(got, want) and np.array_equal(tcg, tcw) and ntg == ntw


def test_block_order_rejects_bad_arguments():
    m = meshgen.workload(0)
    p = np.arange(m["n"], dtype=np.int32)
    with pytest.raises(ValueError):
        lms.block_order(m["row_ptr"], m["col_idx"], m["is_boundary"], p, 0)
    out = np.empty(m["n"], np.int32)
    nt, k = ctypes.c_int32(), ctypes.c_int32()
    rc = lms._lib().lms_block_order(m["n"], m["row_ptr"].ctypes.data, m["col_idx"].ctypes.data,
                                    m["is_boundary"].ctypes.data, p.ctypes.data, -4, out.ctypes.data,
                                    ctypes.byref(nt), out.ctypes.data, ctypes.byref(k))
    assert rc == -1  # LMS_ERR_ARG
    rc = lms._lib().lms_block_order(m["n"], None, m["col_idx"].ctypes.data, m["is_boundary"].ctypes.data,
                                    p.ctypes.data, 8, out.ctypes.data, ctypes.byref(nt), out.ctypes.data,
                                    ctypes.byref(k))
    assert rc == -1


@pytest.mark.parametrize("ordering", [oracle.ORI, oracle.BFS, oracle.RDR, oracle.RANDOM])
def test_block_gs_tables_walk_in_oracle_order(ordering):
    # the device sweep's tables walked in launch order visit the oracle's block order
    for m in (meshgen.workload(1, side=37), meshgen.workload(2, side=23), meshgen.workload(0)):
        p = oracle.order(m, ordering, seed=4)
        colour, nc = oracle.color_greedy(m["row_ptr"], m["col_idx"], m["is_boundary"], p)
        for tile in (1, 7, 128, 333, m["n"] + 2):
            want, _, nt = oracle.block_sequence(m["row_ptr"], m["col_idx"], m["is_boundary"], p, colour, nc, tile)
            got, launches = lms.block_walk(m["row_ptr"], m["col_idx"], m["is_boundary"], p, tile)
            assert np.array_equal(got, want)
            assert 1 <= launches <= nt


def test_handle_setters_reject_null_and_bad_values_without_device_work():
    L = lms._lib()
    t = ctypes.c_int32()
    assert L.lms_set_fp64_arith(None, 0) == -1
    assert L.lms_set_block_tile(None, 64) == -1
    assert L.lms_get_block_tile(None, ctypes.byref(t)) == -1
    assert L.lms_set_inplace_split(None, 1) == -1
    assert L.lms_set_launch(None, 0, 128, 512) == -1
    assert L.lms_smooth(None, 1, 0, -1.0, None) == -1
    # the integer-pipe self-tests check their arguments before any device work
    assert L.lms_selftest_add64(-1, None, None, None) == -1
    assert L.lms_selftest_divint64(-1, None, None, None) == -1
    d = np.array([0], np.int32)
    s = np.zeros(1)
    assert L.lms_selftest_divint64(1, s.ctypes.data, d.ctypes.data, s.ctypes.data) == -1  # divisor 0
    assert L.lms_selftest_add64(0, None, None, None) == 0  # nothing to do


def test_plain_c_program_uses_the_library(tmp_path):
    # the header is plain C99 and a C program can link liblms.so and call its host entry points
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text(r"""
#include <stdio.h>
#include <string.h>
#include "lms.h"
int main(void) {
    /* path 0-1-2-3 with fixed ends: validate, order, colour */
    int32_t rp[5] = {0, 1, 3, 5, 6}, ci[6] = {1, 0, 2, 1, 3, 2}, perm[4], colour[4], nc = 0;
    uint8_t bnd[4] = {1, 0, 0, 1};
    if (lms_validate(4, rp, ci, bnd, 0, NULL) != LMS_OK) return 1;
    if (lms_order_host(4, rp, ci, bnd, NULL, LMS_BFS, 0, perm) != LMS_OK) return 2;
    if (lms_color_host(4, rp, ci, bnd, perm, colour, &nc) != LMS_OK || nc != 2) return 3;
    if (strlen(lms_error_string(LMS_ERR_CSR)) == 0) return 4;
    printf("%d %d %d %d\n", perm[0], perm[1], perm[2], perm[3]);
    return 0;
}
""")
    lib = lms.library_path()
    exe = tmp_path / "use"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(exe), lib, "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    out = subprocess.run([str(exe)], stdout=subprocess.PIPE, check=True).stdout.decode().split()
    assert out == ["0", "1", "2", "3"]


def test_partition_meshes_covers_and_balances():
    """lms_partition_meshes: every mesh on one rank, loads add up, the spread is at most the largest mesh,
    and on tiny inputs the makespan is within Graham's LPT bound (4/3 - 1/(3r)) of the optimum found by
    brute force."""
    import itertools
    rng = np.random.default_rng(5)
    for trial in range(60):
        k = int(rng.integers(1, 9))
        ranks = int(rng.integers(1, 5))
        sizes = rng.integers(1, 50, size=k).astype(np.int32)
        rank_of, load = lms.partition_meshes(sizes, ranks)
        assert rank_of.min() >= 0 and rank_of.max() < ranks
        assert [int(sizes[rank_of == r].sum()) for r in range(ranks)] == list(load)
        assert load.max() - load.min() <= sizes.max()
        best = min(max(sum(int(sizes[i]) for i in range(k) if a[i] == r) for r in range(ranks))
                   for a in itertools.product(range(ranks), repeat=k))
        assert load.max() <= (4 / 3 - 1 / (3 * ranks)) * best + 1e-9
        again, _ = lms.partition_meshes(sizes, ranks)
        assert np.array_equal(again, rank_of)
    # a large batch like the benchmark's: 512 sizes, 8 ranks
    sizes = rng.integers(1000, 200000, size=512).astype(np.int32)
    rank_of, load = lms.partition_meshes(sizes, 8)
    assert load.max() - load.min() <= sizes.max() and load.sum() == sizes.sum()
    for bad in (([], 2), ([3, 0], 2), ([3, 4], 0)):
        with pytest.raises(lms.LmsError):
            lms.partition_meshes(np.asarray(bad[0], np.int32), bad[1])


def test_noalloc_rejects_overlapping_buffers_before_device_work():
    """lms_jacobi_noalloc checks its arguments before any CUDA call: position buffers that share a byte are
    rejected (the addresses below are never dereferenced)."""
    fn = lms._lib().lms_jacobi_noalloc
    n = 100
    base = 0x10000000
    for other in (base, base + 8, base + 16 * n - 8, base - 16 * n + 8):
        assert fn(n, 1, 1, 1, base, other, 1, None) == -1
        assert "overlap" in lms._lib().lms_last_error_detail().decode()
    assert fn(0, 1, 1, 1, base, base + 16 * n, 1, None) == -1
    assert fn(n, 1, 1, 1, base, base + 16 * n, -1, None) == -1
