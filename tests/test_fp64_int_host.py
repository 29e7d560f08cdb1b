"""The FP64 sweep's integer-pipe arithmetic (add_rn_int and div_rn_int in lms_fp64_int.cuh), compiled for
the host from the same header, against IEEE 754 binary64 addition and division rounded to nearest (the
host FPU through numpy); and the per-sweep quality's root of a ratio (root_of_ratio: FP32 seed, two FP64
Newton steps) against sqrt(lo / hi).

The cases are chosen so that a slip anywhere in the routines fails one of them: ties at every exponent
distance around the 53-bit boundary (round-half-even), every alignment the integer path takes and the
wider gaps it hands back, cancellations of every depth (renormalisation and its exponent), carries into
the next binade, opposite signs of equal magnitude (+0), the operands handed to the FPU (zeros,
subnormals, the top binade, subnormal results); for the division every divisor 1..64, exact quotients,
remainders just above zero and just below the divisor, and quotients that underflow."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1606_00803_gb300", "csrc")

HARNESS = r"""
#include "lms_fp64_int.cuh"
extern "C" void add_batch(long n, const double* a, const double* b, double* s) {
    for (long i = 0; i < n; ++i) s[i] = lms::dev::add_rn_int(a[i], b[i]);
}
extern "C" void plus_zero_batch(long n, const double* a, double* s) {
    for (long i = 0; i < n; ++i) s[i] = lms::dev::plus_zero(a[i]);
}
// q[i] = s[i] / d[i] by div_rn_int; declined[i] = 1 where it hands the division back (q[i] untouched)
extern "C" void root_batch(long n, const double* lo, const double* hi, double* r) {
    for (long i = 0; i < n; ++i) r[i] = lms::dev::root_of_ratio(lo[i], hi[i]);
}
extern "C" void div_batch(long n, const double* s, const int* d, double* q, unsigned char* declined) {
    uint32_t magic[130] = {0};
    for (int i = 1; i <= 64; ++i) lms::dev::div_magic(i, magic + 2 * i, magic + 2 * i + 1);
    for (long i = 0; i < n; ++i) declined[i] = !lms::dev::div_rn_int(s[i], d[i], magic, q + i);
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("fp64add")
    src, so = d / "h.cpp", d / "libh.so"
    src.write_text(HARNESS)
    subprocess.run([cxx, "-O2", "-ffp-contract=off", "-shared", "-fPIC", "-I", CSRC, str(src), "-o", str(so)],
                   check=True)
    L = ctypes.CDLL(str(so))
    P = ctypes.c_void_p
    L.add_batch.argtypes = [ctypes.c_long, P, P, P]
    L.plus_zero_batch.argtypes = [ctypes.c_long, P, P]
    L.div_batch.argtypes = [ctypes.c_long, P, P, P, P]
    L.root_batch.argtypes = [ctypes.c_long, P, P, P]
    return L


def emul_add(L, a, b):
    a = np.ascontiguousarray(a, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    s = np.empty_like(a)
    L.add_batch(len(a), a.ctypes.data, b.ctypes.data, s.ctypes.data)
    return s


def from_parts(sign, exp, frac):
    bits = (sign.astype(np.uint64) << np.uint64(63)) | (exp.astype(np.uint64) << np.uint64(52)) | frac.astype(np.uint64)
    return bits.view(np.float64)


def assert_bitwise(L, a, b):
    got = emul_add(L, a, b).view(np.uint64)
    want = (a + b).view(np.uint64)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, "first mismatch: %r + %r -> %r, IEEE %r" % (
        a[bad[0]], b[bad[0]], got[bad[0]:bad[0] + 1].view(np.float64)[0], (a + b)[bad[0]])


def test_random_operands_every_alignment(lib):
    rng = np.random.default_rng(1)
    n = 400_000
    ea = rng.integers(900, 1150, n)
    eb = np.clip(ea + rng.integers(-70, 71, n), 1, 2045)
    a = from_parts(rng.integers(0, 2, n), ea, rng.integers(0, 1 << 52, n, dtype=np.uint64))
    b = from_parts(rng.integers(0, 2, n), eb, rng.integers(0, 1 << 52, n, dtype=np.uint64))
    assert_bitwise(lib, a, b)


def test_carries_into_the_next_binade_with_lost_bits(lib):
    # both significands in [1.5, 2): same-sign sums carry, and with 8..60 bits of alignment the bit shifted
    # out by the renormalisation meets the sticky bit
    rng = np.random.default_rng(5)
    n = 400_000
    half = np.uint64(1 << 51)
    ea = rng.integers(1000, 1050, n)
    a = from_parts(np.zeros(n, np.int64), ea, half | rng.integers(0, 1 << 51, n, dtype=np.uint64))
    b = from_parts(np.zeros(n, np.int64), ea - rng.integers(8, 61, n), half | rng.integers(0, 1 << 51, n, dtype=np.uint64))
    assert_bitwise(lib, a, b)
    assert_bitwise(lib, -a, -b)
    # a within 2^-22 of the next power of two and 11..20 bits of alignment: every sum carries, and the
    # sticky bit lands under the renormalisation shift
    top = np.uint64((1 << 52) - 1) - rng.integers(0, 1 << 30, n, dtype=np.uint64)
    a2 = from_parts(np.zeros(n, np.int64), ea, top)
    b2 = from_parts(np.zeros(n, np.int64), ea - rng.integers(11, 21, n), rng.integers(0, 1 << 52, n, dtype=np.uint64))
    assert_bitwise(lib, a2, b2)


def test_sparse_significands_hit_ties_and_exact_sums(lib):
    # few significant bits: sums are often exact or exactly halfway between two doubles
    rng = np.random.default_rng(2)
    n = 400_000
    top = rng.integers(0, 16, n, dtype=np.uint64) << np.uint64(48)
    low = rng.choice(np.array([0, 1, (1 << 52) - 1, 1 << 20], dtype=np.uint64), n)
    ea = rng.integers(1000, 1050, n)
    a = from_parts(rng.integers(0, 2, n), ea, top | low)
    top2 = rng.integers(0, 16, n, dtype=np.uint64) << np.uint64(48)
    b = from_parts(rng.integers(0, 2, n), np.clip(ea - rng.integers(0, 66, n), 1, 2045), top2)
    assert_bitwise(lib, a, b)


@pytest.mark.parametrize("a,b,want", [
    (1.0, 2.0 ** -53, 1.0),                                  # tie, even neighbour below
    (1.0 + 2.0 ** -52, 2.0 ** -53, 1.0 + 2.0 ** -51),        # tie, odd: up to even
    (1.0, 2.0 ** -53 + 2.0 ** -105, 1.0 + 2.0 ** -52),       # just above the tie (sticky decides)
    (1.0, -(2.0 ** -53), 1.0 - 2.0 ** -53),                  # borrow into the binade below: exact
    (1.0, -(2.0 ** -54), 1.0),                               # tie in the binade below: even is 1.0
    (1.0, -(2.0 ** -53) - 2.0 ** -106, 1.0 - 2.0 ** -53),    # below the binade, sticky jammed
    (0.75, 0.75, 1.5),                                       # carry into the next binade
    (1.5, -1.5, 0.0),                                        # exact cancellation: +0
    (-1.5, 1.5, 0.0),
    (2.0 ** 1022, 2.0 ** 1022, 2.0 ** 1023),                 # into the top binade
])
def test_hand_cases(lib, a, b, want):
    got = emul_add(lib, np.array([a]), np.array([b]))[0]
    assert got == want and np.signbit(got) == np.signbit(want)
    assert got == a + b


def test_cancellation_of_every_depth(lib):
    rng = np.random.default_rng(3)
    n = 300_000
    a = rng.uniform(-4, 4, n)
    bits = a.view(np.uint64).copy()
    # neighbours of -a that differ in the last 0..52 bits
    k = rng.integers(0, 53, n).astype(np.uint64)
    delta = rng.integers(0, 1 << 62, n, dtype=np.uint64) & ((np.uint64(1) << k) - np.uint64(1))
    b = ((bits ^ np.uint64(1 << 63)) ^ delta).view(np.float64)
    assert_bitwise(lib, a, b)
    b2 = -a * (1 + rng.uniform(-1e-3, 1e-3, n))
    assert_bitwise(lib, a, b2)


def test_fpu_hand_offs_and_extremes(lib):
    tiny = np.finfo(np.float64).tiny
    big = np.finfo(np.float64).max
    vals = np.array([0.0, -0.0, tiny, -tiny, tiny / 3, 5e-324, -5e-324, 1.5 * tiny, -1.25 * tiny,
                     big, -big, big / 2, 2.0 ** 1023, 2.0 ** 1022 * 1.75, 1.0, -1.0, 0.3, -2.5e-300,
                     3.0 * 2.0 ** -1021, -(2.0 ** -1021)])
    a, b = np.meshgrid(vals, vals)
    with np.errstate(over="ignore"):
        assert_bitwise(lib, a.ravel(), b.ravel())


def test_coordinate_like_sums(lib):
    # the sweep's own pattern: running sums of 3..12 positions in a box straddling the origin
    rng = np.random.default_rng(4)
    x = rng.uniform(-0.5, 0.5, (200_000, 12))
    x[rng.random(x.shape) < 0.02] = 0.0
    s_emul = np.zeros(len(x))
    s_ieee = np.zeros(len(x))
    for j in range(12):
        s_emul = emul_add(lib, s_emul, x[:, j])
        s_ieee = s_ieee + x[:, j]
        assert np.array_equal(s_emul.view(np.uint64), s_ieee.view(np.uint64))


def test_plus_zero_is_adding_to_zero(lib):
    x = np.array([0.0, -0.0, 1.0, -1.0, 5e-324, -5e-324, np.finfo(np.float64).max, -3.25])
    out = np.empty_like(x)
    lib.plus_zero_batch(len(x), x.ctypes.data, out.ctypes.data)
    assert np.array_equal(out.view(np.uint64), (0.0 + x).view(np.uint64))


def emul_div(L, s, d):
    s = np.ascontiguousarray(s, np.float64)
    d = np.ascontiguousarray(d, np.int32)
    q = np.full_like(s, np.nan)
    declined = np.zeros(len(s), np.uint8)
    L.div_batch(len(s), s.ctypes.data, d.ctypes.data, q.ctypes.data, declined.ctypes.data)
    return q, declined.astype(bool)


def assert_div_bitwise(L, s, d):
    q, declined = emul_div(L, s, d)
    want = s / d
    ok = ~declined
    bad = np.nonzero(q[ok].view(np.uint64) != want[ok].view(np.uint64))[0]
    assert bad.size == 0, "first mismatch: %r / %d -> %r, IEEE %r" % (
        s[ok][bad[0]], d[ok][bad[0]], q[ok][bad[0]], want[ok][bad[0]])
    # declined only for zero or subnormal sums and subnormal quotients
    assert np.all((s[declined] == 0) | (np.abs(s[declined]) < np.finfo(np.float64).tiny)
                  | (np.abs(want[declined]) < np.finfo(np.float64).tiny))
    return declined


def test_division_every_divisor_random_sums(lib):
    rng = np.random.default_rng(6)
    n = 640_000
    d = np.tile(np.arange(1, 65, dtype=np.int32), n // 64)
    s = from_parts(rng.integers(0, 2, n), rng.integers(1, 2047, n), rng.integers(0, 1 << 52, n, dtype=np.uint64))
    declined = assert_div_bitwise(lib, s, d)
    assert declined.mean() < 0.01  # only quotients near the bottom of the exponent range


def test_division_exact_and_near_exact_quotients(lib):
    rng = np.random.default_rng(7)
    n = 400_000
    d = rng.integers(1, 65, n).astype(np.int32)
    m = rng.integers(1, 1 << 46, n).astype(np.float64)
    exact = m * d  # exactly representable, s / d == m
    assert_div_bitwise(lib, exact, d)
    assert_div_bitwise(lib, np.nextafter(exact, np.inf), d)   # remainder just above zero
    assert_div_bitwise(lib, np.nextafter(exact, -np.inf), d)  # remainder just below the divisor
    # the sweep's case: sums of d coordinates
    sums = rng.uniform(-0.5, 0.5, n) * d
    assert_div_bitwise(lib, sums, d)


def test_division_hand_offs(lib):
    tiny = np.finfo(np.float64).tiny
    s = np.array([0.0, -0.0, 5e-324, tiny / 2, tiny, 3 * tiny, 64 * tiny, -tiny * 1.5, 1e-307, np.finfo(np.float64).max])
    s2, d2 = np.meshgrid(s, np.arange(1, 65, dtype=np.int32))
    declined = assert_div_bitwise(lib, s2.ravel(), d2.ravel())
    assert declined[(s2.ravel() == 0)].all()


def emul_root(L, lo, hi):
    lo = np.ascontiguousarray(lo, np.float64)
    hi = np.ascontiguousarray(hi, np.float64)
    r = np.empty_like(lo)
    L.root_batch(len(lo), lo.ctypes.data, hi.ctypes.data, r.ctypes.data)
    return r


def test_root_of_ratio_within_two_ulps(lib):
    # squared edge lengths of every magnitude the seed handles, ratios down to 2^-126
    rng = np.random.default_rng(8)
    n = 600_000
    hi = rng.uniform(1, 2, n) * np.exp2(rng.integers(-950, 950, n).astype(np.float64))
    lo = np.minimum(hi * np.exp2(-rng.uniform(0, 125, n)) * rng.uniform(0.5, 1, n), hi)
    lo[:1000] = hi[:1000]                            # equilateral: ratio exactly 1
    lo[1000:2000] = hi[1000:2000] * 0.25             # exact roots
    got = emul_root(lib, lo, hi)
    want = np.sqrt(lo / hi)
    assert np.all(np.abs(got - want) <= 2 * np.spacing(want))


def test_root_of_ratio_hand_offs_are_the_fpu_result(lib):
    tiny = np.finfo(np.float64).tiny
    hi = np.array([0.0, 1.0, 1.0, 1e-300, 1e300, 1.0, 3.0, 5e-324])
    lo = np.array([0.0, 0.0, 5e-324, 1e-301, 1e299, 2.0 ** -130, tiny, 5e-324])
    with np.errstate(invalid="ignore", divide="ignore"):
        want = np.where(hi > 0, np.sqrt(lo / hi), 0.0)
    assert np.array_equal(emul_root(lib, lo, hi), want)
