"""Seeded synthetic 2D triangle meshes.

Input generator shared by the oracle-side tests, the parity tests and the
benchmark.  It holds none of the method's arithmetic (no smoothing, quality or
ordering); see ``meshgen.c`` for the construction and the order in which the
splitmix64 stream is consumed.

The named workloads stand in for the paper's Triangle-generated test meshes
(Section 5.1, Table 1: 0.3-0.4M vertices, average degree ~6), which are not
available:

  0  64 x 64 jittered grid, random diagonals, no flips/splits (4,096 vertices)
  1  1024 x 1024 jittered grid + 10% interior-edge flips + 5% centroid splits
  2  2048 x 2048 graded grid (x-spacing 1x -> 10x) + the same flips/splits
  3  512 independent meshes built as in 1, side log-uniform in [32, 448]
  4  4096 x 4096 jittered grid + flips/splits (~18.4M vertices)

``side=`` shrinks a workload for tests (same recipe, smaller grid).
"""
import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "meshgen.c")
_LIB = os.path.join(_HERE, "_build", "libmeshgen.so")

BASE_SEED = 0x1606008030000000


def build(force=False):
    """Compile meshgen.c into meshgen/_build/libmeshgen.so (gcc, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                           "-shared", "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


class _MgMesh(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_grid", ctypes.c_int32), ("ntri", ctypes.c_int32),
                ("nnz", ctypes.c_int64), ("nflips", ctypes.c_int32), ("nsplits", ctypes.c_int32),
                ("xy", ctypes.POINTER(ctypes.c_double)), ("row_ptr", ctypes.POINTER(ctypes.c_int32)),
                ("col_idx", ctypes.POINTER(ctypes.c_int32)), ("is_boundary", ctypes.POINTER(ctypes.c_uint8)),
                ("tri", ctypes.POINTER(ctypes.c_int32))]


_lib_handle = None


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build())
        lib.mg_generate.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_uint64, ctypes.POINTER(_MgMesh)]
        lib.mg_generate.restype = ctypes.c_int
        lib.mg_free.argtypes = [ctypes.POINTER(_MgMesh)]
        lib.mg_unit.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
        lib.mg_unit.restype = ctypes.c_double
        _lib_handle = lib
    return _lib_handle


def _copy(ptr, count, dtype):
    if count == 0:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(ptr, shape=(count,)).astype(dtype, copy=True)


def generate(side, graded=False, jitter=0.3, flip_frac=0.0, split_frac=0.0, seed=0):
    """Build one mesh; returns a dict of numpy arrays and counts.

    keys: n, n_grid, ntri, nnz, nflips, nsplits, side,
          xy float64[n,2], row_ptr int32[n+1], col_idx int32[nnz],
          is_boundary uint8[n], tri int32[ntri,3]
    """
    lib = _lib()
    m = _MgMesh()
    rc = lib.mg_generate(int(side), int(bool(graded)), float(jitter), float(flip_frac), float(split_frac),
                         ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), ctypes.byref(m))
    if rc != 0:
        raise RuntimeError("mg_generate failed with %d (side=%d)" % (rc, side))
    try:
        out = dict(n=m.n, n_grid=m.n_grid, ntri=m.ntri, nnz=int(m.nnz), nflips=m.nflips, nsplits=m.nsplits,
                   side=int(side),
                   xy=_copy(m.xy, 2 * m.n, np.float64).reshape(m.n, 2),
                   row_ptr=_copy(m.row_ptr, m.n + 1, np.int32),
                   col_idx=_copy(m.col_idx, int(m.nnz), np.int32),
                   is_boundary=_copy(m.is_boundary, m.n, np.uint8),
                   tri=_copy(m.tri, 3 * m.ntri, np.int32).reshape(m.ntri, 3))
    finally:
        lib.mg_free(ctypes.byref(m))
    return out


def batch_sides(count=512, lo=32, hi=448, seed=BASE_SEED + 3):
    """Side lengths round(exp(U(ln lo, ln hi))) drawn from splitmix64(seed)."""
    lib = _lib()
    st = ctypes.c_uint64(seed)
    sides = []
    for _ in range(count):
        u = lib.mg_unit(ctypes.byref(st))
        sides.append(int(round(math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo))))))
    return sides


WORKLOADS = {
    0: dict(side=64, graded=False, flip_frac=0.0, split_frac=0.0),
    1: dict(side=1024, graded=False, flip_frac=0.10, split_frac=0.05),
    2: dict(side=2048, graded=True, flip_frac=0.10, split_frac=0.05),
    4: dict(side=4096, graded=False, flip_frac=0.10, split_frac=0.05),
}


def workload(config, side=None):
    """Mesh of a named workload (0, 1, 2 or 4); ``side`` overrides the grid size."""
    if config not in WORKLOADS:
        raise ValueError("single-mesh workloads are 0, 1, 2 and 4; use batch_workload() for 3")
    w = dict(WORKLOADS[config])
    if side is not None:
        w["side"] = int(side)
    return generate(w["side"], graded=w["graded"], jitter=0.3, flip_frac=w["flip_frac"],
                    split_frac=w["split_frac"], seed=BASE_SEED + config)


def batch_workload(count=512, lo=32, hi=448):
    """Workload 3: ``count`` independent meshes built as workload 1, sides log-uniform in [lo, hi]."""
    sides = batch_sides(count, lo, hi)
    return [generate(s, graded=False, jitter=0.3, flip_frac=0.10, split_frac=0.05,
                     seed=BASE_SEED + 3 + 1000 + m) for m, s in enumerate(sides)]
