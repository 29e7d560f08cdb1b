"""FP64 CPU oracle for Laplacian mesh smoothing and its orderings.

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()``
and by the benchmark's CPU-baseline leg, never by the library.  It shares no
code with the CUDA path.  The arithmetic lives in ``lms_oracle.c`` (plain C,
``-O2 -ffp-contract=off``); this module only marshals numpy arrays.

Each function follows the paper (Aupy, Park & Raghavan, "Locality-Aware
Laplacian Mesh Smoothing"):
  vertex_quality / mesh_quality   Section 3.2 and Algorithm 1 (global quality)
  jacobi_sweep / inplace_sweep    Eq. 1; Algorithm 1's inner loop
  smooth                          Algorithm 1 + the Section 5.1 stopping rule
  order_random / order_bfs / order_rdr   Section 5.2.1, Algorithm 2
  relabel, color_greedy, color_sequence  storage under an ordering; the
                                  in-place order a coloured Gauss-Seidel follows
  order_rbfs                      reversed BFS (Section 2, Munson and Hovland)
  order_brdr                      block RDR: Algorithm 2 inside blocks of the BFS order
                                  (a data-parallel variant; not in the paper)
  access_trace, reuse_distances, quantile   Section 2.2 / Fig. 1 reuse
                                  distance of one sweep, Table 2 quantiles
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lms_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liblms_oracle.so")

ORI, RANDOM, BFS, RDR, RBFS, BRDR = 0, 1, 2, 3, 4, 5
BRDR_BLOCK = 4096  # block size of the block RDR ordering
DISTINCT, ACCESSES = 0, 1
JACOBI, INPLACE = 0, 1


def build(force=False):
    """Compile lms_oracle.c (gcc -O2 -ffp-contract=off) into oracle/_build/."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                           "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_SRC_OMP = os.path.join(_HERE, "baseline_omp.c")
_LIB_OMP = os.path.join(_HERE, "_build", "liblms_baseline_omp.so")


def build_omp(force=False):
    """Compile baseline_omp.c (the Jacobi sweep under an OpenMP static schedule, a timing baseline only)."""
    if not force and os.path.exists(_LIB_OMP) and os.path.getmtime(_LIB_OMP) >= os.path.getmtime(_SRC_OMP):
        return _LIB_OMP
    os.makedirs(os.path.dirname(_LIB_OMP), exist_ok=True)
    tmp = _LIB_OMP + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
                           "-shared", "-o", tmp, _SRC_OMP])
    os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


_P_I32 = ctypes.POINTER(ctypes.c_int32)
_P_U8 = ctypes.POINTER(ctypes.c_uint8)
_P_F64 = ctypes.POINTER(ctypes.c_double)
_P_I64 = ctypes.POINTER(ctypes.c_int64)
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_handle = None


def _lib():
    global _handle
    if _handle is None:
        lib = ctypes.CDLL(build())
        sig = {
            "or_triangle_quality": [_I32, _P_I32, _P_F64, _P_F64],
            "or_vertex_quality": [_I32, _I32, _P_I32, _P_F64, _P_F64],
            "or_mesh_quality": [_I32, _I32, _P_I32, _P_F64, _P_F64],
            "or_jacobi_sweep": [_I32, _P_I32, _P_I32, _P_U8, _P_F64, _P_F64],
            "or_inplace_sweep": [_I32, _P_I32, _P_I32, _P_U8, _I32, _P_I32, _P_F64],
            "or_smooth": [_I32, _P_I32, _P_I32, _P_U8, _I32, _P_I32, _P_F64, _I32, _I32, _I32, _P_I32,
                          ctypes.c_double, ctypes.c_double, _P_I32, _P_F64],
            "or_order_random": [_I32, ctypes.c_uint64, _P_I32],
            "or_order_bfs": [_I32, _P_I32, _P_I32, _P_I32],
            "or_order_rdr": [_I32, _P_I32, _P_I32, _P_U8, _P_F64, _P_I32],
            "or_relabel": [_I32, _P_I32, _P_I32, _P_I32, _P_I32, _P_I32],
            "or_color_greedy": [_I32, _P_I32, _P_I32, _P_U8, _P_I32, _P_I32, _P_I32],
            "or_color_sequence": [_I32, _P_U8, _P_I32, _P_I32, _I32, _P_I32, _P_I32],
            "or_block_sequence": [_I32, _P_I32, _P_I32, _P_U8, _P_I32, _P_I32, _I32, _I32, _P_I32, _P_I32,
                                  _P_I32, _P_I32],
            "or_order_rbfs": [_I32, _P_I32, _P_I32, _P_I32],
            "or_order_brdr": [_I32, _P_I32, _P_I32, _P_U8, _P_F64, _I32, _P_I32],
            "or_access_trace": [_I32, _P_I32, _P_I32, _P_U8, _I32, _P_I32, _I32, _P_I32, _P_I64],
            "or_reuse_distances": [_I64, _P_I32, _I32, _I32, _P_I64, _P_I64],
            "or_quantile": [_I64, _P_I64, ctypes.c_double, _P_I64],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        _handle = lib
    return _handle


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _check(rc, name):
    if rc != 0:
        raise RuntimeError("%s failed with %d" % (name, rc))


def triangle_quality(tri, xy):
    tri, xy = _i32(tri).reshape(-1, 3), _f64(xy).reshape(-1, 2)
    q = np.empty(len(tri), np.float64)
    _check(_lib().or_triangle_quality(len(tri), _p(tri, _P_I32), _p(xy, _P_F64), _p(q, _P_F64)), "triangle_quality")
    return q


def vertex_quality(n, tri, xy):
    tri, xy = _i32(tri).reshape(-1, 3), _f64(xy).reshape(-1, 2)
    q = np.empty(n, np.float64)
    _check(_lib().or_vertex_quality(n, len(tri), _p(tri, _P_I32), _p(xy, _P_F64), _p(q, _P_F64)), "vertex_quality")
    return q


def mesh_quality(n, tri, xy):
    tri, xy = _i32(tri).reshape(-1, 3), _f64(xy).reshape(-1, 2)
    Q = ctypes.c_double()
    _check(_lib().or_mesh_quality(n, len(tri), _p(tri, _P_I32), _p(xy, _P_F64), ctypes.byref(Q)), "mesh_quality")
    return Q.value


def jacobi_sweep(row_ptr, col_idx, is_boundary, xy):
    row_ptr, col_idx, bnd, src = _i32(row_ptr), _i32(col_idx), _u8(is_boundary), _f64(xy).reshape(-1, 2)
    dst = np.empty_like(src)
    n = len(row_ptr) - 1
    _check(_lib().or_jacobi_sweep(n, _p(row_ptr, _P_I32), _p(col_idx, _P_I32), _p(bnd, _P_U8), _p(src, _P_F64),
                                  _p(dst, _P_F64)), "jacobi_sweep")
    return dst


def inplace_sweep(row_ptr, col_idx, is_boundary, seq, xy):
    row_ptr, col_idx, bnd, seq = _i32(row_ptr), _i32(col_idx), _u8(is_boundary), _i32(seq)
    out = _f64(xy).reshape(-1, 2).copy()
    n = len(row_ptr) - 1
    _check(_lib().or_inplace_sweep(n, _p(row_ptr, _P_I32), _p(col_idx, _P_I32), _p(bnd, _P_U8), len(seq),
                                   _p(seq, _P_I32), _p(out, _P_F64)), "inplace_sweep")
    return out


def smooth(row_ptr, col_idx, is_boundary, xy, iters, mode=JACOBI, seq=None, tri=None, tol=-1.0,
           goal=float("inf")):
    """Algorithm 1 with the Section 5.1 stopping rule; returns (xy, sweeps_done, Q history or None)."""
    row_ptr, col_idx, bnd = _i32(row_ptr), _i32(col_idx), _u8(is_boundary)
    out = _f64(xy).reshape(-1, 2).copy()
    n = len(row_ptr) - 1
    seq = _i32(seq) if seq is not None else None
    tri = _i32(tri).reshape(-1, 3) if tri is not None else None
    hist = np.full(iters + 1, np.nan) if tol >= 0 else None
    done = ctypes.c_int32()
    _check(_lib().or_smooth(n, _p(row_ptr, _P_I32), _p(col_idx, _P_I32), _p(bnd, _P_U8),
                            len(tri) if tri is not None else 0, _p(tri, _P_I32), _p(out, _P_F64), iters, mode,
                            len(seq) if seq is not None else 0, _p(seq, _P_I32), tol, goal, ctypes.byref(done),
                            _p(hist, _P_F64)), "smooth")
    if hist is not None:
        hist = hist[: done.value + 1]
    return out, done.value, hist


_omp_handle = None


def jacobi_omp(row_ptr, col_idx, is_boundary, xy, iters, threads=0):
    """Timing baseline, not a parity reference: ``iters`` Jacobi sweeps with the vertex loop under an OpenMP
    static schedule on ``threads`` host threads (0: all).  Returns (xy, threads used); equals ``smooth``'s
    Jacobi result bit for bit."""
    global _omp_handle
    if _omp_handle is None:
        lib = ctypes.CDLL(build_omp())
        lib.bl_jacobi_omp.argtypes = [_I32, _P_I32, _P_I32, _P_U8, _P_F64, _I32, _I32]
        lib.bl_jacobi_omp.restype = ctypes.c_int
        _omp_handle = lib
    row_ptr, col_idx, bnd = _i32(row_ptr), _i32(col_idx), _u8(is_boundary)
    out = _f64(xy).reshape(-1, 2).copy()
    used = _omp_handle.bl_jacobi_omp(len(row_ptr) - 1, _p(row_ptr, _P_I32), _p(col_idx, _P_I32), _p(bnd, _P_U8),
                                     _p(out, _P_F64), int(iters), int(threads))
    if used < 0:
        raise RuntimeError("bl_jacobi_omp failed")
    return out, used


def order_random(n, seed):
    p = np.empty(n, np.int32)
    _check(_lib().or_order_random(n, ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), _p(p, _P_I32)), "order_random")
    return p


def order_bfs(row_ptr, col_idx):
    row_ptr, col_idx = _i32(row_ptr), _i32(col_idx)
    n = len(row_ptr) - 1
    p = np.empty(n, np.int32)
    _check(_lib().or_order_bfs(n, _p(row_ptr, _P_I32), _p(col_idx, _P_I32), _p(p, _P_I32)), "order_bfs")
    return p


def order_rdr(row_ptr, col_idx, is_boundary, q_v):
    row_ptr, col_idx, bnd, q_v = _i32(row_ptr), _i32(col_idx), _u8(is_boundary), _f64(q_v)
    n = len(row_ptr) - 1
    p = np.empty(n, np.int32)
    _check(_lib().or_order_rdr(n, _p(row_ptr, _P_I32), _p(col_idx, _P_I32), _p(bnd, _P_U8), _p(q_v, _P_F64),
                               _p(p, _P_I32)), "order_rdr")
    return p


def order_rbfs(row_ptr, col_idx):
    row_ptr, col_idx = _i32(row_ptr), _i32(col_idx)
    n = len(row_ptr) - 1
    p = np.empty(n, np.int32)
    _check(_lib().or_order_rbfs(n, _p(row_ptr, _P_I32), _p(col_idx, _P_I32), _p(p, _P_I32)), "order_rbfs")
    return p


def order_brdr(row_ptr, col_idx, is_boundary, q_v, block=BRDR_BLOCK):
    row_ptr, col_idx, bnd, q_v = _i32(row_ptr), _i32(col_idx), _u8(is_boundary), _f64(q_v)
    n = len(row_ptr) - 1
    p = np.empty(n, np.int32)
    _check(_lib().or_order_brdr(n, _p(row_ptr, _P_I32), _p(col_idx, _P_I32), _p(bnd, _P_U8), _p(q_v, _P_F64),
                                int(block), _p(p, _P_I32)), "order_brdr")
    return p


def order(mesh, ordering, seed=0, q_v=None):
    """Permutation new_to_old of a mesh dict for ORI/RANDOM/BFS/RDR/RBFS (RDR keys from its coordinates)."""
    n = mesh["n"]
    if ordering == ORI:
        return np.arange(n, dtype=np.int32)
    if ordering == RANDOM:
        return order_random(n, seed)
    if ordering == BFS:
        return order_bfs(mesh["row_ptr"], mesh["col_idx"])
    if ordering == RDR:
        if q_v is None:
            q_v = vertex_quality(n, mesh["tri"], mesh["xy"])
        return order_rdr(mesh["row_ptr"], mesh["col_idx"], mesh["is_boundary"], q_v)
    if ordering == RBFS:
        return order_rbfs(mesh["row_ptr"], mesh["col_idx"])
    if ordering == BRDR:
        if q_v is None:
            q_v = vertex_quality(n, mesh["tri"], mesh["xy"])
        return order_brdr(mesh["row_ptr"], mesh["col_idx"], mesh["is_boundary"], q_v)
    raise ValueError(ordering)


def relabel(row_ptr, col_idx, new_to_old):
    row_ptr, col_idx, p = _i32(row_ptr), _i32(col_idx), _i32(new_to_old)
    n = len(row_ptr) - 1
    rp, ci = np.empty(n + 1, np.int32), np.empty(len(col_idx), np.int32)
    _check(_lib().or_relabel(n, _p(row_ptr, _P_I32), _p(col_idx, _P_I32), _p(p, _P_I32), _p(rp, _P_I32),
                             _p(ci, _P_I32)), "relabel")
    return rp, ci


def color_greedy(row_ptr, col_idx, is_boundary, new_to_old):
    row_ptr, col_idx, bnd, p = _i32(row_ptr), _i32(col_idx), _u8(is_boundary), _i32(new_to_old)
    n = len(row_ptr) - 1
    colour, nc = np.empty(n, np.int32), ctypes.c_int32()
    _check(_lib().or_color_greedy(n, _p(row_ptr, _P_I32), _p(col_idx, _P_I32), _p(bnd, _P_U8), _p(p, _P_I32),
                                  _p(colour, _P_I32), ctypes.byref(nc)), "color_greedy")
    return colour, nc.value


def color_sequence(is_boundary, new_to_old, colour, ncolours):
    bnd, p, colour = _u8(is_boundary), _i32(new_to_old), _i32(colour)
    n = len(bnd)
    seq, m = np.empty(n, np.int32), ctypes.c_int32()
    _check(_lib().or_color_sequence(n, _p(bnd, _P_U8), _p(p, _P_I32), _p(colour, _P_I32), ncolours,
                                    _p(seq, _P_I32), ctypes.byref(m)), "color_sequence")
    return seq[: m.value]


def block_sequence(row_ptr, col_idx, is_boundary, new_to_old, colour, ncolours, tile):
    """Block order of the in-place sweep: (tile colour, tile, vertex colour, storage position).  Returns
    (seq of original ids, tile colours, number of tile colours)."""
    rp, ci, bnd, p, colour = _i32(row_ptr), _i32(col_idx), _u8(is_boundary), _i32(new_to_old), _i32(colour)
    n = len(rp) - 1
    ntiles = (n + tile - 1) // tile
    tc, nt = np.empty(ntiles, np.int32), ctypes.c_int32()
    seq, m = np.empty(n, np.int32), ctypes.c_int32()
    _check(_lib().or_block_sequence(n, _p(rp, _P_I32), _p(ci, _P_I32), _p(bnd, _P_U8), _p(p, _P_I32),
                                    _p(colour, _P_I32), ncolours, tile, _p(tc, _P_I32), ctypes.byref(nt),
                                    _p(seq, _P_I32), ctypes.byref(m)), "block_sequence")
    return seq[: m.value], tc, nt.value


def block_gs_smooth(mesh, new_to_old, tile, iters, tol=-1.0):
    """Block Gauss-Seidel reference: in-place sweeps in block order over the first-fit colouring."""
    colour, nc = color_greedy(mesh["row_ptr"], mesh["col_idx"], mesh["is_boundary"], new_to_old)
    seq, _, _ = block_sequence(mesh["row_ptr"], mesh["col_idx"], mesh["is_boundary"], new_to_old, colour, nc, tile)
    return smooth(mesh["row_ptr"], mesh["col_idx"], mesh["is_boundary"], mesh["xy"], iters, mode=INPLACE, seq=seq,
                  tri=mesh["tri"] if tol >= 0 else None, tol=tol)


def gs_smooth(mesh, new_to_old, iters, tol=-1.0):
    """Coloured Gauss-Seidel reference: in-place sweeps in (colour, storage position) order."""
    colour, nc = color_greedy(mesh["row_ptr"], mesh["col_idx"], mesh["is_boundary"], new_to_old)
    seq = color_sequence(mesh["is_boundary"], new_to_old, colour, nc)
    return smooth(mesh["row_ptr"], mesh["col_idx"], mesh["is_boundary"], mesh["xy"], iters, mode=INPLACE, seq=seq,
                  tri=mesh["tri"] if tol >= 0 else None, tol=tol)


def access_trace(row_ptr, col_idx, is_boundary, seq, with_vertex=True):
    """Original ids accessed by one sweep visiting the interior vertices of seq (Fig. 3 pattern)."""
    row_ptr, col_idx, bnd, seq = _i32(row_ptr), _i32(col_idx), _u8(is_boundary), _i32(seq)
    n = len(row_ptr) - 1
    ln = ctypes.c_int64()
    args = (n, _p(row_ptr, _P_I32), _p(col_idx, _P_I32), _p(bnd, _P_U8), len(seq), _p(seq, _P_I32), int(with_vertex))
    _check(_lib().or_access_trace(*args, None, ctypes.byref(ln)), "access_trace")
    trace = np.empty(ln.value, np.int32)
    _check(_lib().or_access_trace(*args, _p(trace, _P_I32), ctypes.byref(ln)), "access_trace")
    return trace


def reuse_distances(trace, n, measure=DISTINCT):
    """Reuse distance of every non-first access of trace (elements 0..n-1), in trace order."""
    trace = _i32(trace)
    m = ctypes.c_int64()
    dist = np.empty(len(trace), np.int64)
    _check(_lib().or_reuse_distances(len(trace), _p(trace, _P_I32), n, measure, _p(dist, _P_I64), ctypes.byref(m)),
           "reuse_distances")
    return dist[: m.value]


def quantile(values, X):
    """Table 2's X quantile: the ceil(X m)-th smallest of the m values (clamped to [1, m])."""
    values = np.ascontiguousarray(values, dtype=np.int64)
    out = ctypes.c_int64()
    _check(_lib().or_quantile(len(values), _p(values, _P_I64), X, ctypes.byref(out)), "quantile")
    return out.value
