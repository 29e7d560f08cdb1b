"""GB300 Laplacian mesh smoothing with locality-aware vertex orderings.

Thin Python binding of the C ABI in ``include/lms.h`` (liblms.so, built
in-tree by ``_build.build()``).  This module only marshals arguments: every
step of the method runs in the library (host orderings in C++, sweeps,
quality reductions and relabelling in sm_103a kernels).  There is no Python or
CPU fallback; a missing library raises.

PyTorch, when present with a GPU, supplies the CUDA stream (the current
stream at call time) and the device memory (the library allocates through
torch's caching allocator).

Method: Aupy, Park & Raghavan, "Locality-Aware Laplacian Mesh Smoothing"
(Eq. 1, Algorithm 1, Section 3.2 quality, Section 5.1 stopping rule,
Algorithm 2 RDR ordering).
"""
import ctypes
import os

import numpy as np

from . import _build

FP64, FP32 = 0, 1
KERNEL_DIRECT, KERNEL_STAGED, KERNEL_SELL, KERNEL_PACKED = 0, 1, 2, 3
ORI, RANDOM, BFS, RDR, RBFS, BRDR = 0, 1, 2, 3, 4, 5
BRDR_BLOCK = 4096  # LMS_BRDR_BLOCK
JACOBI, COLORED_GS, INPLACE_STATIC, BLOCK_GS = 0, 1, 2, 3
REUSE_DISTINCT, REUSE_ACCESSES = 0, 1
FP64_ARITH_FPU, FP64_ARITH_INT_ADDS, FP64_ARITH_INT, FP64_ARITH_MIXED2, FP64_ARITH_MIXED3 = 0, 1, 2, 3, 4
ORDERINGS = {"ori": ORI, "random": RANDOM, "bfs": BFS, "rdr": RDR, "rbfs": RBFS, "brdr": BRDR}
MODES = {"jacobi": JACOBI, "gs": COLORED_GS, "colored_gs": COLORED_GS, "inplace_static": INPLACE_STATIC}
PRECISIONS = {"fp64": FP64, "fp32": FP32}

LMS_OK = 0
ERRORS = {-1: "LMS_ERR_ARG", -2: "LMS_ERR_CSR", -3: "LMS_ERR_ISOLATED", -4: "LMS_ERR_NO_TRIANGLES",
          -5: "LMS_ERR_CUDA", -6: "LMS_ERR_OOM", -7: "LMS_ERR_TIMEOUT", -8: "LMS_ERR_STATE"}


class LmsError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        msg = "%s failed: %s (%s)" % (where, ERRORS.get(status, status), _lib().lms_error_string(status).decode())
        if detail:
            msg += ": " + detail
        super().__init__(msg)


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
_D = ctypes.c_double
_PI32 = ctypes.POINTER(ctypes.c_int32)
_PI64 = ctypes.POINTER(ctypes.c_int64)
_PD = ctypes.POINTER(ctypes.c_double)


class MeshDesc(ctypes.Structure):
    _fields_ = [("n", _I32), ("row_ptr", _P), ("col_idx", _P), ("xy", _P), ("is_boundary", _P), ("ntri", _I32),
                ("tri", _P)]


_SIGS = {
    "lms_error_string": ([ctypes.c_int], ctypes.c_char_p),
    "lms_last_error_detail": ([], ctypes.c_char_p),
    "lms_set_device_allocator": ([_P, _P, _P], ctypes.c_int),
    "lms_validate": ([_I32, _P, _P, _P, _I32, _P], ctypes.c_int),
    "lms_order_host": ([_I32, _P, _P, _P, _P, ctypes.c_int, _U64, _P], ctypes.c_int),
    "lms_color_host": ([_I32, _P, _P, _P, _P, _P, _PI32], ctypes.c_int),
    "lms_reuse_profile": ([_I32, _P, _P, _P, _P, _I32, _I32, _I32, _P, _P, _PD, _PI64, _PI64, _P], ctypes.c_int),
    "lms_create": ([_I32, _P, _P, _P, _P, _I32, _P, ctypes.c_int, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "lms_reorder": ([_P, ctypes.c_int, _U64], ctypes.c_int),
    "lms_smooth": ([_P, _I32, ctypes.c_int, _D, _PI32], ctypes.c_int),
    "lms_quality": ([_P, _PD], ctypes.c_int),
    "lms_set_launch": ([_P, _I32, _I32, _I32], ctypes.c_int),
    "lms_get_coords": ([_P, _P], ctypes.c_int),
    "lms_set_coords": ([_P, _P], ctypes.c_int),
    "lms_get_permutation": ([_P, _P], ctypes.c_int),
    "lms_get_colors": ([_P, _P, _PI32], ctypes.c_int),
    "lms_get_csr": ([_P, _P, _P, _P], ctypes.c_int),
    "lms_last_stats": ([_P, _PD, _PD, _PD, _PD], ctypes.c_int),
    "lms_last_error_stats": ([_P, _PD, _PD], ctypes.c_int),
    "lms_last_launches": ([_P, _PI64], ctypes.c_int),
    "lms_last_reorder_ms": ([_P, _PD, _PD], ctypes.c_int),
    "lms_set_inplace_split": ([_P, _I32], ctypes.c_int),
    "lms_block_order": ([_I32, _P, _P, _P, _P, _I32, _P, _P, _P, _P], ctypes.c_int),
    "lms_block_walk": ([_I32, _P, _P, _P, _P, _I32, _P, _PI32, _PI32], ctypes.c_int),
    "lms_set_fp64_arith": ([_P, _I32], ctypes.c_int),
    "lms_set_block_tile": ([_P, _I32], ctypes.c_int),
    "lms_set_block_staging": ([_P, _I32], ctypes.c_int),
    "lms_get_block_tile": ([_P, _PI32], ctypes.c_int),
    "lms_destroy": ([_P], None),
    "lms_selftest_div64": ([_I32, _P, _P, _P], ctypes.c_int),
    "lms_selftest_div32": ([_I32, _P, _P, _P], ctypes.c_int),
    "lms_selftest_add64": ([_I32, _P, _P, _P], ctypes.c_int),
    "lms_selftest_divint64": ([_I32, _P, _P, _P], ctypes.c_int),
    "lms_selftest_timeout": ([_I32], ctypes.c_int),
    "lms_debug_checks": ([_PI32, ctypes.POINTER(ctypes.c_uint64), _I32], ctypes.c_int),
    "lms_jacobi_noalloc": ([_I32, _P, _P, _P, _P, _P, _I32, _P], ctypes.c_int),
    "lms_batch_create": ([_I32, ctypes.POINTER(MeshDesc), ctypes.c_int, _U64, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "lms_batch_smooth": ([_P, _I32], ctypes.c_int),
    "lms_batch_get_coords": ([_P, _I32, _P], ctypes.c_int),
    "lms_batch_get_all_coords": ([_P, _P], ctypes.c_int),
    "lms_batch_set_all_coords": ([_P, _P], ctypes.c_int),
    "lms_batch_run": ([_P, _P, _P, _I32, _I32], ctypes.c_int),
    "lms_batch_info": ([_P, _PI64, _PI64, _PI64, _PI32], ctypes.c_int),
    "lms_batch_get_config": ([_P, _PI32, _PI32, _PI32, _PI32, _PI32], ctypes.c_int),
    "lms_batch_set_config": ([_P, _I32, _I32, _I32, _I32, _I32], ctypes.c_int),
    "lms_batch_autotune": ([_P, _PI32, _PI32, _PI32, _PI32, _PI32], ctypes.c_int),
    "lms_batch_get_permutation": ([_P, _I32, _P], ctypes.c_int),
    "lms_batch_set_layout": ([_P, _I32], ctypes.c_int),
    "lms_batch_set_chains": ([_P, _I32], ctypes.c_int),
    "lms_batch_get_chains": ([_P, _PI32], ctypes.c_int),
    "lms_partition_meshes": ([_I32, _P, _I32, _P, _P], ctypes.c_int),
    "lms_batch_get_layout": ([_P, _PI32], ctypes.c_int),
    "lms_batch_last_launches": ([_P, _PI64], ctypes.c_int),
    "lms_batch_destroy": ([_P], None),
}

_handle = None


def library_path():
    return _build.LIB_CHECKED if os.environ.get("LMS_LIBRARY") == "checked" else _build.LIB


def _lib():
    """Load liblms.so, building it first when it is missing or stale."""
    global _handle
    if _handle is None:
        # launch configurations picked by lms_batch_autotune persist next to the library
        os.environ.setdefault("LMS_AUTOTUNE_CACHE", os.path.join(_build.OUT_DIR, "autotune_cache.txt"))
        # LMS_LIBRARY=checked loads the debug build with device bounds checks (built on demand)
        path = _build.build(checked=os.environ.get("LMS_LIBRARY") == "checked")
        lib = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _handle = lib
        _install_torch_allocator(lib)
    return _handle


def _check(status, where):
    if status != LMS_OK:
        detail = _lib().lms_last_error_detail().decode(errors="replace")
        raise LmsError(status, where, detail)


# ---------------------------------------------------------------- torch plumbing

_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_callbacks = []


def _torch_cuda():
    try:
        import torch
        return torch if torch.cuda.is_available() else None
    except Exception:
        return None


def _install_torch_allocator(lib):
    torch = _torch_cuda()
    if torch is None or os.environ.get("LMS_NO_TORCH_ALLOCATOR"):
        return

    def alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:
            return None

    def free(ptr, ctx):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    a, f = _ALLOC_T(alloc), _FREE_T(free)
    _callbacks.append((a, f))
    _check(lib.lms_set_device_allocator(ctypes.cast(a, _P), ctypes.cast(f, _P), None), "lms_set_device_allocator")


def current_stream():
    """cudaStream_t of torch's current stream (0 = legacy default stream when torch has no GPU)."""
    torch = _torch_cuda()
    return int(torch.cuda.current_stream().cuda_stream) if torch is not None else 0


# ---------------------------------------------------------------- marshalling

def _arr(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):  # torch tensor (e.g. page-locked host buffer)
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _host_f64(xy, n):
    if hasattr(xy, "data_ptr"):
        if xy.is_cuda or str(xy.dtype) != "torch.float64" or not xy.is_contiguous() or xy.numel() != 2 * n:
            raise ValueError("coordinates must be a contiguous host float64 tensor of 2n values")
        return xy
    a = _arr(xy, np.float64)
    if a.size != 2 * n:
        raise ValueError("expected %d coordinates, got %d" % (2 * n, a.size))
    return a


def validate(row_ptr, col_idx, is_boundary, tri=None):
    """lms_validate: LMS_OK or a negative status (no exception)."""
    rp, ci, b = _arr(row_ptr, np.int32), _arr(col_idx, np.int32), _arr(is_boundary, np.uint8)
    t = _arr(tri, np.int32) if tri is not None else None
    return _lib().lms_validate(len(rp) - 1, _ptr(rp), _ptr(ci), _ptr(b), 0 if t is None else t.size // 3, _ptr(t))


def order_host(row_ptr, col_idx, is_boundary, ordering, seed=0, q_v=None):
    """lms_order_host: new_to_old of ORI / RANDOM / BFS / RDR / RBFS / BRDR (RDR and BRDR need q_v)."""
    rp, ci, b = _arr(row_ptr, np.int32), _arr(col_idx, np.int32), _arr(is_boundary, np.uint8)
    q = _arr(q_v, np.float64) if q_v is not None else None
    n = len(rp) - 1
    out = np.empty(n, np.int32)
    _check(_lib().lms_order_host(n, _ptr(rp), _ptr(ci), _ptr(b), _ptr(q), int(ordering), seed & (2**64 - 1),
                                 _ptr(out)), "lms_order_host")
    return out


def partition_meshes(n_vertices, ranks):
    """lms_partition_meshes: (rank of each mesh, vertices per rank) - whole meshes balanced by vertex count."""
    nv = _arr(n_vertices, np.int32)
    rank_of, load = np.empty(len(nv), np.int32), np.empty(max(1, int(ranks)), np.int64)
    _check(_lib().lms_partition_meshes(len(nv), _ptr(nv), int(ranks), _ptr(rank_of), _ptr(load)),
           "lms_partition_meshes")
    return rank_of, load


def color_host(row_ptr, col_idx, is_boundary, new_to_old):
    """lms_color_host: (colour by original id, number of colours)."""
    rp, ci, b, p = (_arr(row_ptr, np.int32), _arr(col_idx, np.int32), _arr(is_boundary, np.uint8),
                    _arr(new_to_old, np.int32))
    n = len(rp) - 1
    colour, nc = np.empty(n, np.int32), ctypes.c_int32()
    _check(_lib().lms_color_host(n, _ptr(rp), _ptr(ci), _ptr(b), _ptr(p), _ptr(colour), ctypes.byref(nc)),
           "lms_color_host")
    return colour, nc.value


def reuse_profile(row_ptr, col_idx, is_boundary, new_to_old=None, with_vertex=True, measure=REUSE_DISTINCT,
                  quantiles=(0.5, 0.75, 0.9, 1.0)):
    """lms_reuse_profile: reuse distances of one sweep's access trace (Section 2.2, Table 2).

    Returns a dict: quantiles {X: value}, mean, accesses (trace length), reuses (accesses with
    a previous access of the same element) and hist (33 log2 buckets)."""
    rp, ci, b = _arr(row_ptr, np.int32), _arr(col_idx, np.int32), _arr(is_boundary, np.uint8)
    p = _arr(new_to_old, np.int32) if new_to_old is not None else None
    qs = _arr(list(quantiles), np.float64)
    out_q = np.empty(len(qs), np.int64)
    hist = np.zeros(33, np.int64)
    mean, acc, reu = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
    _check(_lib().lms_reuse_profile(len(rp) - 1, _ptr(rp), _ptr(ci), _ptr(b), _ptr(p), int(bool(with_vertex)),
                                    int(measure), len(qs), _ptr(qs), _ptr(out_q), ctypes.byref(mean),
                                    ctypes.byref(acc), ctypes.byref(reu), _ptr(hist)), "lms_reuse_profile")
    return {"quantiles": {float(x): int(v) for x, v in zip(qs, out_q)}, "mean": mean.value, "accesses": acc.value,
            "reuses": reu.value, "hist": hist}


def jacobi_noalloc(row_ptr, col_idx, is_boundary, xy, xy_tmp, iters, stream=None):
    """lms_jacobi_noalloc on caller-owned device tensors: row_ptr / col_idx int32, is_boundary uint8,
    xy / xy_tmp float64 (2n values each, contiguous, on the current CUDA device).  Positions are updated in
    xy; returns nothing and raises LmsError on a bad status."""
    tensors = (row_ptr, col_idx, is_boundary, xy, xy_tmp)
    wanted = ("torch.int32", "torch.int32", "torch.uint8", "torch.float64", "torch.float64")
    for t, w in zip(tensors, wanted):
        if not hasattr(t, "data_ptr") or not t.is_cuda or str(t.dtype) != w or not t.is_contiguous():
            raise ValueError("jacobi_noalloc takes contiguous CUDA tensors (int32 CSR, uint8 flags, float64 xy)")
    n = row_ptr.numel() - 1
    if xy.numel() != 2 * n or xy_tmp.numel() != 2 * n or is_boundary.numel() != n:
        raise ValueError("tensor sizes do not match the CSR")
    s = current_stream() if stream is None else int(stream)
    _check(_lib().lms_jacobi_noalloc(n, _ptr(row_ptr), _ptr(col_idx), _ptr(is_boundary), _ptr(xy), _ptr(xy_tmp),
                                     int(iters), ctypes.c_void_p(s)), "lms_jacobi_noalloc")


def debug_checks(reset=False):
    """lms_debug_checks: (bounds checks compiled in, failed checks since the last reset)."""
    en, v = ctypes.c_int32(), ctypes.c_uint64()
    _check(_lib().lms_debug_checks(ctypes.byref(en), ctypes.byref(v), int(bool(reset))), "lms_debug_checks")
    return bool(en.value), v.value


def selftest_timeout(wait_us=2000):
    """lms_selftest_timeout: status of a bounded device wait that is made to expire (LMS_ERR_TIMEOUT = -7)."""
    return _lib().lms_selftest_timeout(int(wait_us))


def block_order(row_ptr, col_idx, is_boundary, new_to_old, tile):
    """Block order of the in-place sweep (lms_block_order): (order of original ids, tile colours, count)."""
    rp, ci = _arr(row_ptr, np.int32), _arr(col_idx, np.int32)
    bnd, p = _arr(is_boundary, np.uint8), _arr(new_to_old, np.int32)
    n = len(rp) - 1
    if int(tile) < 1:
        raise ValueError("tile must be positive")
    tc = np.empty((n + int(tile) - 1) // int(tile), np.int32)
    order = np.empty(n, np.int32)
    nt, m = ctypes.c_int32(), ctypes.c_int32()
    _check(_lib().lms_block_order(n, _ptr(rp), _ptr(ci), _ptr(bnd), _ptr(p), int(tile), _ptr(tc), ctypes.byref(nt),
                                  _ptr(order), ctypes.byref(m)), "lms_block_order")
    return order[: m.value], tc, nt.value


def block_walk(row_ptr, col_idx, is_boundary, new_to_old, tile):
    """The BLOCK_GS tables walked in launch order (lms_block_walk): (visited original ids, launches)."""
    rp, ci = _arr(row_ptr, np.int32), _arr(col_idx, np.int32)
    bnd, p = _arr(is_boundary, np.uint8), _arr(new_to_old, np.int32)
    n = len(rp) - 1
    seq = np.empty(n, np.int32)
    m, launches = ctypes.c_int32(), ctypes.c_int32()
    _check(_lib().lms_block_walk(n, _ptr(rp), _ptr(ci), _ptr(bnd), _ptr(p), int(tile), _ptr(seq), ctypes.byref(m),
                                 ctypes.byref(launches)), "lms_block_walk")
    return seq[: m.value], launches.value


def selftest_add64(a, b):
    """Device sums a+b by the FP64 sweep's integer-pipe addition (lms_selftest_add64)."""
    a, b = _arr(a, np.float64), _arr(b, np.float64)
    if a.shape != b.shape:
        raise ValueError("a and b differ in shape")
    s = np.empty_like(a)
    _check(_lib().lms_selftest_add64(len(a), _ptr(a), _ptr(b), _ptr(s)), "lms_selftest_add64")
    return s


def selftest_divint64(s, d):
    """Device quotients s/d by the FP64 sweep's integer-pipe division (lms_selftest_divint64)."""
    s, d = _arr(s, np.float64), _arr(d, np.int32)
    q = np.empty_like(s)
    _check(_lib().lms_selftest_divint64(len(s), _ptr(s), _ptr(d), _ptr(q)), "lms_selftest_divint64")
    return q


def selftest_div32(s, d):
    """lms_selftest_div32: s / d by the FP32 sweeps' mean routine on the device (float32 arrays)."""
    sa, da = _arr(s, np.float32), _arr(d, np.int32)
    q = np.empty(len(sa), np.float32)
    _check(_lib().lms_selftest_div32(len(sa), _ptr(sa), _ptr(da), _ptr(q)), "lms_selftest_div32")
    return q


def selftest_div64(s, d):
    """Device quotients s/d by the FP64 sweep's division routine (lms_selftest_div64)."""
    s, d = _arr(s, np.float64), _arr(d, np.int32)
    q = np.empty_like(s)
    _check(_lib().lms_selftest_div64(len(s), _ptr(s), _ptr(d), _ptr(q)), "lms_selftest_div64")
    return q


class Mesh:
    """One mesh on the device (lms_handle)."""

    def __init__(self, row_ptr, col_idx, xy, is_boundary, tri=None, precision=FP64, stream=None):
        lib = _lib()
        self.precision = PRECISIONS.get(precision, precision)
        rp, ci, b = _arr(row_ptr, np.int32), _arr(col_idx, np.int32), _arr(is_boundary, np.uint8)
        self.n = len(rp) - 1
        self.nnz = int(rp[-1])
        xy = _host_f64(xy, self.n)
        t = _arr(tri, np.int32) if tri is not None else None
        self.ntri = 0 if t is None else t.size // 3
        self.stream = current_stream() if stream is None else int(stream)
        h = ctypes.c_void_p()
        _check(lib.lms_create(self.n, _ptr(rp), _ptr(ci), _ptr(xy), _ptr(b), self.ntri, _ptr(t), self.precision,
                              ctypes.c_void_p(self.stream), ctypes.byref(h)), "lms_create")
        self._h = h

    @classmethod
    def from_dict(cls, m, precision=FP64, stream=None):
        return cls(m["row_ptr"], m["col_idx"], m["xy"], m["is_boundary"], m.get("tri"), precision, stream)

    def _handle(self):
        if self._h is None:
            raise LmsError(-8, "Mesh", "handle closed")
        return self._h

    def reorder(self, ordering, seed=0):
        _check(_lib().lms_reorder(self._handle(), ORDERINGS.get(ordering, ordering), seed & (2**64 - 1)),
               "lms_reorder")

    def smooth(self, iters, mode=JACOBI, tol=-1.0):
        done = ctypes.c_int32()
        _check(_lib().lms_smooth(self._handle(), int(iters), MODES.get(mode, mode), float(tol), ctypes.byref(done)),
               "lms_smooth")
        return done.value

    def set_launch(self, kernel, block=256, tile=512):
        _check(_lib().lms_set_launch(self._handle(), kernel, block, tile), "lms_set_launch")

    def quality(self):
        q = ctypes.c_double()
        _check(_lib().lms_quality(self._handle(), ctypes.byref(q)), "lms_quality")
        return q.value

    def coords(self, out=None):
        out = np.empty((self.n, 2), np.float64) if out is None else out
        _check(_lib().lms_get_coords(self._handle(), _ptr(out)), "lms_get_coords")
        return out

    def set_coords(self, xy):
        xy = _host_f64(xy, self.n)
        _check(_lib().lms_set_coords(self._handle(), _ptr(xy)), "lms_set_coords")
        self._keep = xy  # the copy is asynchronous for page-locked buffers

    def permutation(self):
        p = np.empty(self.n, np.int32)
        _check(_lib().lms_get_permutation(self._handle(), _ptr(p)), "lms_get_permutation")
        return p

    def colors(self):
        c, nc = np.empty(self.n, np.int32), ctypes.c_int32()
        _check(_lib().lms_get_colors(self._handle(), _ptr(c), ctypes.byref(nc)), "lms_get_colors")
        return c, nc.value

    def csr(self):
        rp, ci, p = np.empty(self.n + 1, np.int32), np.empty(max(1, self.nnz), np.int32), np.empty(self.n, np.int32)
        _check(_lib().lms_get_csr(self._handle(), _ptr(rp), _ptr(ci), _ptr(p)), "lms_get_csr")
        return rp, ci[: self.nnz], p

    def last_stats(self):
        d, ms, q0, q1 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(_lib().lms_last_stats(self._handle(), ctypes.byref(d), ctypes.byref(ms), ctypes.byref(q0),
                                     ctypes.byref(q1)), "lms_last_stats")
        return dict(max_disp=d.value, ms=ms.value, q_first=q0.value, q_last=q1.value)

    def last_error_stats(self):
        """lms_last_error_stats: (largest displacement of the last sweep, device ms) of the last smooth."""
        d, ms = ctypes.c_double(), ctypes.c_double()
        _check(_lib().lms_last_error_stats(self._handle(), ctypes.byref(d), ctypes.byref(ms)), "lms_last_error_stats")
        return d.value, ms.value

    def last_launches(self):
        k = ctypes.c_int64()
        _check(_lib().lms_last_launches(self._handle(), ctypes.byref(k)), "lms_last_launches")
        return k.value

    def set_inplace_split(self, threads):
        """GPU threads of INPLACE_STATIC sweeps (0 = default, 1 = sequential Algorithm 1)."""
        _check(_lib().lms_set_inplace_split(self._handle(), int(threads)), "lms_set_inplace_split")

    def set_block_staging(self, on):
        """lms_set_block_staging: LMS_BLOCK_GS through shared memory (tile + halo) or from global memory."""
        _check(_lib().lms_set_block_staging(self._handle(), int(on)), "lms_set_block_staging")

    def set_block_tile(self, tile):
        """Tile (storage positions) of BLOCK_GS sweeps; 0 = by mesh size."""
        _check(_lib().lms_set_block_tile(self._handle(), int(tile)), "lms_set_block_tile")

    def block_tile(self):
        """Tile the next BLOCK_GS sweep uses."""
        t = ctypes.c_int32()
        _check(_lib().lms_get_block_tile(self._handle(), ctypes.byref(t)), "lms_get_block_tile")
        return t.value

    def set_fp64_arith(self, mode):
        """Where FP64 sums and means run: FP64_ARITH_* (every mode gives the same results)."""
        _check(_lib().lms_set_fp64_arith(self._handle(), int(mode)), "lms_set_fp64_arith")

    def last_reorder_ms(self):
        """(ordering ms, relabelled-layout ms) of the last reorder."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(_lib().lms_last_reorder_ms(self._handle(), ctypes.byref(a), ctypes.byref(b)), "lms_last_reorder_ms")
        return a.value, b.value

    def close(self):
        if getattr(self, "_h", None) is not None:
            _lib().lms_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent meshes smoothed by one persistent work-queue kernel per sweep (FP32)."""

    def __init__(self, meshes, ordering=RDR, seed=0, stream=None):
        lib = _lib()
        self._keep = []
        descs = (MeshDesc * len(meshes))()
        self.sizes = []
        for i, m in enumerate(meshes):
            rp, ci = _arr(m["row_ptr"], np.int32), _arr(m["col_idx"], np.int32)
            xy, b = _arr(m["xy"], np.float64), _arr(m["is_boundary"], np.uint8)
            t = _arr(m["tri"], np.int32) if m.get("tri") is not None else None
            self._keep.append((rp, ci, xy, b, t))
            n = len(rp) - 1
            self.sizes.append(n)
            descs[i] = MeshDesc(n, _ptr(rp).value, _ptr(ci).value, _ptr(xy).value, _ptr(b).value,
                                0 if t is None else t.size // 3, None if t is None else _ptr(t).value)
        self.k = len(meshes)
        self.stream = current_stream() if stream is None else int(stream)
        h = ctypes.c_void_p()
        _check(lib.lms_batch_create(self.k, descs, ORDERINGS.get(ordering, ordering), seed & (2**64 - 1),
                                    ctypes.c_void_p(self.stream), ctypes.byref(h)), "lms_batch_create")
        self._keep = None
        self._h = h
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        self.n_total = int(self.offsets[-1])

    def _handle(self):
        if self._h is None:
            raise LmsError(-8, "Batch", "handle closed")
        return self._h

    def smooth(self, iters):
        _check(_lib().lms_batch_smooth(self._handle(), int(iters)), "lms_batch_smooth")

    def coords(self, mesh):
        out = np.empty((self.sizes[mesh], 2), np.float64)
        _check(_lib().lms_batch_get_coords(self._handle(), int(mesh), _ptr(out)), "lms_batch_get_coords")
        return out

    def all_coords(self, out=None):
        out = np.empty((self.n_total, 2), np.float64) if out is None else out
        _check(_lib().lms_batch_get_all_coords(self._handle(), _ptr(out)), "lms_batch_get_all_coords")
        return out

    def set_all_coords(self, xy):
        xy = _host_f64(xy, self.n_total)
        _check(_lib().lms_batch_set_all_coords(self._handle(), _ptr(xy)), "lms_batch_set_all_coords")
        self._pending = xy

    def run(self, xy_in, iters, groups=4, out=None):
        """lms_batch_run: positions in (host), iters sweeps, positions out (host), pipelined over groups of
        meshes.  xy_in / out: contiguous FP64 host arrays or page-locked torch tensors of 2 * n_total values."""
        xy_in = _host_f64(xy_in, self.n_total)
        if out is None:
            out = np.empty((self.n_total, 2), np.float64)
        else:
            out = _host_f64(out, self.n_total)
        _check(_lib().lms_batch_run(self._handle(), _ptr(xy_in), _ptr(out), int(iters), int(groups)), "lms_batch_run")
        return out

    def permutation(self, mesh):
        p = np.empty(self.sizes[mesh], np.int32)
        _check(_lib().lms_batch_get_permutation(self._handle(), int(mesh), _ptr(p)), "lms_batch_get_permutation")
        return p

    def info(self):
        n, ni, nnz, tiles = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _check(_lib().lms_batch_info(self._handle(), ctypes.byref(n), ctypes.byref(ni), ctypes.byref(nnz),
                                     ctypes.byref(tiles)), "lms_batch_info")
        return dict(n_total=n.value, n_interior=ni.value, nnz_total=nnz.value, tiles=tiles.value)

    _CFG = ("kernel", "block", "chunk", "tile", "ctas_per_sm")

    def config(self):
        v = [ctypes.c_int32() for _ in range(5)]
        _check(_lib().lms_batch_get_config(self._handle(), *[ctypes.byref(x) for x in v]), "lms_batch_get_config")
        return dict(zip(self._CFG, [x.value for x in v]))

    def set_config(self, kernel, block, chunk, tile, ctas_per_sm=0):
        _check(_lib().lms_batch_set_config(self._handle(), kernel, block, chunk, tile, ctas_per_sm),
               "lms_batch_set_config")

    def autotune(self):
        """lms_batch_autotune: the chosen launch configuration, with the storage layout's window."""
        v = [ctypes.c_int32() for _ in range(5)]
        _check(_lib().lms_batch_autotune(self._handle(), *[ctypes.byref(x) for x in v]), "lms_batch_autotune")
        cfg = dict(zip(self._CFG, [x.value for x in v]))
        cfg["window"] = self.layout()
        cfg["chains"] = self.chains()
        return cfg

    def set_chains(self, chains):
        """lms_batch_set_chains: parallel chains of sweeps in the smoothing graph (results do not change)."""
        _check(_lib().lms_batch_set_chains(self._handle(), int(chains)), "lms_batch_set_chains")

    def chains(self):
        c = ctypes.c_int32()
        _check(_lib().lms_batch_get_chains(self._handle(), ctypes.byref(c)), "lms_batch_get_chains")
        return c.value

    def set_layout(self, window):
        """lms_batch_set_layout: store each run of `window` ordering positions grouped by row length (0: the
        ordering itself)."""
        _check(_lib().lms_batch_set_layout(self._handle(), int(window)), "lms_batch_set_layout")

    def layout(self):
        w = ctypes.c_int32()
        _check(_lib().lms_batch_get_layout(self._handle(), ctypes.byref(w)), "lms_batch_get_layout")
        return w.value

    def last_launches(self):
        k = ctypes.c_int64()
        _check(_lib().lms_batch_last_launches(self._handle(), ctypes.byref(k)), "lms_batch_last_launches")
        return k.value

    def close(self):
        if getattr(self, "_h", None) is not None:
            _lib().lms_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
