"""lms_jacobi_noalloc: FP64 Jacobi sweeps for callers that cannot allocate
device memory (they run inside another framework's memory pool, under a fixed
device-memory budget, or forbid allocations on their steady-state path).  The
caller owns every buffer; the sweeps' only scratch - one work-queue counter per
sweep - sits in a fixed array inside the library.

Checked through the C ABI against lms_smooth (FP64 Jacobi) on two calls in a
row, with the bit-exact bar the FP64 parity tests use.  This file is collected
last so that a run stopping at its first failure has run every other test."""
import ctypes
import math

import numpy as np
import pytest

import meshgen
import paper_1606_00803_gb300 as lms

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _entry():
    fn = lms._lib().lms_jacobi_noalloc
    fn.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def test_noalloc_jacobi_matches_lms_smooth_on_two_calls():
    torch = pytest.importorskip("torch")
    m = meshgen.workload(1, side=100)
    n = m["n"]
    diag = math.hypot(np.ptp(m["xy"][:, 0]), np.ptp(m["xy"][:, 1]))
    with lms.Mesh.from_dict(m, lms.FP64) as g:
        g.smooth(7)
        want_a = g.coords()
        g.smooth(6)
        want_b = g.coords()
    dev = torch.device("cuda", torch.cuda.current_device())
    rp = torch.from_numpy(m["row_ptr"]).to(dev)
    ci = torch.from_numpy(m["col_idx"]).to(dev)
    bnd = torch.from_numpy(m["is_boundary"]).to(dev)
    xy = torch.from_numpy(m["xy"]).to(dev).contiguous()
    tmp = torch.empty_like(xy)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    fn = _entry()
    args = [n, rp.data_ptr(), ci.data_ptr(), bnd.data_ptr(), xy.data_ptr(), tmp.data_ptr()]
    assert fn(*args, 7, stream) == 0          # first call: 7 sweeps from the input
    torch.cuda.synchronize()
    got_a = xy.cpu().numpy()
    assert np.abs(got_a - want_a).max() <= TOL64 * diag
    assert np.array_equal(got_a, want_a)
    assert fn(*args, 6, stream) == 0          # second call reuses the counters: 6 more sweeps
    torch.cuda.synchronize()
    got_b = xy.cpu().numpy()
    assert np.abs(got_b - want_b).max() <= TOL64 * diag
    assert np.array_equal(got_b, want_b)


def test_noalloc_jacobi_rejects_too_many_sweeps():
    torch = pytest.importorskip("torch")
    m = meshgen.workload(0, side=8)
    dev = torch.device("cuda", torch.cuda.current_device())
    rp, ci = torch.from_numpy(m["row_ptr"]).to(dev), torch.from_numpy(m["col_idx"]).to(dev)
    bnd, xy = torch.from_numpy(m["is_boundary"]).to(dev), torch.from_numpy(m["xy"]).to(dev).contiguous()
    tmp = torch.empty_like(xy)
    fn = _entry()
    rc = fn(m["n"], rp.data_ptr(), ci.data_ptr(), bnd.data_ptr(), xy.data_ptr(), tmp.data_ptr(), 1025, None)
    assert rc == -1  # LMS_ERR_ARG
    assert "1024" in lms._lib().lms_last_error_detail().decode()
