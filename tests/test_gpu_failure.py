"""Failure detection on the device without faulting the GPU.

Every device-side wait in the library is bounded.  The self-test makes one such wait expire (an
mbarrier phase that nothing completes); the host must report LMS_ERR_TIMEOUT, and the CUDA context must
stay usable for the next call.
"""
import numpy as np
import pytest

import meshgen
import oracle
import paper_1606_00803_gb300 as lms

pytestmark = pytest.mark.gpu


def test_expired_wait_reports_timeout_and_context_survives():
    assert lms.selftest_timeout(2000) == -7  # LMS_ERR_TIMEOUT
    m = meshgen.workload(0)
    want, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 5)
    with lms.Mesh.from_dict(m, lms.FP64) as g:
        g.smooth(5)
        assert np.array_equal(g.coords(), want)
    assert lms.selftest_timeout(500) == -7
