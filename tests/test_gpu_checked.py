"""The debug build with device-side bounds checks (-DLMS_CHECKS) on the parity cases.

compute-sanitizer is not available, so the kernels can be built to test every neighbour id against the
vertex count before using it.  A subprocess loads that build and runs the sweep, ordering and batch paths
against the oracle; every check must pass (zero violations) and the results must still match.
"""
import os
import subprocess
import sys

import pytest

from conftest import ROOT

pytestmark = pytest.mark.gpu

SCRIPT = r"""
import numpy as np, torch
import meshgen, oracle
import paper_1606_00803_gb300 as lms
enabled, _ = lms.debug_checks(reset=True)
assert enabled, "not the checked build"
m = meshgen.workload(1, side=70)
for o in (lms.ORI, lms.RDR, lms.BFS, lms.BRDR):
    p = oracle.order(m, o)
    with lms.Mesh.from_dict(m, lms.FP64) as g:
        g.reorder(o)
        assert np.array_equal(g.permutation(), p)
        g.smooth(9)
        want, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 9)
        assert np.array_equal(g.coords(), want)
        g.smooth(3, mode=lms.COLORED_GS)
        g.set_inplace_split(1)
        g.smooth(2, mode=lms.INPLACE_STATIC)
    with lms.Mesh.from_dict(m, lms.FP32) as g:
        g.reorder(o)
        g.smooth(9)
        g.smooth(3, mode=lms.COLORED_GS)
        g.smooth(2, mode=lms.INPLACE_STATIC)
meshes = [meshgen.generate(s, jitter=0.3, flip_frac=0.1, split_frac=0.05, seed=300 + s) for s in (12, 31, 50)]
xy = np.concatenate([mm["xy"] for mm in meshes])
for o in (lms.RDR, lms.BFS, lms.BRDR):
    with lms.Batch(meshes, ordering=o) as b:
        b.set_config(lms.KERNEL_DIRECT, 128, 4, 256)
        got = b.run(xy, 11, groups=2)
        for i, mm in enumerate(meshes):
            off = sum(x["n"] for x in meshes[:i])
            w, _, _ = oracle.smooth(mm["row_ptr"], mm["col_idx"], mm["is_boundary"], mm["xy"], 11)
            assert np.abs(got[off:off + mm["n"]] - w).max() <= 2e-6 * 1.5
dev = torch.device("cuda")
rp = torch.tensor(m["row_ptr"], dtype=torch.int32, device=dev)
ci = torch.tensor(m["col_idx"], dtype=torch.int32, device=dev)
bd = torch.tensor(m["is_boundary"], dtype=torch.uint8, device=dev)
x = torch.tensor(m["xy"], dtype=torch.float64, device=dev).reshape(-1)
tmp = torch.empty_like(x)
lms.jacobi_noalloc(rp, ci, bd, x, tmp, 4)
torch.cuda.synchronize()
enabled, violations = lms.debug_checks()
assert violations == 0, violations
print("checked ok")
"""


def test_checked_build_runs_the_parity_cases_without_violations():
    env = dict(os.environ, LMS_LIBRARY="checked")
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked ok" in r.stdout
