"""The debug build with device-side bounds checks (-DLMS_CHECKS) on the parity cases.

compute-sanitizer is not available, so the kernels can be built to test every neighbour id against the
vertex count before using it.  A subprocess loads that build and runs every sweep mode (Jacobi, coloured
GS, the one-thread in-place sweep, block GS, the tile-staged kernel), the orderings, the batch kernels
(direct, staged, SELL) and the no-alloc entry point against the oracle: every check must pass (zero
violations), FP64 results must equal the oracle bit for bit and FP32 results stay within 2e-6 x the
bounding-box diagonal.
"""
import os
import subprocess
import sys

import pytest

from conftest import ROOT

pytestmark = pytest.mark.gpu

SCRIPT = r"""
import math
import numpy as np, torch
import meshgen, oracle
import paper_1606_00803_gb300 as lms
TOL32 = 2e-6
def diag(mm):
    return math.hypot(np.ptp(mm["xy"][:, 0]), np.ptp(mm["xy"][:, 1]))
def close32(got, want, mm):
    e = np.abs(got - want).max() / diag(mm)
    assert e <= TOL32, e
enabled, _ = lms.debug_checks(reset=True)
assert enabled, "not the checked build"
m = meshgen.workload(1, side=70)
xy0 = m["xy"]
for o in (lms.ORI, lms.RDR, lms.BFS, lms.BRDR):
    p = oracle.order(m, o)
    want_j, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], xy0, 9)
    want_gs, _, _ = oracle.gs_smooth(m, p, 3)
    want_seq, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], xy0, 2, mode=oracle.INPLACE, seq=p)
    want_blk, _, _ = oracle.block_gs_smooth(m, p, 96, 4)
    for prec in (lms.FP64, lms.FP32):
        with lms.Mesh.from_dict(m, prec) as g:
            g.reorder(o)
            assert np.array_equal(g.permutation(), p)
            runs = [("jacobi", lambda: g.smooth(9), want_j),
                    ("gs", lambda: g.smooth(3, mode=lms.COLORED_GS), want_gs),
                    ("inplace1", lambda: (g.set_inplace_split(1), g.smooth(2, mode=lms.INPLACE_STATIC)), want_seq),
                    ("block_gs", lambda: (g.set_block_tile(96), g.smooth(4, mode=lms.BLOCK_GS)), want_blk),
                    ("block_gs_staged", lambda: (g.set_block_staging(1), g.smooth(4, mode=lms.BLOCK_GS),
                                                 g.set_block_staging(0)), want_blk)]
            for name, run, want in runs:
                g.set_coords(xy0)
                run()
                got = g.coords()
                if prec == lms.FP64:
                    assert np.array_equal(got, want), (o, name)
                else:
                    close32(got, want, m)
            g.set_launch(lms.KERNEL_STAGED, 256, 256)
            g.set_coords(xy0)
            g.smooth(9)
            if prec == lms.FP64:
                assert np.array_equal(g.coords(), want_j), (o, "staged")
            else:
                close32(g.coords(), want_j, m)
meshes = [meshgen.generate(s, jitter=0.3, flip_frac=0.1, split_frac=0.05, seed=300 + s) for s in (12, 31, 50)]
xy = np.concatenate([mm["xy"] for mm in meshes])
wants = [oracle.smooth(mm["row_ptr"], mm["col_idx"], mm["is_boundary"], mm["xy"], 11)[0] for mm in meshes]
for o in (lms.RDR, lms.BFS, lms.BRDR):
    for cfg in ((lms.KERNEL_DIRECT, 128, 4, 256), (lms.KERNEL_STAGED, 128, 1, 256), (lms.KERNEL_SELL, 128, 4, 256),
                (lms.KERNEL_PACKED, 128, 4, 256)):
        with lms.Batch(meshes, ordering=o) as b:
            b.set_config(*cfg)
            got = b.run(xy, 11, groups=1 if cfg[0] == lms.KERNEL_SELL else 2)
            for i, mm in enumerate(meshes):
                off = sum(x["n"] for x in meshes[:i])
                close32(got[off:off + mm["n"]], wants[i], mm)
dev = torch.device("cuda")
rp = torch.tensor(m["row_ptr"], dtype=torch.int32, device=dev)
ci = torch.tensor(m["col_idx"], dtype=torch.int32, device=dev)
bd = torch.tensor(m["is_boundary"], dtype=torch.uint8, device=dev)
x = torch.tensor(m["xy"], dtype=torch.float64, device=dev).reshape(-1)
tmp = torch.empty_like(x)
lms.jacobi_noalloc(rp, ci, bd, x, tmp, 4)
torch.cuda.synchronize()
want4, _, _ = oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], xy0, 4)
assert np.array_equal(x.cpu().numpy().reshape(-1, 2), want4)
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
