"""Storage layouts of the batched sweep (lms_batch_set_layout): every run of `window` ordering positions
stored grouped by row length.  Jacobi reads each row in its stored entry order, so the FP32 results must
equal the plain layout's bit for bit and stay within 2e-6 x bbox diagonal of the FP64 oracle (Eq. 1); the
reported ordering (Algorithm 2 for RDR) must not change."""
import math

import numpy as np
import pytest

import meshgen
import oracle
import paper_1606_00803_gb300 as lms

pytestmark = pytest.mark.gpu

TOL32 = 2e-6


def diag(m):
    return math.hypot(np.ptp(m["xy"][:, 0]), np.ptp(m["xy"][:, 1]))


def small_batch():
    sides = [12, 13, 17, 20, 25, 31, 40, 47, 55, 64, 90, 130]
    return [meshgen.generate(s, jitter=0.3, flip_frac=0.10, split_frac=0.05, seed=2000 + i)
            for i, s in enumerate(sides)]


@pytest.mark.parametrize("ordering", [lms.RDR, lms.BFS, lms.RANDOM])
def test_layout_windows_bit_identical_and_match_oracle(ordering):
    meshes = small_batch()
    wants = [oracle.smooth(m["row_ptr"], m["col_idx"], m["is_boundary"], m["xy"], 40)[0] for m in meshes]
    with lms.Batch(meshes, ordering=ordering, seed=11) as b:
        perms = [b.permutation(i) for i in range(len(meshes))]
        ref = None
        for window in (0, 32, 64, 256, 4096, 0):
            b.set_layout(window)
            assert b.layout() == window
            for cfg in ((lms.KERNEL_DIRECT, 128, 5, 512), (lms.KERNEL_DIRECT, 256, 6, 1024),
                        (lms.KERNEL_PACKED, 128, 4, 512),
                        (lms.KERNEL_SELL, 128, 4, 256), (lms.KERNEL_STAGED, 128, 1, 256)):
                b.set_config(*cfg)
                b.set_all_coords(np.concatenate([m["xy"] for m in meshes]))
                b.smooth(40)
                got = b.all_coords()
                if ref is None:
                    ref = got
                assert np.array_equal(got, ref), (window, cfg)
            for i, m in enumerate(meshes):
                assert np.array_equal(b.permutation(i), perms[i])
        for i, m in enumerate(meshes):
            o = int(b.offsets[i])
            assert np.abs(ref[o:o + m["n"]] - wants[i]).max() <= TOL32 * diag(m)
        if ordering == lms.RDR:
            for i, m in enumerate(meshes):
                assert np.array_equal(perms[i], oracle.order(m, oracle.RDR))


def test_layout_keeps_coordinates_and_run_path():
    meshes = small_batch()[:8]
    xy = np.concatenate([m["xy"] for m in meshes])
    with lms.Batch(meshes, ordering=lms.RDR) as b:
        b.set_config(lms.KERNEL_DIRECT, 128, 5, 512)
        b.smooth(9)
        before = b.all_coords()
        b.set_layout(128)
        assert np.array_equal(b.all_coords(), before)  # the held coordinates move with the layout
        b.smooth(11)
        mid = b.all_coords()
        b.set_layout(0)
        b.smooth(0)
        assert np.array_equal(b.all_coords(), mid)
        b.set_layout(64)
        got = b.run(xy, 20, groups=3)
    with lms.Batch(meshes, ordering=lms.RDR) as b0:
        b0.set_config(lms.KERNEL_DIRECT, 128, 5, 512)
        want = b0.run(xy, 20, groups=3)
    assert np.array_equal(got, want)
    assert np.array_equal(mid, want)


def test_layout_rejects_bad_windows():
    with lms.Batch(small_batch()[:2], ordering=lms.ORI) as b:
        for w in (-32, 31, 48, 65536 + 32):
            with pytest.raises(lms.LmsError):
                b.set_layout(w)
        assert b.layout() == 0
