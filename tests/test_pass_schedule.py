"""The progressive-refinement schedule (Sec. 3.2: after each pass the
distance between the grid's sample points shrinks by a constant factor,
read as 2, the points already evaluated kept): drc_pass_points, a host-only
call of the C ABI, needs no GPU."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def drc():
    from paper_1910_02480_gb300 import build
    build.build()
    import paper_1910_02480_gb300 as m
    return m


def _grid(width, height, s):
    ys, xs = np.meshgrid(np.arange(0, height, s), np.arange(0, width, s), indexing="ij")
    return set(zip(xs.ravel().tolist(), ys.ravel().tolist()))


@pytest.mark.parametrize("width,height,s0", [(1920, 1080, 64), (37, 29, 8), (16, 16, 16), (5, 3, 1)])
def test_passes_partition_the_halving_grids(drc, width, height, s0):
    seen = set()
    t = 0
    while True:
        pts = drc.pass_points(width, height, s0, t)
        s = s0 >> t
        if s < 1:
            assert len(pts) == 0  # finer than every pixel: nothing new
            break
        cur = set(map(tuple, pts.tolist()))
        assert len(cur) == len(pts)            # no point twice within a pass
        assert not (cur & seen)                # nor in two passes
        seen |= cur
        assert seen == _grid(width, height, s)  # passes 0..t: exactly the grid of spacing s_t
        if t > 0:
            assert all(not (x % (2 * s) == 0 and y % (2 * s) == 0) for x, y in cur)
        # row-major order of (y, x)
        assert np.all(np.diff(pts[:, 1] * width + pts[:, 0]) > 0) if len(pts) > 1 else True
        t += 1
    assert seen == _grid(width, height, 1)


def test_pass_counts_1080p(drc):
    """1920 x 1080 from a 64-pixel grid: 30 x 17 points, then three quarters
    of each finer grid's points are new."""
    counts = [len(drc.pass_points(1920, 1080, 64, t)) for t in range(4)]
    assert counts == [30 * 17, 60 * 34 - 30 * 17, 120 * 68 - 60 * 34, 240 * 135 - 120 * 68]


def test_pass_points_argument_errors(drc):
    import ctypes
    lib = drc.load_library()
    cnt = ctypes.c_int(-1)
    assert lib.drc_pass_points(64, 64, 12, 0, None, 0, ctypes.byref(cnt)) == drc.ERR_INVALID_ARG  # not a power of 2
    assert lib.drc_pass_points(0, 64, 8, 0, None, 0, ctypes.byref(cnt)) == drc.ERR_INVALID_ARG
    assert lib.drc_pass_points(64, 64, 8, -1, None, 0, ctypes.byref(cnt)) == drc.ERR_INVALID_ARG
    assert lib.drc_pass_points(64, 64, 8, 0, None, 0, None) == drc.ERR_INVALID_ARG
    # too small an output array: the count is still reported
    buf = (ctypes.c_int * 2)()
    assert lib.drc_pass_points(64, 64, 8, 0, buf, 1, ctypes.byref(cnt)) == drc.ERR_INVALID_ARG
    assert cnt.value == 64
