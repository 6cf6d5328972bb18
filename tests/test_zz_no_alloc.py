"""drc_interpolate_static: the interpolation for callers that cannot allocate
device memory (a host application that owns the memory budget, or a frame
loop where cudaMalloc's implicit synchronisation is not allowed).  It keeps
its cache grid in a static device array instead of a context's buffer.

Checked through the C ABI against drc_interpolate, on calls in a row with
different scenes (small, large, small), so that anything left in the shared
array by one call would show in the next.  This file is collected last on
purpose."""
import ctypes

import numpy as np
import pytest

from paper_1910_02480_gb300 import synth
from parity import FP32_TOL, rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def drc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_02480_gb300 import build
    build.build()
    import paper_1910_02480_gb300 as m
    return m


def _scene(width, height, gx, gy, seed, maps=False):
    g = synth.gbuffer(width, height, seed=seed)
    c = synth.cache_grid(g, gx, gy)
    rng = np.random.default_rng(seed + 1)
    c["payload"] = rng.uniform(0.0, 2.0, size=(gx * gy, 3)).astype(np.float32)
    if maps:
        c["maps"] = rng.uniform(0.0, 3.0, size=(gx * gy, 3, 8, 8)).astype(np.float32)
    return ({k: torch.from_numpy(v).cuda() if isinstance(v, np.ndarray) else v for k, v in g.items()},
            {k: torch.from_numpy(v).cuda() for k, v in c.items()})


def _static_call(drc, caches, gbuf, k, metric, wp, mode, r, out, nbr):
    lib = drc.load_library()
    c = drc.Caches()
    c.n = int(caches["nrm"].shape[0])
    m = caches.get("maps")
    c.H, c.W = (int(m.shape[2]), int(m.shape[3])) if m is not None else (0, 0)
    c.maps = ctypes.c_void_p(m.data_ptr()) if m is not None else None
    c.payload = ctypes.c_void_p(caches["payload"].data_ptr())
    c.pos = ctypes.c_void_p(caches["pos"].data_ptr())
    c.nrm = ctypes.c_void_p(caches["nrm"].data_ptr())
    c.pix = ctypes.c_void_p(caches["pix"].data_ptr())
    g = drc.GBuffer()
    g.width, g.height = gbuf["width"], gbuf["height"]
    g.pos = ctypes.c_void_p(gbuf["pos"].data_ptr())
    g.nrm = ctypes.c_void_p(gbuf["nrm"].data_ptr())
    g.dir = ctypes.c_void_p(gbuf["dir"].data_ptr())
    p = drc.InterpParams()
    p.k, p.metric, p.wp_form, p.mode = k, metric, wp, mode
    p.r, p.eps, p.delta_rel = r, 1e-6, 1e-3
    p.nbr_out = ctypes.c_void_p(nbr.data_ptr()) if nbr is not None else None
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.drc_interpolate_static(ctypes.byref(c), ctypes.byref(g), ctypes.byref(p),
                                      ctypes.c_void_p(out.data_ptr()), stream)


def test_static_matches_context_entry_point_on_two_calls(drc):
    """Three calls in a row -- small, large, small -- so that the large call
    carves a bigger grid than the one before it and the last small call reads
    an array the large one left behind; with and without the neighbour list
    (the list takes the exact walk, its absence the two-walk query)."""
    ctx = drc.Context([16], synth.he_weights([16]), precision="fp32")
    small_image = (_scene(96, 64, 6, 4, seed=9, maps=True), 8, drc.METRIC_IMAGE, drc.WP_LINEAR,
                   drc.INTERP_LOOKUP, synth.image_radius(96, 64, 6, 4))
    large_world = (_scene(192, 128, 24, 16, seed=5), 16, drc.METRIC_WORLD, drc.WP_INVERSE,
                   drc.INTERP_IRRADIANCE, synth.world_radius(24 * 16))
    small_world = (_scene(64, 48, 6, 6, seed=11), 8, drc.METRIC_WORLD, drc.WP_INVERSE,
                   drc.INTERP_IRRADIANCE, synth.world_radius(36))
    for want_nbr in (True, False):
        for (gbuf, caches), k, metric, wp, mode, r in (small_image, large_world, small_world):
            P = gbuf["width"] * gbuf["height"]
            ref_nbr = torch.empty((P, k), dtype=torch.int32, device="cuda") if want_nbr else None
            ref = ctx.interpolate(caches, gbuf, k, metric, wp, mode, r, nbr_out=ref_nbr)
            out = torch.full((P, 3), float("nan"), device="cuda")
            nbr = torch.full((P, k), -7, dtype=torch.int32, device="cuda") if want_nbr else None
            rc = _static_call(drc, caches, gbuf, k, metric, wp, mode, r, out, nbr)
            assert rc == drc.OK
            torch.cuda.synchronize()
            assert ctx.status() == drc.OK
            if want_nbr:
                np.testing.assert_array_equal(nbr.cpu().numpy(), ref_nbr.cpu().numpy())
            assert rel_err(out.cpu().numpy(), ref.cpu().numpy()) <= FP32_TOL


def test_static_call_allocates_nothing(drc):
    """After a warm-up call, a further call changes neither the device's free
    memory nor the allocator's counters."""
    (gbuf, caches) = _scene(192, 128, 24, 16, seed=5)
    P = gbuf["width"] * gbuf["height"]
    out = torch.empty((P, 3), device="cuda")
    r = synth.world_radius(24 * 16)
    assert _static_call(drc, caches, gbuf, 16, drc.METRIC_WORLD, drc.WP_INVERSE, drc.INTERP_IRRADIANCE,
                        r, out, None) == drc.OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for _ in range(3):
        assert _static_call(drc, caches, gbuf, 16, drc.METRIC_WORLD, drc.WP_INVERSE,
                            drc.INTERP_IRRADIANCE, r, out, None) == drc.OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == stats0


def test_static_rejects_more_caches_than_its_array_holds(drc):
    gbuf, caches = _scene(16, 16, 4, 4, seed=3)
    lib = drc.load_library()
    c = drc.Caches()
    c.n = 65537
    c.nrm = ctypes.c_void_p(caches["nrm"].data_ptr())
    c.pos = ctypes.c_void_p(caches["pos"].data_ptr())
    c.payload = ctypes.c_void_p(caches["payload"].data_ptr())
    g = drc.GBuffer()
    g.width, g.height = 16, 16
    g.pos = ctypes.c_void_p(gbuf["pos"].data_ptr())
    g.nrm = ctypes.c_void_p(gbuf["nrm"].data_ptr())
    p = drc.InterpParams()
    p.k, p.metric, p.wp_form, p.mode, p.r, p.eps, p.delta_rel = 4, drc.METRIC_WORLD, 0, 0, 0.3, 1e-6, 1e-3
    out = torch.empty((256, 3), device="cuda")
    rc = lib.drc_interpolate_static(ctypes.byref(c), ctypes.byref(g), ctypes.byref(p),
                                    ctypes.c_void_p(out.data_ptr()), None)
    assert rc == drc.ERR_INVALID_ARG
