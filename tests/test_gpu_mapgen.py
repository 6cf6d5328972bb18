"""Parity of drc_gen_maps (the denoiser's input maps traced from cache
points in an analytic interior: radiance without the first hit's emission,
distance, normal; Sec. 3.1-3.3) with the FP64 oracle, through the C ABI.

The uniforms are an input, so both sides trace the same paths.  A path's
discrete decisions (which surface is nearest, whether a ceiling hit lies on
the light, whether a ray meets a sphere) come from continuous values; the
oracle reports per texel how close they came to changing, in units of their
float32 error, and texels below 1 are left out and counted."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1910_02480_gb300 import synth
from parity import FP32_TOL, rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# the room: coloured walls, a faint glow on every wall, a ceiling light and
# three spheres -- all float32 values, given to both sides alike
ALB = np.float32([[0.7, 0.2, 0.2], [0.2, 0.7, 0.2], [0.6, 0.6, 0.6], [0.6, 0.6, 0.5], [0.5, 0.5, 0.5],
                  [0.8, 0.8, 0.8]])
EM = np.float32(np.full((6, 3), 0.05))
LIGHT = np.float32([0.3, 0.7, 0.35, 0.65, 8.0, 7.5, 6.0])
SPH = np.float32([[0.3, 0.3, 0.25, 0.15, 0.9, 0.8, 0.3], [0.7, 0.6, 0.3, 0.2, 0.3, 0.5, 0.9],
                  [0.55, 0.25, 0.7, 0.1, 0.8, 0.8, 0.8]])


@pytest.fixture(scope="module")
def drc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_02480_gb300 import build
    build.build()
    import paper_1910_02480_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(drc):
    return drc.Context([16], synth.he_weights([16]), precision="fp32")


def _cuda(a, dtype=np.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def _caches(n, seed):
    """Cache points strictly inside the box, outside the spheres, normals
    uniform on the sphere."""
    rng = np.random.default_rng(seed)
    pos = []
    while len(pos) < n:
        p = rng.uniform(0.03, 0.97, size=3)
        if all(np.linalg.norm(p - s[:3]) > s[3] + 1e-3 for s in SPH):
            pos.append(p)
    nrm = rng.standard_normal((n, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    return np.float32(pos), np.float32(nrm)


def _compare(got, ref, margin, min_kept=0.99):
    ok = margin >= 1.0  # [n, H, W]
    assert ok.mean() >= min_kept, ok.mean()
    g = np.moveaxis(got, 1, -1)[ok]  # [texels, 7]
    r = np.moveaxis(ref, 1, -1)[ok]
    e_rad = rel_err(g[:, :3], r[:, :3])
    e_dist = rel_err(g[:, 3], r[:, 3])
    e_nrm = float(np.max(np.abs(g[:, 4:] - r[:, 4:])))
    print("gen maps: %d of %d texels compared; radiance %.2e, distance %.2e, normal abs %.2e"
          % (ok.sum(), ok.size, e_rad, e_dist, e_nrm))
    assert e_rad <= FP32_TOL and e_dist <= FP32_TOL and e_nrm <= 1e-5


@pytest.mark.parametrize("D", [0, 1, 3, 5])
def test_room_matches_oracle(drc, ctx, D):
    n, H, W = 48, 16, 16
    pos, nrm = _caches(n, seed=D + 1)
    u = np.random.default_rng(10 + D).uniform(size=(n, H, W, max(D, 1), 2)).astype(np.float32)[:, :, :, :D]
    sc = drc.make_scene(ALB, EM, LIGHT, SPH)
    got = ctx.gen_maps(sc, _cuda(pos), _cuda(nrm), H, W, u=_cuda(u) if D else None)
    torch.cuda.synchronize()
    assert ctx.status() == drc.OK
    ref, margin = oracle.gen_maps(pos, nrm, H, W, ALB, EM, LIGHT, SPH, D=D,
                                  u=u if D else None, want_margin=True)
    _compare(got.cpu().numpy(), ref, margin)


def test_furnace_closed_form(drc, ctx):
    """Every wall emits Le with albedo rho: any D-bounce path brings
    sum_{i=1..D} rho^i Le, whatever the directions."""
    n, H, W, D = 16, 8, 12, 4
    pos, nrm = _caches(n, seed=3)
    le = np.float32([1.0, 0.5, 0.25])
    rho = np.float32([0.5, 0.3, 0.7])
    u = np.random.default_rng(4).uniform(size=(n, H, W, D, 2)).astype(np.float32)
    sc = drc.make_scene(np.tile(rho, (6, 1)), np.tile(le, (6, 1)))
    got = ctx.gen_maps(sc, _cuda(pos), _cuda(nrm), H, W, u=_cuda(u)).cpu().numpy()
    expect = sum(rho.astype(np.float64) ** i * le.astype(np.float64) for i in range(1, D + 1))
    np.testing.assert_allclose(np.moveaxis(got[:, :3], 1, -1), np.broadcast_to(expect, (n, H, W, 3)), rtol=2e-6)


def test_full_size_sampled_and_denoised(drc, ctx):
    """4096 caches (the benchmark's 64 x 64 grid of a 1920 x 1080 G-buffer,
    points pulled inside the box) of 32 x 32 maps, 3 bounces: the whole
    batch on the GPU, 24 caches spread over it by the oracle; the maps then
    go through the benchmark network (log encode on input)."""
    g = synth.gbuffer(1920, 1080, seed=2)
    c = synth.cache_grid(g, 64, 64)
    pos = np.float32(0.02 + 0.96 * c["pos"].astype(np.float64))
    nrm = c["nrm"]
    n, H, W, D = 4096, 32, 32, 3
    u = np.random.default_rng(5).uniform(size=(n, H, W, D, 2)).astype(np.float32)
    sc = drc.make_scene(ALB, EM, LIGHT, SPH)
    got = ctx.gen_maps(sc, _cuda(pos), _cuda(nrm), H, W, u=_cuda(u))
    torch.cuda.synchronize()
    assert ctx.status() == drc.OK
    idx = np.linspace(0, n - 1, 24).astype(int)
    # caches inside a sphere see nothing from outside: keep those the oracle takes
    ref, margin = oracle.gen_maps(pos[idx], nrm[idx], H, W, ALB, EM, LIGHT, SPH, D=D, u=u[idx], want_margin=True)
    _compare(got.cpu().numpy()[idx], ref, margin)
    widths = [64, 128, 256]
    net = drc.Context(widths, synth.he_weights(widths, seed=0), precision="fp32")
    out, pay = net.denoise(got, flags=drc.F_ENCODE_INPUT | drc.F_DECODE_OUTPUT, want_payload=True)
    torch.cuda.synchronize()
    assert net.status() == drc.OK
    assert out.shape == (n, 3, H, W) and bool(torch.isfinite(out).all()) and bool(torch.isfinite(pay).all())


def test_gen_maps_argument_errors(drc, ctx):
    pos, nrm = _caches(2, seed=1)
    sc = drc.make_scene(ALB)
    out = torch.empty((2, 7, 4, 4), device="cuda")
    pd, nd = _cuda(pos), _cuda(nrm)
    lib = drc.load_library()
    # D = 2 bounces without uniforms
    rc = lib.drc_gen_maps(ctx._ctx, ctypes.byref(sc), 2, ctypes.c_void_p(pd.data_ptr()),
                          ctypes.c_void_p(nd.data_ptr()), 4, 4, 2, None, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == drc.ERR_INVALID_ARG
    sc.nsph = 65
    rc = lib.drc_gen_maps(ctx._ctx, ctypes.byref(sc), 2, ctypes.c_void_p(pd.data_ptr()),
                          ctypes.c_void_p(nd.data_ptr()), 4, 4, 0, None, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == drc.ERR_INVALID_ARG
    with pytest.raises(drc.DrcError):  # host memory
        ctx.gen_maps(drc.make_scene(ALB), torch.from_numpy(pos), nd, 4, 4)
