"""Parity of drc_indirect (the indirect term of Eq. 3 by multiple importance
sampling between the blended cached maps and the BRDF, Sec. 3.2; plus the
emission and direct terms) with the FP64 oracle, through the C ABI.

The uniforms are an input, so both sides draw the same samples.  The map
and the environment texel are chosen from running float32 sums that both
sides form alike.  The other discrete decisions come from continuous values
(the texel a direction falls in, the hemisphere tests, the frame's up
vector); the oracle reports per pixel how close they came to a boundary in
units of their float32 error, and pixels below 1 (where fp32 may rightly
decide the other way) are left out and counted."""
import numpy as np
import pytest

import oracle
from paper_1910_02480_gb300 import synth
from parity import FP32_TOL, rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
MARGIN = 1.0


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


def _skewed_maps(rng, n, H, W, zero_frac=0.2):
    maps = rng.gamma(0.5, 1.0, size=(n, 3, H, W))
    maps[rng.uniform(size=maps.shape) < zero_frac] = 0.0
    return maps.astype(np.float32)


def _scene(width, height, gx, gy, k, H, W, seed=2, maps="skewed"):
    """A G-buffer, its cache grid with maps, and each pixel's k nearest
    caches with their normalised weights (from the oracle's interpolation,
    rounded to float32 -- the inputs both sides receive)."""
    g = synth.gbuffer(width, height, seed=seed)
    c = synth.cache_grid(g, gx, gy)
    n = gx * gy
    rng = np.random.default_rng(seed + 7)
    if maps == "skewed":
        c["maps"] = _skewed_maps(rng, n, H, W)
    else:  # the lobe field, decoded to linear radiance
        x, _ = synth.hemisphere_maps(c["pos"], c["nrm"], H=H, W=W, seed=seed + 1)
        c["maps"] = np.ascontiguousarray(np.expm1(np.clip(x[:, :3], 0.0, None)), dtype=np.float32)
    c["payload"] = np.zeros((n, 3), np.float32)
    r = synth.world_radius(n)
    _, idx, _, wts = oracle.interpolate(c, g, k, oracle.METRIC_WORLD, oracle.WP_INVERSE,
                                        oracle.INTERP_IRRADIANCE, r, want_neighbors=True, want_weights=True)
    P = width * height
    alb = rng.uniform(0.2, 0.9, size=(P, 3)).astype(np.float32)
    return g, c, idx.astype(np.int32), wts.astype(np.float32), alb


def _uniforms(P, S, seed):
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=(P, S, 4)).astype(np.float32)


def _gpu(ctx, c, g, idx, wts, u, alb, emit=None, direct=None):
    out = ctx.indirect(_cuda(c["maps"]), _cuda(c["nrm"]), _cuda(g["nrm"]), g["width"], g["height"],
                       _cuda(idx, np.int32), _cuda(wts), _cuda(u), _cuda(alb),
                       emit=None if emit is None else _cuda(emit), direct=None if direct is None else _cuda(direct))
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _check(got, ref, margin, min_kept=0.98):
    ok = margin > MARGIN
    assert ok.mean() >= min_kept, ok.mean()
    err = rel_err(got[ok], ref[ok])
    print("indirect: %d of %d pixels compared, max rel %.3e" % (ok.sum(), ok.size, err))
    assert err <= FP32_TOL


@pytest.mark.parametrize("S", [1, 2, 5, 8])
@pytest.mark.parametrize("k", [1, 4, 8])
def test_indirect_matches_oracle(drc, ctx, S, k):
    g, c, idx, wts, alb = _scene(48, 32, 6, 4, k, 16, 16)
    u = _uniforms(48 * 32, S, seed=S + 10 * k)
    got = _gpu(ctx, c, g, idx, wts, u, alb)
    assert ctx.status() == drc.OK
    ref, margin = oracle.mis_indirect(c, idx, wts, g["nrm"], alb, u, want_margin=True)
    _check(got, ref, margin)


def test_emission_and_direct_are_added(drc, ctx):
    """Eq. 3: L_o = L_e + the indirect integral + the direct integral."""
    g, c, idx, wts, alb = _scene(40, 24, 5, 4, 6, 8, 16)
    P = 40 * 24
    rng = np.random.default_rng(3)
    emit = rng.uniform(0.0, 0.5, size=(P, 3)).astype(np.float32)
    direct = rng.uniform(0.0, 2.0, size=(P, 3)).astype(np.float32)
    u = _uniforms(P, 6, seed=4)
    got = _gpu(ctx, c, g, idx, wts, u, alb, emit=emit, direct=direct)
    ref, margin = oracle.mis_indirect(c, idx, wts, g["nrm"], alb, u, want_margin=True)
    _check(got, ref + emit.astype(np.float64) + direct.astype(np.float64), margin)


def test_degenerate_maps_normals_and_missing_neighbours(drc, ctx):
    """Black maps (no environment distribution), caches with zero normals,
    pixels with zero normals, and neighbour slots marked -1."""
    g, c, idx, wts, alb = _scene(32, 32, 4, 4, 5, 8, 8)
    c["maps"][3] = 0.0
    c["nrm"][5] = 0.0
    g = dict(g, nrm=g["nrm"].copy())
    g["nrm"][7::50] = 0.0
    idx = idx.copy()
    wts = wts.copy()
    idx[::3, -1] = -1  # fewer neighbours: renormalise the rest
    wts[::3, -1] = 0.0
    wts /= wts.sum(axis=1, keepdims=True)
    u = _uniforms(32 * 32, 7, seed=5)
    got = _gpu(ctx, c, g, idx, wts, u, alb)
    ref, margin = oracle.mis_indirect(c, idx, wts, g["nrm"], alb, u, want_margin=True)
    _check(got, ref, margin)
    assert np.all(got[7::50] == 0.0)


def test_neighbours_and_weights_from_interpolation(drc, ctx):
    """drc_interpolate's neighbour list and normalised weights feed
    drc_indirect: the weights match the oracle's, and the estimate from the
    GPU's own neighbours matches the oracle given the same ones."""
    g, c, idx_o, w_o, alb = _scene(64, 48, 8, 6, 8, 16, 16)
    P, k = 64 * 48, 8
    r = synth.world_radius(48)
    gd = {"width": 64, "height": 48, "pos": _cuda(g["pos"]), "nrm": _cuda(g["nrm"])}
    cd = {"pos": _cuda(c["pos"]), "nrm": _cuda(c["nrm"]), "pix": _cuda(c["pix"], np.int32),
          "payload": _cuda(c["payload"])}
    nbr = torch.empty((P, k), dtype=torch.int32, device="cuda")
    nw = torch.empty((P, k), dtype=torch.float32, device="cuda")
    ctx.interpolate(cd, gd, k, drc.METRIC_WORLD, drc.WP_INVERSE, drc.INTERP_IRRADIANCE, r, nbr_out=nbr, nbr_w=nw)
    torch.cuda.synchronize()
    nbr, nw = nbr.cpu().numpy(), nw.cpu().numpy()
    same = np.all(nbr == idx_o, axis=1)
    assert same.mean() > 0.99
    np.testing.assert_allclose(nw[same], w_o[same], rtol=2e-6, atol=1e-7)
    np.testing.assert_allclose(nw.sum(axis=1), 1.0, rtol=1e-6)
    u = _uniforms(P, 8, seed=6)
    got = _gpu(ctx, c, g, nbr, nw, u, alb)
    ref, margin = oracle.mis_indirect(c, nbr, nw, g["nrm"], alb, u, want_margin=True)
    _check(got, ref, margin)


def test_full_size_sampled(drc, ctx):
    """1920x1080 pixels, 64x64 caches with 32x32 maps of the lobe field,
    k = 16, S = 8: the whole frame on the GPU, three row bands by the
    oracle."""
    W_, H_ = 1920, 1080
    g = synth.gbuffer(W_, H_, seed=2)
    c = synth.cache_grid(g, 64, 64)
    x, _ = synth.hemisphere_maps(c["pos"], c["nrm"], H=32, W=32, seed=3)
    c["maps"] = np.ascontiguousarray(np.expm1(np.clip(x[:, :3], 0.0, None)), dtype=np.float32)
    c["payload"] = np.zeros((4096, 3), np.float32)
    k, S, P = 16, 8, W_ * H_
    gd = {"width": W_, "height": H_, "pos": _cuda(g["pos"]), "nrm": _cuda(g["nrm"])}
    cd = {"pos": _cuda(c["pos"]), "nrm": _cuda(c["nrm"]), "pix": _cuda(c["pix"], np.int32),
          "payload": _cuda(c["payload"])}
    nbr = torch.empty((P, k), dtype=torch.int32, device="cuda")
    nw = torch.empty((P, k), dtype=torch.float32, device="cuda")
    ctx.interpolate(cd, gd, k, drc.METRIC_WORLD, drc.WP_INVERSE, drc.INTERP_IRRADIANCE,
                    synth.world_radius(4096), nbr_out=nbr, nbr_w=nw)
    rng = np.random.default_rng(8)
    alb = rng.uniform(0.2, 0.9, size=(P, 3)).astype(np.float32)
    u = _uniforms(P, S, seed=9)
    out = ctx.indirect(_cuda(c["maps"]), cd["nrm"], gd["nrm"], W_, H_, nbr, nw, _cuda(u), _cuda(alb))
    torch.cuda.synchronize()
    assert ctx.status() == drc.OK
    out, nbr, nw = out.cpu().numpy(), nbr.cpu().numpy(), nw.cpu().numpy()
    assert np.all(np.isfinite(out))
    for p0 in (0, 1920 * 540 + 3, P - 2048):
        sl = slice(p0, p0 + 2048)
        ref, margin = oracle.mis_indirect(c, nbr[sl], nw[sl], g["nrm"][sl], alb[sl], u[sl], want_margin=True)
        _check(out[sl], ref, margin)


def test_indirect_argument_errors(drc, ctx):
    g, c, idx, wts, alb = _scene(8, 8, 2, 2, 2, 8, 8)
    u = _uniforms(64, 2, seed=1)
    with pytest.raises(drc.DrcError):  # S = 0
        ctx.indirect(_cuda(c["maps"]), _cuda(c["nrm"]), _cuda(g["nrm"]), 8, 8, _cuda(idx, np.int32), _cuda(wts),
                     _cuda(u[:, :0]), _cuda(alb))
    with pytest.raises(drc.DrcError):  # host memory
        ctx.indirect(_cuda(c["maps"]), _cuda(c["nrm"]), torch.from_numpy(g["nrm"]), 8, 8, _cuda(idx, np.int32),
                     _cuda(wts), _cuda(u), _cuda(alb))
