"""Parity of drc_interpolate (k-nearest caches, w = w_p w_n + w_p + eps,
normalised blend; Sec. 3.2) with the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
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


@pytest.fixture(scope="module")
def ctx(drc):
    return drc.Context([16], synth.he_weights([16]), precision="fp32")


def _scene(width, height, gx, gy, with_maps=False, seed=2, H=16, W=16):
    g = synth.gbuffer(width, height, seed=seed)
    c = synth.cache_grid(g, gx, gy)
    rng = np.random.default_rng(seed + 1)
    n = gx * gy
    c["payload"] = rng.uniform(0.0, 2.0, size=(n, 3)).astype(np.float32)
    if with_maps:
        c["maps"] = rng.uniform(0.0, 3.0, size=(n, 3, H, W)).astype(np.float32)
    return g, c


def _cuda(d):
    out = {}
    for k, v in d.items():
        out[k] = torch.from_numpy(np.ascontiguousarray(v)).cuda() if isinstance(v, np.ndarray) else v
    return out


def _ambiguous(d2, k, rel=1e-5):
    """Pixels whose k-th and (k+1)-th squared distances are too close for a
    float32 evaluation to order them the way the float64 oracle does."""
    a, b = d2[:, k - 1], d2[:, k]
    return np.abs(b - a) <= rel * np.maximum(b, 1e-30)


def _run(drc, ctx, g, c, k, metric, wp, mode, r, p_range=None):
    P = g["width"] * g["height"]
    nbr = torch.empty((P, k), dtype=torch.int32, device="cuda")
    out = ctx.interpolate(_cuda(c), _cuda(g), k, metric, wp, mode, r, nbr_out=nbr)
    torch.cuda.synchronize()
    assert ctx.status() == drc.OK
    ref, idx, d2 = oracle.interpolate(c, g, k, metric, wp, mode, r, p_range=p_range, want_neighbors=True)
    p0, p1 = p_range if p_range else (0, P)
    return out.cpu().numpy()[p0:p1], nbr.cpu().numpy()[p0:p1], ref, idx, d2


@pytest.mark.parametrize("k", [1, 8, 16])
@pytest.mark.parametrize("wp", [0, 1])
def test_image_metric_is_exact(drc, ctx, k, wp):
    """IMAGE distances are integers: the selection is bit-exact, including
    ties (broken by cache index)."""
    g, c = _scene(128, 128, 8, 8)
    r = synth.image_radius(128, 128, 8, 8)
    out, nbr, ref, idx, _ = _run(drc, ctx, g, c, k, drc.METRIC_IMAGE, wp, drc.INTERP_IRRADIANCE, r)
    np.testing.assert_array_equal(nbr, idx)
    assert rel_err(out, ref) <= FP32_TOL


@pytest.mark.parametrize("k", [1, 4, 16, 32])
def test_world_metric(drc, ctx, k):
    g, c = _scene(96, 64, 16, 12)
    r = synth.world_radius(16 * 12)
    out, nbr, ref, idx, d2 = _run(drc, ctx, g, c, k, drc.METRIC_WORLD, drc.WP_INVERSE,
                                  drc.INTERP_IRRADIANCE, r)
    amb = _ambiguous(d2, k) if k < 16 * 12 else np.zeros(len(out), bool)
    ok = ~amb
    assert ok.mean() > 0.99
    np.testing.assert_array_equal(np.sort(nbr[ok], axis=1), np.sort(idx[ok], axis=1))
    assert rel_err(out[ok], ref[ok]) <= FP32_TOL


@pytest.mark.parametrize("metric", [0, 1])
def test_lookup_mode(drc, ctx, metric):
    g, c = _scene(64, 48, 8, 6, with_maps=True)
    k = 8
    r = synth.image_radius(64, 48, 8, 6) if metric == 0 else synth.world_radius(48)
    out, nbr, ref, idx, d2 = _run(drc, ctx, g, c, k, metric, drc.WP_INVERSE, drc.INTERP_LOOKUP, r)
    ok = ~_ambiguous(d2, k) if metric == 1 else np.ones(len(out), bool)
    # directions grazing a cache's horizon switch its contribution on or off
    n = c["nrm"].astype(np.float64)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    d = g["dir"].astype(np.float64)
    lz = np.einsum("pc,pkc->pk", d, n[idx])
    ok &= ~np.any(np.abs(lz) < 1e-5, axis=1)
    assert ok.mean() > 0.99
    np.testing.assert_array_equal(np.sort(nbr[ok], axis=1), np.sort(idx[ok], axis=1))
    assert rel_err(out[ok], ref[ok]) <= FP32_TOL


def test_constant_payload_reproduced(drc, ctx):
    g, c = _scene(64, 64, 8, 8)
    c["payload"] = np.tile(np.float32([0.25, 1.5, 3.0]), (64, 1))
    out = ctx.interpolate(_cuda(c), _cuda(g), 8, drc.METRIC_WORLD, drc.WP_INVERSE,
                          drc.INTERP_IRRADIANCE, 0.2)
    np.testing.assert_allclose(out.cpu().numpy(), np.tile([0.25, 1.5, 3.0], (64 * 64, 1)), rtol=3e-6)


def test_fewer_caches_than_k(drc, ctx):
    g, c = _scene(16, 16, 2, 1)
    out, nbr, ref, idx, _ = _run(drc, ctx, g, c, 4, drc.METRIC_IMAGE, drc.WP_INVERSE,
                                 drc.INTERP_IRRADIANCE, 8.0)
    np.testing.assert_array_equal(nbr, idx)
    assert rel_err(out, ref) <= FP32_TOL


def test_full_size_world_sampled(drc, ctx):
    """1920x1080 G-buffer, 64x64 caches, k = 16, WORLD metric: the whole
    frame on the GPU, three row bands recomputed by the oracle."""
    g, c = _scene(1920, 1080, 64, 64)
    k = 16
    r = synth.world_radius(4096)
    P = 1920 * 1080
    nbr = torch.empty((P, k), dtype=torch.int32, device="cuda")
    out = ctx.interpolate(_cuda(c), _cuda(g), k, drc.METRIC_WORLD, drc.WP_INVERSE,
                          drc.INTERP_IRRADIANCE, r, nbr_out=nbr)
    torch.cuda.synchronize()
    assert ctx.status() == drc.OK
    out, nbr = out.cpu().numpy(), nbr.cpu().numpy()
    for p0 in (0, 1920 * 540 + 7, P - 4096):
        p1 = p0 + 4096
        ref, idx, d2 = oracle.interpolate(c, g, k, drc.METRIC_WORLD, drc.WP_INVERSE,
                                          drc.INTERP_IRRADIANCE, r, p_range=(p0, p1), want_neighbors=True)
        ok = ~_ambiguous(d2, k)
        np.testing.assert_array_equal(np.sort(nbr[p0:p1][ok], axis=1), np.sort(idx[ok], axis=1))
        assert rel_err(out[p0:p1][ok], ref[ok]) <= FP32_TOL


def test_interp_argument_errors(drc, ctx):
    g, c = _scene(16, 16, 4, 4)
    with pytest.raises(drc.DrcError):
        ctx.interpolate(_cuda(c), _cuda(g), 0, drc.METRIC_IMAGE, 0, 0, 4.0)
    with pytest.raises(drc.DrcError):
        ctx.interpolate(_cuda(c), _cuda(g), 33, drc.METRIC_IMAGE, 0, 0, 4.0)
    with pytest.raises(drc.DrcError):
        ctx.interpolate(_cuda(c), _cuda(g), 4, drc.METRIC_IMAGE, 0, 0, -1.0)
    with pytest.raises(drc.DrcError):
        ctx.interpolate(_cuda(c), _cuda(g), 4, drc.METRIC_IMAGE, 0, drc.INTERP_LOOKUP, 4.0)


def test_empty_and_single_pixel_gbuffer(drc, ctx):
    """P = 0 enqueues nothing and leaves the output alone; a 1 x 1 G-buffer
    (one pixel, every cache a candidate) matches the oracle."""
    g, c = _scene(16, 16, 4, 4)
    r = synth.world_radius(16)
    g0 = dict(g)
    g0["width"], g0["height"] = 0, 0
    g0["pos"], g0["nrm"] = g["pos"][:0], g["nrm"][:0]
    out0 = torch.full((1, 3), 7.0, device="cuda")
    ctx.interpolate(_cuda(c), _cuda(g0), 4, drc.METRIC_WORLD, drc.WP_INVERSE, drc.INTERP_IRRADIANCE, r, out=out0)
    torch.cuda.synchronize()
    assert ctx.status() == drc.OK and bool(torch.all(out0 == 7.0))
    g1 = dict(g)
    g1["width"], g1["height"] = 1, 1
    g1["pos"], g1["nrm"] = np.ascontiguousarray(g["pos"][5:6]), np.ascontiguousarray(g["nrm"][5:6])
    out, nbr, ref, idx, d2 = _run(drc, ctx, g1, c, 16, drc.METRIC_WORLD, drc.WP_INVERSE, drc.INTERP_IRRADIANCE, r)
    np.testing.assert_array_equal(np.sort(nbr, axis=1), np.sort(idx, axis=1))  # k = n: every cache
    assert rel_err(out, ref) <= FP32_TOL
