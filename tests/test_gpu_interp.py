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


@pytest.mark.parametrize("mode", [0, 1])
def test_full_size_world_fast_sampled(drc, ctx, mode):
    """Exactly what the benchmark times: 1920x1080 G-buffer, 64x64 caches,
    k = 16, WORLD metric, no neighbour list (the fast query), IRRADIANCE or
    LOOKUP (32x32 maps); four row bands recomputed by the oracle, ambiguous
    and horizon-grazing pixels excluded."""
    g, c = _scene(1920, 1080, 64, 64, with_maps=mode == 1, H=32, W=32)
    k = 16
    r = synth.world_radius(4096)
    P = 1920 * 1080
    out = ctx.interpolate(_cuda(c), _cuda(g), k, drc.METRIC_WORLD, drc.WP_INVERSE, mode, r)
    torch.cuda.synchronize()
    assert ctx.status() == drc.OK
    out = out.cpu().numpy()
    assert np.all(np.isfinite(out))
    for p0 in (0, 1920 * 300 + 11, 1920 * 540 + 7, P - 3072):
        p1 = p0 + 3072
        ref, idx, d2 = oracle.interpolate(c, g, k, drc.METRIC_WORLD, drc.WP_INVERSE, mode, r,
                                          p_range=(p0, p1), want_neighbors=True)
        ok = ~_ambiguous(d2, k)
        if mode == 1:
            ok &= _horizon_ok(c, dict(g, dir=g["dir"][p0:p1]), idx)
        assert ok.mean() > 0.99
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


def _window(g, x0, y0, w, h):
    """A w x h sub-window of a G-buffer, as a G-buffer of its own."""
    W, H = g["width"], g["height"]
    pos = g["pos"].reshape(H, W, 3)[y0:y0 + h, x0:x0 + w]
    nrm = g["nrm"].reshape(H, W, 3)[y0:y0 + h, x0:x0 + w]
    return {"width": w, "height": h, "pos": np.ascontiguousarray(pos.reshape(-1, 3)),
            "nrm": np.ascontiguousarray(nrm.reshape(-1, 3))}


@pytest.mark.parametrize("gx,gy,win,k", [(64, 64, (3, 2), 16), (160, 150, (128, 96), 4)])
def test_many_caches_few_pixels(drc, ctx, gx, gy, win, k):
    """More cache-grid cells than pixel-order bins.  4096 caches over 3 x 2
    pixels: every pixel goes to one order bin.  24000 caches with k = 4 (one
    cache per grid cell): the prefix sum over the cache cells spans two tiles
    of bins and a ragged tail."""
    big, c = _scene(2 * gx, 2 * gy, gx, gy)
    g = _window(big, 50, 60, *win)
    r = synth.world_radius(gx * gy)
    out, nbr, ref, idx, d2 = _run(drc, ctx, g, c, k, drc.METRIC_WORLD, drc.WP_INVERSE, drc.INTERP_IRRADIANCE, r)
    ok = ~_ambiguous(d2, k)
    assert ok.mean() > 0.99
    np.testing.assert_array_equal(np.sort(nbr[ok], axis=1), np.sort(idx[ok], axis=1))
    assert rel_err(out[ok], ref[ok]) <= FP32_TOL


def _horizon_ok(c, g, idx):
    """Pixels whose direction grazes none of their caches' horizons (a LOOKUP
    term switches on or off there)."""
    n = c["nrm"].astype(np.float64)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    lz = np.einsum("pc,pkc->pk", g["dir"].astype(np.float64), n[idx])
    return ~np.any(np.abs(lz) < 1e-5, axis=1)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("k", [1, 4, 8, 13, 16, 32])
def test_world_without_neighbour_list(drc, ctx, k, mode):
    """WORLD metric with no neighbour list asked for: the k-th distance from
    32-bit keys, then every candidate at or below it, blended in visit order.
    Same images as the oracle and as the exact (d^2, index) path."""
    g, c = _scene(96, 64, 16, 12, with_maps=mode == 1)
    r = synth.world_radius(16 * 12)
    fast = ctx.interpolate(_cuda(c), _cuda(g), k, drc.METRIC_WORLD, drc.WP_INVERSE, mode, r)
    torch.cuda.synchronize()
    assert ctx.status() == drc.OK
    fast = fast.cpu().numpy()
    exact, nbr, ref, idx, d2 = _run(drc, ctx, g, c, k, drc.METRIC_WORLD, drc.WP_INVERSE, mode, r)
    ok = ~_ambiguous(d2, k)
    if mode == 1:
        ok &= _horizon_ok(c, g, idx)
    assert ok.mean() > 0.99
    assert rel_err(fast[ok], ref[ok]) <= FP32_TOL
    np.testing.assert_allclose(fast[ok], exact[ok], rtol=1e-5, atol=1e-6)


def _coop_case(name, seed=21):
    """Cache layouts that drive the warp-cooperative query's edge paths."""
    rng = np.random.default_rng(seed)
    if name == "few_caches":  # fewer caches than k + 1: every warp gathers the whole grid
        g = synth.gbuffer(40, 30, seed=seed)
        pos = rng.uniform(0.2, 0.8, size=(5, 3)).astype(np.float32)
    elif name == "one_point":  # every cache at one point: buffer overflow, exact walk, ties by index
        g = synth.gbuffer(48, 40, seed=seed)
        pos = np.tile(np.float32([[0.4, 0.55, 0.3]]), (600, 1))
    elif name == "coplanar":  # caches on a plane, pixels all around it: a 2-D grid, 3-D queries
        g = synth.gbuffer(64, 48, seed=seed)
        pos = rng.uniform(0.0, 1.0, size=(300, 3)).astype(np.float32)
        pos[:, 2] = 0.5
    elif name == "clustered":  # half the caches in a small ball: densities far from the mean
        g = synth.gbuffer(96, 64, seed=seed)
        pos = rng.uniform(0.0, 1.0, size=(400, 3))
        pos[:200] = 0.3 + 0.03 * rng.normal(size=(200, 3))
        pos = pos.astype(np.float32)
    else:  # "ragged": a pixel count that is not a multiple of a warp, uniform caches
        g = synth.gbuffer(37, 29, seed=seed)
        pos = rng.uniform(0.0, 1.0, size=(250, 3)).astype(np.float32)
    n = len(pos)
    nrm = rng.normal(size=(n, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    c = {"pos": pos, "nrm": nrm.astype(np.float32), "pix": np.zeros((n, 2), np.int32),
         "payload": rng.uniform(0.0, 2.0, size=(n, 3)).astype(np.float32)}
    return g, c


@pytest.mark.parametrize("name", ["few_caches", "one_point", "coplanar", "clustered", "ragged"])
@pytest.mark.parametrize("k", [4, 16, 32])
def test_cooperative_query_edge_layouts(drc, ctx, name, k):
    """The WORLD query without a neighbour list (warp-cooperative gathers,
    second gathers, overflow and tie fallbacks) against the oracle on cache
    layouts far from the uniform benchmark scene."""
    g, c = _coop_case(name)
    n = len(c["pos"])
    r = synth.world_radius(n)
    out = ctx.interpolate(_cuda(c), _cuda(g), k, drc.METRIC_WORLD, drc.WP_INVERSE, drc.INTERP_IRRADIANCE, r)
    torch.cuda.synchronize()
    assert ctx.status() == drc.OK
    out = out.cpu().numpy()
    ref, idx, d2 = oracle.interpolate(c, g, k, drc.METRIC_WORLD, drc.WP_INVERSE, drc.INTERP_IRRADIANCE, r,
                                      want_neighbors=True)
    if name in ("few_caches", "one_point"):
        ok = np.ones(len(out), bool)  # every cache taken, or all tied: (d^2, index) decides on both sides
    else:
        ok = ~_ambiguous(d2, k)
        assert ok.mean() > 0.98
    assert rel_err(out[ok], ref[ok]) <= FP32_TOL


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("k", [4, 5, 9, 16])
def test_world_ties_at_kth_distance(drc, ctx, k, mode):
    """Every cache twice (same point, its own payload and map, index + n):
    each distance comes in a pair.  Odd k cuts a pair at the k-th distance,
    where only the lower index belongs: more than k candidates reach the k-th
    distance and the pixel takes the exact (d^2, index) walk.  Even k keeps
    pairs whole.  Pixels are compared where the distinct distances around
    the cut are not near-equal."""
    g, c = _scene(96, 64, 16, 12, with_maps=mode == 1)
    n = len(c["pos"])
    rng = np.random.default_rng(9)
    c2 = {"pos": np.concatenate([c["pos"], c["pos"]]), "nrm": np.concatenate([c["nrm"], c["nrm"]]),
          "pix": np.concatenate([c["pix"], c["pix"]]),
          "payload": np.concatenate([c["payload"], rng.uniform(0.0, 2.0, size=(n, 3)).astype(np.float32)])}
    if mode == 1:
        c2["maps"] = np.concatenate([c["maps"], rng.uniform(0.0, 3.0, size=c["maps"].shape).astype(np.float32)])
    r = synth.world_radius(n)
    out = ctx.interpolate(_cuda(c2), _cuda(g), k, drc.METRIC_WORLD, drc.WP_INVERSE, mode, r)
    torch.cuda.synchronize()
    assert ctx.status() == drc.OK
    out = out.cpu().numpy()
    ref, idx, _ = oracle.interpolate(c2, g, k, drc.METRIC_WORLD, drc.WP_INVERSE, mode, r, want_neighbors=True)
    dd = np.sort(((g["pos"].astype(np.float64)[:, None, :] - c["pos"].astype(np.float64)[None, :, :]) ** 2).sum(-1),
                 axis=1)
    m = (k + 1) // 2  # distinct distances taken, the last possibly once
    ok = ~_ambiguous(dd, m)  # which pair is the m-th
    if k % 2 == 1 and m > 1:
        ok &= ~_ambiguous(dd, m - 1)  # which pair is cut
    if mode == 1:
        ok &= _horizon_ok(c2, g, idx)
    assert ok.mean() > 0.97
    if k % 2 == 1:  # the lower index of the cut pair is the one kept
        assert np.all(idx[ok, -1] < n)
    assert rel_err(out[ok], ref[ok]) <= FP32_TOL
