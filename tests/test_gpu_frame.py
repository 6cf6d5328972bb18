"""drc_frame_host: one frame from host memory (maps denoised, image
interpolated from their payloads, Sec. 3.3 feeding Sec. 3.2) through the C
ABI with the uploads and the download inside the call.

The overlapped call must give what the two device calls give on the same
inputs: the same kernels run on the same data, so the images agree to fp32
rounding of the payload sums.  The device path itself is pinned to the FP64 oracle elsewhere
(test_gpu_denoise, test_gpu_interp); here one case is also checked against
the oracle end to end."""
import numpy as np
import pytest

import oracle
from paper_1910_02480_gb300 import synth
from parity import FP32_TOL, rel_err

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

WIDTHS = [32, 64, 128]


@pytest.fixture(scope="module")
def drc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_02480_gb300 import build
    build.build()
    import paper_1910_02480_gb300 as m
    return m


def _frame(width, height, gx, gy, seed):
    g = synth.gbuffer(width, height, seed=seed)
    c = synth.cache_grid(g, gx, gy)
    x, _ = synth.hemisphere_maps(c["pos"], c["nrm"], H=32, W=32, seed=seed + 1)
    return g, c, np.ascontiguousarray(x, dtype=np.float32)


def _device_reference(drc, ctx, g, c, x, k, r):
    xd = torch.from_numpy(x).cuda()
    pay = torch.empty((x.shape[0], 3), device="cuda")
    ctx.denoise(xd, payload=pay)
    cd = {"pos": torch.from_numpy(c["pos"]).cuda(), "nrm": torch.from_numpy(c["nrm"]).cuda(),
          "pix": torch.from_numpy(c["pix"]).cuda(), "payload": pay}
    gd = {"width": g["width"], "height": g["height"], "pos": torch.from_numpy(g["pos"]).cuda(),
          "nrm": torch.from_numpy(g["nrm"]).cuda()}
    out = ctx.interpolate(cd, gd, k, drc.METRIC_WORLD, drc.WP_INVERSE, drc.INTERP_IRRADIANCE, r)
    torch.cuda.synchronize()
    return out.cpu().numpy(), cd


def _host(g, x):
    gh = {"width": g["width"], "height": g["height"], "pos": torch.from_numpy(g["pos"]).pin_memory(),
          "nrm": torch.from_numpy(g["nrm"]).pin_memory()}
    return torch.from_numpy(x).pin_memory(), gh


@pytest.mark.parametrize("gx,gy", [(8, 8), (7, 1), (3, 1), (9, 5)])  # 64, 7, 3, 45 maps
def test_frame_matches_device_calls(drc, gx, gy):
    ctx = drc.Context(WIDTHS, synth.he_weights(WIDTHS, seed=0, bias=True), precision="fp32")
    g, c, x = _frame(96, 64, gx, gy, seed=5)
    r = synth.world_radius(gx * gy)
    k = min(8, gx * gy)
    ref, cd = _device_reference(drc, ctx, g, c, x, k, r)
    xh, gh = _host(g, x)
    rgb = ctx.frame_host(xh, cd, gh, k, drc.METRIC_WORLD, drc.WP_INVERSE, r)
    torch.cuda.synchronize()
    assert ctx.status() == drc.OK
    got = rgb.numpy()
    np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-6)
    ctx.close()


def test_consecutive_frames_overlap_correctly(drc):
    """Three frames enqueued back to back (uploads of one under the compute
    of the previous), synchronised once: each image is its own frame's."""
    ctx = drc.Context(WIDTHS, synth.he_weights(WIDTHS, seed=0, bias=True), precision="fp32")
    outs, refs = [], []
    for seed in (11, 21, 31):
        g, c, x = _frame(128, 96, 8, 8, seed=seed)
        r = synth.world_radius(64)
        ref, cd = _device_reference(drc, ctx, g, c, x, 8, r)
        refs.append(ref)
        outs.append((g, c, x, cd, r))
    rgbs = []
    for g, c, x, cd, r in outs:
        xh, gh = _host(g, x)
        rgbs.append((ctx.frame_host(xh, cd, gh, 8, drc.METRIC_WORLD, drc.WP_INVERSE, r), xh, gh))
    torch.cuda.synchronize()
    assert ctx.status() == drc.OK
    for (rgb, _, _), ref in zip(rgbs, refs):
        np.testing.assert_allclose(rgb.numpy(), ref, rtol=1e-5, atol=1e-6)
    ctx.close()


def test_frame_against_oracle(drc):
    """End to end against the FP64 oracle: forward, payload, interpolation."""
    w = synth.he_weights(WIDTHS, seed=0, bias=True)
    ctx = drc.Context(WIDTHS, w, precision="fp32")
    g, c, x = _frame(64, 48, 6, 6, seed=7)
    r = synth.world_radius(36)
    k = 8
    cd = {"pos": torch.from_numpy(c["pos"]).cuda(), "nrm": torch.from_numpy(c["nrm"]).cuda(),
          "pix": torch.from_numpy(c["pix"]).cuda()}
    xh, gh = _host(g, x)
    rgb = ctx.frame_host(xh, cd, gh, k, drc.METRIC_WORLD, drc.WP_INVERSE, r)
    torch.cuda.synchronize()
    out = oracle.forward(w, x, WIDTHS)
    cc = dict(c)
    cc["payload"] = oracle.payload(np.expm1(out)).astype(np.float32)
    ref, idx, d2 = oracle.interpolate(cc, g, k, oracle.METRIC_WORLD, oracle.WP_INVERSE, oracle.INTERP_IRRADIANCE, r,
                                      want_neighbors=True)
    a, b = d2[:, k - 1], d2[:, k]
    ok = np.abs(b - a) > 1e-5 * np.maximum(b, 1e-30)
    assert ok.mean() > 0.99
    assert rel_err(rgb.numpy()[ok], ref[ok]) <= FP32_TOL


def test_frame_argument_errors(drc):
    ctx = drc.Context(WIDTHS, synth.he_weights(WIDTHS, seed=0), precision="fp32")
    g, c, x = _frame(32, 32, 4, 4, seed=3)
    cd = {"pos": torch.from_numpy(c["pos"]).cuda(), "nrm": torch.from_numpy(c["nrm"]).cuda(),
          "pix": torch.from_numpy(c["pix"]).cuda()}
    xh, gh = _host(g, x)
    with pytest.raises(ValueError):
        ctx.frame_host(torch.from_numpy(x).cuda(), cd, gh, 4, drc.METRIC_WORLD, drc.WP_INVERSE, 0.3)
    with pytest.raises(drc.DrcError):  # caches->n != N
        ctx.frame_host(xh[:5], cd, gh, 4, drc.METRIC_WORLD, drc.WP_INVERSE, 0.3)
    ctx.close()
