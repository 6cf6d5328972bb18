"""Parity of drc_denoise (tensor-core implicit-GEMM autoencoder, Sec. 3.3)
with the FP64 oracle, element by element, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_1910_02480_gb300 import synth
from parity import FP32_TOL, median_rel, rel_err

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


def _maps(N, H, W, seed=3, linear=False):
    g = synth.gbuffer(max(N, 1), 1, seed=seed + 10)
    maps, _ = synth.hemisphere_maps(g["pos"][:N], g["nrm"][:N], H=H, W=W, seed=seed)
    if linear:
        maps = maps.copy()
        maps[:, :3] = np.expm1(np.clip(maps[:, :3], 0.0, None))
    return np.ascontiguousarray(maps, dtype=np.float32)


CASES = [
    # widths, N, H, W, bias, flags, out_relu
    ([16], 2, 8, 8, False, 0, False),
    ([16], 3, 8, 12, True, 0, True),
    ([16, 32], 3, 16, 16, True, 1, False),
    ([32, 64, 128], 64, 32, 32, False, 0, False),
    ([32, 64, 128], 5, 32, 32, True, 3, True),
    ([16, 32, 48, 64], 3, 32, 48, True, 0, False),
    ([64, 128, 256], 9, 32, 32, True, 0, False),
    ([64, 128, 256, 512], 2, 64, 64, True, 0, False),
    ([96, 128], 3, 32, 48, True, 0, False),   # head over 96 channels: staged weights, halo column in the map
    ([128], 2, 64, 64, True, 2, True),        # head over 128 channels on 2 x 2 tiles per map
]


@pytest.mark.parametrize("widths,N,H,W,bias,flags,out_relu", CASES)
def test_fp32_matches_oracle(drc, widths, N, H, W, bias, flags, out_relu):
    w = synth.he_weights(widths, seed=0, bias=bias)
    x = _maps(N, H, W, linear=bool(flags & 1))
    s = 0.75 if flags else 1.0
    ctx = drc.Context(widths, w, precision="fp32", exposure=s, out_relu=out_relu)
    xd = torch.from_numpy(x).cuda()
    out, pay = ctx.denoise(xd, flags=flags, want_payload=True)
    torch.cuda.synchronize()
    assert ctx.status() == drc.OK
    ref = oracle.forward(w, x, widths, out_relu=out_relu, exposure=s, flags=flags)
    g = out.cpu().numpy()
    err = rel_err(g, ref)
    print("fp32 widths=%s N=%d %dx%d: max rel %.3e, median %.3e" % (widths, N, H, W, err, median_rel(g, ref)))
    assert err <= FP32_TOL
    ref_log = ref if not (flags & 2) else np.log1p(s * ref)
    ref_pay = oracle.payload(np.expm1(ref_log) / s)
    perr = rel_err(pay.cpu().numpy(), ref_pay)
    assert perr <= FP32_TOL, perr


def test_fp32_full_size_sampled(drc):
    """4096 maps of 7x32x32, widths 64/128/256: the whole batch on the GPU in
    one call, eight maps spread over it recomputed by the oracle."""
    widths, N = [64, 128, 256], 4096
    w = synth.he_weights(widths, seed=0)
    g = synth.gbuffer(64, 64, seed=2)
    c = synth.cache_grid(g, 64, 64)
    x, _ = synth.hemisphere_maps(c["pos"], c["nrm"])
    ctx = drc.Context(widths, w, precision="fp32")
    xd = torch.from_numpy(x).cuda()
    out, pay = ctx.denoise(xd, want_payload=True)
    torch.cuda.synchronize()
    assert ctx.status() == drc.OK
    idx = np.array([0, 1, 777, 1500, 2048, 3001, 4094, 4095])
    ref = oracle.forward(w, x[idx], widths)
    err = rel_err(out.cpu().numpy()[idx], ref)
    print("fp32 full size sampled: max rel %.3e" % err)
    assert err <= FP32_TOL
    assert rel_err(pay.cpu().numpy()[idx], oracle.payload(np.expm1(ref))) <= FP32_TOL
    assert np.all(np.isfinite(out.cpu().numpy()))


def test_fp32_full_size_autotuned_sampled(drc):
    """The benchmark's configuration exactly: 4096 maps of 7x32x32, widths
    64/128/256, with the tiles and A paths drc_autotune picks for that batch
    shape (the setting the benchmark times), and the payload; maps spread over
    the batch -- both ends, the middle, tile boundaries -- recomputed by the
    oracle."""
    widths, N = [64, 128, 256], 4096
    w = synth.he_weights(widths, seed=0)
    g = synth.gbuffer(1920, 1080, seed=2)
    c = synth.cache_grid(g, 64, 64)
    x, _ = synth.hemisphere_maps(c["pos"], c["nrm"], H=32, W=32, seed=3)
    ctx = drc.Context(widths, w, precision="fp32", max_maps=N, max_hw=32 * 32)
    ctx.autotune(N, 32, 32)
    tiles = [ctx.describe_layer(li) for li in range(2 * len(widths))]
    print("autotuned (tile_n, a_path) per layer:", tiles)
    xd = torch.from_numpy(x).cuda()
    out, pay = ctx.denoise(xd, want_payload=True)
    torch.cuda.synchronize()
    assert ctx.status() == drc.OK
    idx = np.array([0, 1, 127, 128, 1023, 2047, 2048, 3071, 4094, 4095])
    ref = oracle.forward(w, x[idx], widths)
    err = rel_err(out.cpu().numpy()[idx], ref)
    print("fp32 full size autotuned sampled: max rel %.3e" % err)
    assert err <= FP32_TOL
    assert rel_err(pay.cpu().numpy()[idx], oracle.payload(np.expm1(ref))) <= FP32_TOL
    assert np.all(np.isfinite(out.cpu().numpy()))


@pytest.mark.parametrize("widths,N,H,W", [([32, 64, 128], 64, 32, 32), ([16, 32], 3, 16, 16)])
def test_bf16_error_reported(drc, widths, N, H, W):
    w = synth.he_weights(widths, seed=0)
    x = _maps(N, H, W)
    ctx = drc.Context(widths, w, precision="bf16")
    out = ctx.denoise(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    assert ctx.status() == drc.OK
    ref = oracle.forward(w, x, widths)
    g = out.cpu().numpy()
    err = rel_err(g, ref)
    rms = np.sqrt(np.mean(ref ** 2))
    normwise = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    print("bf16 widths=%s: max rel %.3e median %.3e, max|err|/rms %.3e, normwise %.3e"
          % (widths, err, median_rel(g, ref), np.max(np.abs(g - ref)) / rms, normwise))
    # bf16 keeps 8 significant bits (unit roundoff 2^-9 ~ 2e-3) in every stored
    # activation and operand; five layers of it give a normwise error of a few
    # 1e-3 and a largest deviation of a few percent of the output rms
    assert normwise < 1e-2
    assert np.max(np.abs(g - ref)) / rms < 0.1


def test_zero_maps_is_a_no_op(drc):
    ctx = drc.Context([16], synth.he_weights([16]), precision="fp32")
    x = torch.empty((0, 7, 8, 8), device="cuda")
    out = ctx.denoise(x)
    assert out.shape == (0, 3, 8, 8)
    assert ctx.status() == drc.OK


def test_argument_errors_are_reported(drc):
    ctx = drc.Context([16, 32], synth.he_weights([16, 32]), precision="fp32")
    x = torch.zeros((2, 7, 16, 16), device="cuda")
    with pytest.raises(drc.DrcError) as e:
        ctx.denoise(torch.zeros((2, 7, 18, 16), device="cuda"))  # H not a multiple of 4
    assert e.value.code == drc.ERR_INVALID_ARG
    with pytest.raises(drc.DrcError) as e:
        ctx.denoise(x, out=torch.zeros((2, 3, 16, 16)))  # host output
    assert e.value.code == drc.ERR_INVALID_ARG
    with pytest.raises(drc.DrcError) as e:
        ctx.denoise(x, flags=0x80)
    assert e.value.code == drc.ERR_INVALID_ARG
    with pytest.raises(ValueError):
        drc.Context([16, 32], np.zeros(10, np.float32))


def test_stalled_wait_times_out_and_context_recovers(drc):
    """A wait that nothing completes (test flag) gives up after the context's
    timeout and latches DRC_ERR_TIMEOUT; the next call runs normally."""
    widths = [16, 32]
    w = synth.he_weights(widths, seed=0)
    ctx = drc.Context(widths, w, precision="fp32", wait_timeout_ms=50)
    x = _maps(3, 16, 16)
    xd = torch.from_numpy(x).cuda()
    ctx.denoise(xd, flags=drc.F_DEBUG_STALL)
    assert ctx.status() == drc.ERR_TIMEOUT
    out = ctx.denoise(xd)
    assert ctx.status() == drc.OK
    assert rel_err(out.cpu().numpy(), oracle.forward(w, x, widths)) <= FP32_TOL


def test_launch_count_and_timing(drc):
    """One denoise call launches the input staging kernel, S encoder convs,
    S-1 decoder convTs and the head; with timing on each gets a device time,
    and timing changes no result."""
    widths = [16, 32, 48]
    w = synth.he_weights(widths, seed=0, bias=True)
    ctx = drc.Context(widths, w, precision="fp32")
    x = torch.from_numpy(_maps(4, 32, 32)).cuda()
    ref = ctx.denoise(x).clone()
    n0 = ctx.launch_count()
    ctx.set_timing(True)
    out = ctx.denoise(x)
    out = ctx.denoise(x, out=out)
    ctx.set_timing(False)
    assert ctx.launch_count() - n0 == 2 * (1 + 2 * len(widths))
    t = ctx.read_timing()
    names = ["stage input", "conv e1", "conv e2", "conv e3", "convT d3", "convT d2", "head"]
    assert list(t) == names
    for n in names:
        assert t[n][0] == 2 and t[n][1] > 0.0
    assert ctx.read_timing() == {}
    assert ctx.status() == drc.OK
    assert torch.equal(out, ref)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_autotuned_context_keeps_parity(drc, precision):
    """drc_autotune may change every layer's tile width and A path; the
    results stay those of the oracle (FP32 bar) / of the untuned context."""
    widths = [32, 64, 128]
    w = synth.he_weights(widths, seed=3, bias=True)
    x = torch.from_numpy(_maps(40, 32, 32)).cuda()
    base = drc.Context(widths, w, precision=precision)
    ref = base.denoise(x).cpu().numpy()
    ctx = drc.Context(widths, w, precision=precision)
    ctx.autotune(40, 32, 32)
    tiles = [ctx.describe_layer(li) for li in range(2 * len(widths))]
    print(precision, "autotuned (tile N, A path):", tiles)
    assert tiles[-1][0] == 0
    for li, (bn, _) in enumerate(tiles[:-1]):
        cout = widths[li] if li < len(widths) else widths[2 * len(widths) - 2 - li]
        assert bn in (cout, cout // 2)
    g = ctx.denoise(x).cpu().numpy()
    assert ctx.status() == drc.OK
    if precision == "fp32":
        assert rel_err(g, oracle.forward(w, x.cpu().numpy(), widths)) <= FP32_TOL
    d = np.max(np.abs(g - ref)) / np.sqrt(np.mean(ref * ref))
    print("max |tuned - untuned| / rms:", d)
    if precision == "fp32":  # the A paths differ at most in the split of A's tf32 parts (see the pair tests)
        assert d <= 1e-5
    else:
        assert rel_err(g, ref) <= 1e-2


PAIR_CASES = [
    # widths, N, H, W: decoder layers of <= 64 output channels run as phase pairs
    ([32, 64, 128], 5, 32, 32),     # d3 (64 channels, 128-column pairs), d2 (32, 64-column pairs); ragged M
    ([64, 128, 256], 9, 32, 32),    # d2 only (d3 has 128 channels)
    ([16, 32, 48, 64], 3, 64, 64),  # d4 .. d2: 48, 32 and 16 channels (96, 64, 32 columns)
]


@pytest.mark.parametrize("mode", [8, 9])
@pytest.mark.parametrize("widths,N,H,W", PAIR_CASES)
def test_phase_pairs_match_oracle(drc, widths, N, H, W, mode, tmp_path):
    """Decoder layers forced onto the phase-pair form (A path 8: A in tensor
    memory, 9: in shared memory; applied through a tile cache entry, every
    other layer on its default tiles) keep the oracle's FP32 bar, and agree
    with the one-GEMM-per-parity form.  With A in tensor memory the pair adds
    zero-weight taps only, whole K blocks of exact zero products: bit for bit.
    With A in shared memory the decoder forms split A as trunc_tf32(A) (read
    by the MMAs from the TMA box itself) + the tf32 remainder, where the
    tensor-memory form rounds both parts to nearest; per product the two
    splits' errors differ by about 2^-20 relative, so the outputs differ by
    far less than 1e-5 of their rms."""
    import json
    w = synth.he_weights(widths, seed=5, bias=True)
    x = torch.from_numpy(_maps(N, H, W, seed=7)).cuda()
    S = len(widths)
    base = drc.Context(widths, w, precision="fp32")
    ref = base.denoise(x).cpu().numpy()
    tiles = [base.describe_layer(li) for li in range(2 * S)]  # the defaults ref ran with
    cache = str(tmp_path / "tiles.jsonl")
    assert base.autotune(N, H, W, cache=cache) is False
    entry = json.loads(open(cache).read().splitlines()[-1])
    entry["tile_n"] = [t[0] for t in tiles]
    entry["a_path"] = [-1] * (2 * S)
    paired = []
    for li in range(S, 2 * S - 1):  # convT d_S .. d_2
        cout = widths[2 * S - 2 - li]
        if 2 * cout <= 128 and cout % 16 == 0:
            entry["a_path"][li] = mode
            paired.append(li)
    assert paired
    with open(cache, "a") as f:
        f.write(json.dumps(entry) + "\n")
    ctx = drc.Context(widths, w, precision="fp32")
    assert ctx.autotune(N, H, W, cache=cache) is True
    assert [ctx.describe_layer(li)[1] for li in paired] == [mode] * len(paired)
    g = ctx.denoise(x).cpu().numpy()
    assert ctx.status() == drc.OK
    err = rel_err(g, oracle.forward(w, x.cpu().numpy(), widths))
    d = np.max(np.abs(g - ref)) / np.sqrt(np.mean(ref * ref))
    print("pairs on layers %s: max rel %.3e vs oracle, max |paired - unpaired| / rms %.3e" % (paired, err, d))
    assert err <= FP32_TOL
    if mode == 8:
        assert np.array_equal(g, ref)
    else:
        assert d <= 1e-5


def test_phase_pairs_full_size(drc, tmp_path):
    """The benchmark's batch (4096 maps of 7x32x32, widths 64/128/256) with d2
    forced onto its phase pairs with A in shared memory (the path the
    autotuner picks there): every output equals the four-GEMM form's bit for
    bit but for the split of A (shared-memory A truncates its tf32 high part,
    see test_phase_pairs_match_oracle: within 1e-5 of the rms), and sampled
    maps meet the oracle's FP32 bar.  The four-GEMM result is still in flight
    when drc_autotune starts on the same context: the tuner's timing
    launches, which reuse the workspace, wait for it (a race there corrupted
    whole maps, far beyond this bound)."""
    import json
    widths, N = [64, 128, 256], 4096
    w = synth.he_weights(widths, seed=8, bias=True)
    g = synth.gbuffer(1920, 1080, seed=5)
    c = synth.cache_grid(g, 64, 64)
    x, _ = synth.hemisphere_maps(c["pos"], c["nrm"], H=32, W=32, seed=6)
    xd = torch.from_numpy(x).cuda()
    base = drc.Context(widths, w, precision="fp32", max_maps=N, max_hw=32 * 32)
    ref = base.denoise(xd)
    cache = str(tmp_path / "tiles.jsonl")
    base.autotune(N, 32, 32, cache=cache)
    entry = json.loads(open(cache).read().splitlines()[-1])
    entry["tile_n"] = [64, 128, 256, 128, 64, 0]  # the default tiles, d2 paired
    entry["a_path"] = [-1, -1, -1, -1, 9, -1]
    with open(cache, "a") as f:
        f.write(json.dumps(entry) + "\n")
    ctx = drc.Context(widths, w, precision="fp32", max_maps=N, max_hw=32 * 32)
    assert ctx.autotune(N, 32, 32, cache=cache) is True
    assert ctx.describe_layer(4) == (64, 9)
    out = ctx.denoise(xd)
    torch.cuda.synchronize()
    assert ctx.status() == drc.OK
    idx = np.array([0, 63, 64, 2047, 2048, 4095])
    o = oracle.forward(w, x[idx], widths)
    err = rel_err(out.cpu().numpy()[idx], o)
    err_ref = rel_err(ref.cpu().numpy()[idx], o)
    d = ((out - ref).abs().max() / ref.pow(2).mean().sqrt()).item()
    print("d2 phase pairs, 4096 maps: max rel %.3e (four GEMMs: %.3e) on the sampled maps; max |paired - four GEMMs|"
          " / rms %.3e" % (err, err_ref, d))
    assert err <= FP32_TOL and err_ref <= FP32_TOL
    assert d <= 1e-5
