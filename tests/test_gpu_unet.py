"""The paper's own network form (Sec. 3.3, a U-Net) through
drc_unet_forward against the FP64 oracle's unet_forward."""
import numpy as np
import pytest

import oracle
from paper_1910_02480_gb300 import synth
from parity import FP32_TOL, rel_err, unet_float32

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

# The bar: the FP32 bar and a normwise one, or twice what a plain IEEE
# float32 evaluation of the same inputs misses the FP64 oracle by, whichever
# is larger.  The U-Net chains 17 layers of up to 9 x 768 terms with
# batch-normalisation gains, and the floored max error of a float32
# evaluation sits near the FP32 bar itself: 6.0e-5 on the paper-size case
# below (normwise 8.3e-7), above 1e-4 on some single maps.  The CUDA-core
# kernel sums each output in two levels (72-term partial sums, then their
# total; one serial sum measured 1.5e-4 here, two levels 3.6e-5); the
# tensor-core form accumulates in chunks of one K block (4.1e-5).
UNET_NORMWISE = 1e-5


def unet_bars(params, x, ref, base, levels, cin=7, cout=3):
    f32 = unet_float32(params, x, base, levels, cin, cout)
    nw32 = np.linalg.norm(f32 - ref) / np.linalg.norm(ref)
    return max(FP32_TOL, 2 * rel_err(f32, ref)), max(UNET_NORMWISE, 2 * nw32)


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


@pytest.mark.parametrize("base,levels,N,H,W,cin,cout,tc", [
    # tensor cores (stride-1 implicit GEMMs of the conv kernel family)
    (64, 3, 2, 32, 32, 7, 3, True),    # the paper's network: 7.8 M parameters, 4 x 4 bottleneck
    (32, 2, 3, 16, 16, 7, 5, True),    # ragged last tile at 8 x 8 (192 rows); two head groups
    (32, 1, 5, 8, 8, 7, 3, True),      # whole maps per tile at both levels, ragged
    (32, 2, 2, 32, 16, 7, 3, True),    # non-square maps
    (32, 1, 3, 8, 8, 32, 3, True),     # 32 input channels: whole K blocks instead of tap boxes
    # CUDA cores (channel counts that are not whole K blocks)
    (8, 2, 5, 16, 16, 7, 3, False),
    (20, 1, 5, 4, 4, 7, 3, False),     # whole maps per block, 20 / 40 channels (not multiples of 16)
    (4, 2, 3, 32, 16, 7, 3, False),    # non-square maps, several tiles per map
])
def test_unet_matches_oracle(drc, ctx, base, levels, N, H, W, cin, cout, tc):
    assert drc.unet_tensor_cores(base, levels, H, W, cin, cout) == tc
    params = synth.unet_params(base, levels, cin=cin, cout=cout, seed=base + levels)
    x = np.random.default_rng(N * H + W).standard_normal((N, cin, H, W)).astype(np.float32)
    net = drc.UNet(ctx, params, base, levels, in_ch=cin, out_ch=cout)
    y = net.forward(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    assert ctx.status() == drc.OK
    ref = oracle.unet_forward(params, x, base, levels, cin=cin, cout=cout)
    assert np.abs(ref).max() > 0  # ReLU head: not all zero
    yh = y.cpu().numpy()
    bar, nbar = unet_bars(params, x, ref, base, levels, cin, cout)
    assert rel_err(yh, ref) <= bar
    assert np.linalg.norm(yh - ref) <= nbar * np.linalg.norm(ref)


def test_unet_tensor_cores_at_bench_size_sampled(drc, ctx):
    """The benchmarked launch (4096 maps of 32 x 32, the paper's network) on
    the tensor cores; maps are independent (inference statistics), so three
    of them are checked against the oracle one by one."""
    N, base, levels = 4096, 64, 3
    assert drc.unet_tensor_cores(base, levels, 32, 32)
    params = synth.unet_params(base, levels, seed=11)
    x = np.random.default_rng(5).standard_normal((N, 7, 32, 32)).astype(np.float32)
    net = drc.UNet(ctx, params, base, levels)
    y = net.forward(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    assert ctx.status() == drc.OK
    yh = y.cpu().numpy()
    for n in (0, 2047, 4095):
        ref = oracle.unet_forward(params, x[n:n + 1], base, levels)
        bar, nbar = unet_bars(params, x[n:n + 1], ref, base, levels)
        assert rel_err(yh[n:n + 1], ref) <= bar, n
        assert np.linalg.norm(yh[n:n + 1] - ref) <= nbar * np.linalg.norm(ref), n


def test_unet_argument_errors(drc, ctx):
    params = synth.unet_params(4, 2)
    net = drc.UNet(ctx, params, 4, 2)
    net.forward(torch.zeros((0, 7, 8, 8), device="cuda"))  # N = 0: nothing
    with pytest.raises(drc.DrcError):
        net.forward(torch.zeros((1, 7, 6, 8), device="cuda"))  # 6 is not a multiple of 4
    x = torch.zeros((1, 7, 8, 8), device="cuda")
    out = torch.empty((1, 3, 8, 8), device="cuda")
    ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    rc = ctx._lib.drc_unet_forward(ctx._ctx, 7, 3, 4, 2, net.params.data_ptr(), x.data_ptr(), out.data_ptr(), 1, 8, 8,
                                   ws.data_ptr(), ws.numel(), None)
    assert rc == drc.ERR_INVALID_ARG  # workspace too small
    assert drc.unet_param_count(4, 0) == 0 and drc.unet_param_count(0, 2) == 0
    with pytest.raises(ValueError):
        drc.UNet(ctx, params[:-1], 4, 2)
