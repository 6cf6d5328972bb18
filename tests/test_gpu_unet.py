"""The paper's own network form (Sec. 3.3, a U-Net) through
drc_unet_forward against the FP64 oracle's unet_forward."""
import numpy as np
import pytest

import oracle
from paper_1910_02480_gb300 import synth
from parity import FP32_TOL, rel_err

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

# The FP32 bar, and a normwise one.  The U-Net chains 17 layers of up to
# 9 x 768 terms with batch-normalisation gains: a float32 PyTorch evaluation
# of the paper-size case below differs from the FP64 oracle by 6.0e-5
# (floored, max) and 8.3e-7 (normwise).  The kernel sums each output in
# two levels (72-term partial sums, then their total); with one serial sum
# it measured 1.5e-4 here, with two levels 3.6e-5 and 6.7e-7.
UNET_NORMWISE = 1e-5


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


@pytest.mark.parametrize("base,levels,N,H,W", [
    (64, 3, 2, 32, 32),   # the paper's network: 7.8 M parameters, 4 x 4 bottleneck
    (8, 2, 5, 16, 16),
    (20, 1, 5, 4, 4),     # whole maps per block, 20 / 40 channels (not multiples of 16)
    (4, 2, 3, 32, 16),    # non-square maps, several tiles per map
])
def test_unet_matches_oracle(drc, ctx, base, levels, N, H, W):
    params = synth.unet_params(base, levels, seed=base + levels)
    x = np.random.default_rng(N * H + W).standard_normal((N, 7, H, W)).astype(np.float32)
    net = drc.UNet(ctx, params, base, levels)
    y = net.forward(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    assert ctx.status() == drc.OK
    ref = oracle.unet_forward(params, x, base, levels)
    assert np.abs(ref).max() > 0  # ReLU head: not all zero
    yh = y.cpu().numpy()
    assert rel_err(yh, ref) <= FP32_TOL
    assert np.linalg.norm(yh - ref) <= UNET_NORMWISE * np.linalg.norm(ref)


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
