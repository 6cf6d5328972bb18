"""drc_weight_grad: one layer's weight gradient (the per-layer step of the
training pass, Sec. 3.3) against the FP64 oracle's conv_weight_grad (pinned
in test_oracle_backward by the adjoint identity and a brute-force sum).

The operands are rounded to bfloat16 on the host before either side sees
them, so both compute the same exact products; the GPU differs only in fp32
summation order.  Bound, element by element: |dW - ref| <= tol * S with
S = sum |R| |Q| over the same terms (the oracle on |R|, |Q|) and
tol = 2^-22 (sqrt(K) + 16) for K pixels -- a random-walk estimate of fp32
rounding over the chained partial sums (tensor-core accumulator, split K,
atomics) with a factor 2 for accumulators that truncate.  At the small sizes
this is below the weight of one pixel (~S/K), so a dropped or doubled pixel,
tap or channel fails.  The shapes cover every kernel (tensor cores, wide
form: Mr a multiple of 128, Qc of 64; narrow form: Qc = 8, Mr a multiple of
64; both need 64-pixel blocks of whole rows of whole maps; CUDA cores
otherwise, and FP32), ragged tails, several m and q tiles, and the layers of
the training benchmark (256 maps of 64 x 64, widths 64/128/256/512) at full
size."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_02480_gb300 import build
    build.build()
    import paper_1910_02480_gb300 as m
    c = m.Context([64, 128, 256], None, precision="bf16")
    yield c
    c.close()


def _operands(N, Hb, Wb, Mr, Qc, seed, dtype):
    """R: output-gradient-like (random signs, a third zero); Q: activation-
    like (ReLU of a normal: half zero, non-negative).  NHWC, rounded to the
    operand dtype on the host."""
    rng = np.random.default_rng(seed)
    R = rng.normal(size=(N, Hb, Wb, Mr)) * (rng.random((N, Hb, Wb, Mr)) > 1 / 3)
    Q = np.maximum(rng.normal(size=(N, 2 * Hb, 2 * Wb, Qc)), 0.0)
    tR = torch.from_numpy(R.astype(np.float32)).to(dtype)
    tQ = torch.from_numpy(Q.astype(np.float32)).to(dtype)
    return tR, tQ


def _check(ctx, N, Hb, Wb, Mr, Qc, Qraw, dtype, seed=0, transposed=False):
    tR, tQ = _operands(N, Hb, Wb, Mr, Qc, seed, dtype)
    dW = ctx.weight_grad(tR.cuda(), tQ.cuda(), qraw=Qraw)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    g = dW.cpu().numpy().astype(np.float64)
    R = tR.float().numpy().astype(np.float64).transpose(0, 3, 1, 2)  # NCHW
    Q = tQ.float().numpy().astype(np.float64).transpose(0, 3, 1, 2)
    if transposed:  # a transposed conv: R its input, Q its output gradient
        ref = oracle.conv_weight_grad(R, Q, transposed=True)
        S = oracle.conv_weight_grad(np.abs(R), np.abs(Q), transposed=True)
    else:  # a conv: Q its input, R its output gradient
        ref = oracle.conv_weight_grad(Q, R)
        S = oracle.conv_weight_grad(np.abs(Q), np.abs(R))
    ref, S = ref[:, :Qraw], S[:, :Qraw]
    K = N * Hb * Wb
    tol = 2.0 ** -22 * (np.sqrt(K) + 16)
    ratio = np.abs(g - ref) / np.maximum(S, 1e-30)
    print("wgrad %s N=%d %dx%d Mr=%d Qc=%d Qraw=%d: max |err|/S %.2e (bound %.2e), one pixel ~ %.1e" % (
        str(dtype).split(".")[-1], N, Hb, Wb, Mr, Qc, Qraw, ratio.max(), tol, 1.0 / K))
    assert g.shape == (Mr, Qraw, 3, 3)
    assert np.all(np.abs(g - ref) <= tol * S + 1e-30), ratio.max()


@pytest.mark.parametrize("N,Hb,Wb,Mr,Qc,Qraw", [
    (37, 8, 8, 128, 64, 64),      # one map per 64-pixel block, many splits
    (13, 4, 4, 256, 128, 128),    # four maps per block, last block one map
    (3, 16, 16, 128, 64, 64),     # four rows per block, blocks inside a map
    (21, 2, 2, 128, 128, 128),    # sixteen maps per block, ragged
    (5, 8, 8, 128, 64, 50),       # only Qraw of Qc channels in dW
    (2, 1, 64, 128, 64, 64),      # one 64-pixel row per map
    (9, 4, 8, 384, 192, 192),     # three m tiles, three 64-wide q tiles
])
def test_tensor_core_shapes(ctx, N, Hb, Wb, Mr, Qc, Qraw):
    _check(ctx, N, Hb, Wb, Mr, Qc, Qraw, torch.bfloat16, seed=N)


def test_transposed_layer_orientation(ctx):
    _check(ctx, 6, 8, 8, 128, 64, 64, torch.bfloat16, seed=4, transposed=True)


@pytest.mark.parametrize("N,Hb,Wb,Mr,Qc,Qraw", [
    (3, 16, 16, 64, 8, 7),     # the first layer: 8 stored input channels, 7 in dW
    (7, 8, 8, 64, 8, 3),       # the head: dL/dout in 8 channels, 3 in dW
    (5, 4, 4, 128, 8, 8),      # four maps per block, ragged
    (3, 8, 8, 320, 8, 8),      # five 64-channel column tiles
    (2, 16, 16, 256, 8, 7),    # one 256-column tile
])
def test_tensor_core_narrow_shapes(ctx, N, Hb, Wb, Mr, Qc, Qraw):
    _check(ctx, N, Hb, Wb, Mr, Qc, Qraw, torch.bfloat16, seed=N + 7)


@pytest.mark.parametrize("N,Hb,Wb,Mr,Qc,Qraw,dt", [
    (4, 8, 8, 64, 32, 32, "bf16"),   # Mr not a multiple of 128
    (4, 3, 5, 128, 64, 64, "bf16"),  # rows of 5 pixels: no whole-row blocks
    (4, 8, 8, 128, 64, 64, "fp32"),  # FP32 operands
    (3, 8, 8, 48, 8, 7, "bf16"),     # 8 Q channels, Mr not a multiple of 64
    (3, 8, 8, 64, 16, 16, "bf16"),   # 16 Q channels
])
def test_cuda_core_shapes(ctx, N, Hb, Wb, Mr, Qc, Qraw, dt):
    _check(ctx, N, Hb, Wb, Mr, Qc, Qraw, torch.bfloat16 if dt == "bf16" else torch.float32, seed=N + 1)


@pytest.mark.parametrize("Hb,Mr,Qc,Qraw", [
    (16, 128, 64, 64),    # encoder stage 2 (and decoder stage 2 transposed)
    (8, 256, 128, 128),   # stage 3
    (4, 512, 256, 256),   # stage 4: four m tiles, two q tiles
    (32, 64, 8, 7),       # stage 1: narrow form
])
def test_training_benchmark_layers_full_size(ctx, Hb, Mr, Qc, Qraw):
    _check(ctx, 256, Hb, Hb, Mr, Qc, Qraw, torch.bfloat16, seed=Hb)


def test_training_benchmark_head_full_size(ctx):
    """The head's weight gradient: R = t_1 (64 channels, 32 x 32), Q = dL/dout
    in 8 bf16 channels at 64 x 64, 3 of them in dW."""
    _check(ctx, 256, 32, 32, 64, 8, 3, torch.bfloat16, seed=31)


def test_empty_batch_and_accumulation(ctx):
    R = torch.zeros((0, 4, 4, 128), dtype=torch.bfloat16, device="cuda")
    Q = torch.zeros((0, 8, 8, 64), dtype=torch.bfloat16, device="cuda")
    dW = torch.full((128, 64, 3, 3), 2.5, device="cuda")
    ctx.weight_grad(R, Q, dW=dW)
    torch.cuda.synchronize()
    assert bool(torch.all(dW == 2.5))
    # accumulation: two calls add
    tR, tQ = _operands(4, 4, 4, 128, 64, 3, torch.bfloat16)
    a = ctx.weight_grad(tR.cuda(), tQ.cuda())
    b = ctx.weight_grad(tR.cuda(), tQ.cuda(), dW=a.clone())
    torch.cuda.synchronize()
    assert torch.allclose(b, 2 * a, rtol=1e-5, atol=1e-6)


def test_argument_errors(ctx):
    import paper_1910_02480_gb300 as m
    R = torch.zeros((2, 4, 4, 128), dtype=torch.bfloat16, device="cuda")
    Q = torch.zeros((2, 8, 8, 64), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(ValueError):
        ctx.weight_grad(R, Q.float())
    with pytest.raises(ValueError):
        ctx.weight_grad(R, Q[:, :6])
    with pytest.raises(m.DrcError):
        ctx.weight_grad(R, Q, qraw=65)
