"""Pins of the oracle's convolutions and network (Sec. 3.3) against values the
mathematics fixes: hand-worked examples, an independent im2col formulation,
PyTorch's float64 CPU convolutions, the adjoint identity, delta kernels, a
closed-form network and linearity."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1910_02480_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_handworked_conv_and_convT():
    g = json.load(open(os.path.join(GOLD, "conv_handworked.json")))
    w = np.ones((1, 1, 3, 3))
    x = np.array(g["conv"]["x"], dtype=np.float64)[None, None]
    np.testing.assert_array_equal(oracle.conv3x3s2(x, w)[0, 0], g["conv"]["y"])
    x = np.array(g["convT"]["x"], dtype=np.float64)[None, None]
    np.testing.assert_array_equal(oracle.convT3x3s2(x, w)[0, 0], g["convT"]["y"])


def _im2col_conv(x, w, b):
    """Independent formulation: zero-pad, gather the 3x3 patch at every
    stride-2 position into a matrix, multiply by the flattened kernels."""
    N, C, H, W = x.shape
    Co = w.shape[0]
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    Ho, Wo = H // 2, W // 2
    cols = np.empty((N, Ho, Wo, C, 3, 3))
    for u in range(3):
        for v in range(3):
            cols[..., u, v] = xp[:, :, u:u + 2 * Ho:2, v:v + 2 * Wo:2].transpose(0, 2, 3, 1)
    y = cols.reshape(N * Ho * Wo, C * 9) @ w.reshape(Co, C * 9).T + b
    return y.reshape(N, Ho, Wo, Co).transpose(0, 3, 1, 2)


def _dilate_convT(x, w, b):
    """Independent formulation of the transposed conv: insert zeros between
    input pixels, pad (1 before, 2 after), correlate with the flipped and
    transposed kernel at stride 1."""
    N, C, H, W = x.shape
    Co = w.shape[1]
    z = np.zeros((N, C, 2 * H - 1, 2 * W - 1))
    z[:, :, ::2, ::2] = x
    zp = np.pad(z, ((0, 0), (0, 0), (1, 2), (1, 2)))
    wf = w[:, :, ::-1, ::-1].transpose(1, 0, 2, 3)  # [Co, C, 3, 3]
    y = np.zeros((N, Co, 2 * H, 2 * W))
    for u in range(3):
        for v in range(3):
            y += np.einsum("nchw,oc->nohw", zp[:, :, u:u + 2 * H, v:v + 2 * W], wf[:, :, u, v])
    return y + b[None, :, None, None]


@pytest.mark.parametrize("N,C,Co,H", [(1, 1, 1, 4), (2, 3, 2, 4), (2, 3, 5, 8), (1, 7, 4, 6)])
def test_conv_brute_force(N, C, Co, H):
    rng = np.random.default_rng(10 + H + C)
    x = rng.normal(size=(N, C, H, H))
    w = rng.normal(size=(Co, C, 3, 3))
    b = rng.normal(size=Co)
    np.testing.assert_allclose(oracle.conv3x3s2(x, w, b), _im2col_conv(x, w, b), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("N,C,Co,H", [(1, 1, 1, 2), (2, 3, 2, 4), (2, 2, 5, 3), (1, 4, 3, 5)])
def test_convT_brute_force(N, C, Co, H):
    rng = np.random.default_rng(20 + H + C)
    x = rng.normal(size=(N, C, H, H + 1))
    w = rng.normal(size=(C, Co, 3, 3))
    b = rng.normal(size=Co)
    np.testing.assert_allclose(oracle.convT3x3s2(x, w, b), _dilate_convT(x, w, b), rtol=1e-12, atol=1e-12)


def test_against_torch_float64():
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    rng = np.random.default_rng(3)
    x = rng.normal(size=(2, 5, 8, 8))
    w = rng.normal(size=(6, 5, 3, 3))
    b = rng.normal(size=6)
    ref = F.conv2d(torch.from_numpy(x), torch.from_numpy(w), torch.from_numpy(b), stride=2, padding=1)
    np.testing.assert_allclose(oracle.conv3x3s2(x, w, b), ref.numpy(), rtol=1e-12, atol=1e-12)
    xt = rng.normal(size=(2, 6, 4, 4))
    wt = rng.normal(size=(6, 3, 3, 3))
    bt = rng.normal(size=3)
    ref = F.conv_transpose2d(torch.from_numpy(xt), torch.from_numpy(wt), torch.from_numpy(bt),
                             stride=2, padding=1, output_padding=1)
    np.testing.assert_allclose(oracle.convT3x3s2(xt, wt, bt), ref.numpy(), rtol=1e-12, atol=1e-12)


def test_adjoint_identity():
    """<conv_W(x), y> = <x, convT_W(y)> for the same kernel array, b = 0."""
    rng = np.random.default_rng(4)
    x = rng.normal(size=(2, 3, 8, 8))
    y = rng.normal(size=(2, 5, 4, 4))
    w = rng.normal(size=(5, 3, 3, 3))
    lhs = np.sum(oracle.conv3x3s2(x, w) * y)
    rhs = np.sum(x * oracle.convT3x3s2(y, w))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_delta_kernels():
    rng = np.random.default_rng(5)
    x = rng.normal(size=(2, 3, 8, 8))
    w = np.zeros((3, 3, 3, 3))
    for c in range(3):
        w[c, c, 1, 1] = 1.0
    np.testing.assert_array_equal(oracle.conv3x3s2(x, w), x[:, :, ::2, ::2])
    y = oracle.convT3x3s2(x, w)
    z = np.zeros((2, 3, 16, 16))
    z[:, :, ::2, ::2] = x
    np.testing.assert_array_equal(y, z)


def _delta_net(widths, biases, dec_scale):
    """Packed weights for cin=7, cout=3 whose taps are all centre deltas."""
    parts = []
    for kind, wshape, blen in synth.layer_shapes(widths):
        w = np.zeros(wshape)
        if kind == "conv":
            for c in range(min(wshape[0], wshape[1])):
                w[c, c, 1, 1] = 1.0
        else:
            for c in range(min(wshape[0], wshape[1])):
                w[c, c, 1, 1] = dec_scale
        parts += [w.ravel(), np.full(blen, biases[len(parts) // 2])]
    return np.concatenate(parts).astype(np.float32)


def test_delta_network_closed_form():
    """Centre-delta kernels make every layer a subsample / zero insertion, so
    the network has a closed form; the biases separate 'ReLU then add the skip'
    from 'add the skip then ReLU'."""
    widths = [8, 8]
    biases = [0.25, -0.125, -0.5, 0.375]  # conv1, conv2, convT2, convT1
    wts = _delta_net(widths, biases, -1.0)
    rng = np.random.default_rng(6)
    x = rng.normal(size=(2, 7, 8, 8)).astype(np.float32)
    out = oracle.forward(wts, x, widths)
    xd = x.astype(np.float64)
    relu = lambda a: np.maximum(a, 0.0)
    e1 = np.full((2, 8, 4, 4), biases[0])
    e1[:, :7] += xd[:, :, ::2, ::2]
    e1 = relu(e1)
    e2 = relu(e1[:, :, ::2, ::2] + biases[1])
    zd = np.full((2, 8, 4, 4), biases[2])
    zd[:, :, ::2, ::2] += -e2
    t1 = relu(zd) + e1
    ref = np.full((2, 3, 8, 8), biases[3])
    ref[:, :, ::2, ::2] += -t1[:, :3]
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-15)


def test_linearity_when_relus_are_inactive():
    """With non-negative weights and inputs and b = 0 every ReLU passes its
    input through, so the network is linear: f(a x + b y) = a f(x) + b f(y)."""
    widths = [8, 16]
    w = np.abs(synth.he_weights(widths, seed=9)).astype(np.float32)
    rng = np.random.default_rng(7)
    # dyadic inputs, so that a x + b y is exact in float32 as well
    x = (rng.integers(0, 256, size=(2, 7, 8, 8)) / 256.0).astype(np.float32)
    y = (rng.integers(0, 256, size=(2, 7, 8, 8)) / 256.0).astype(np.float32)
    a, b = 0.75, 1.5
    z = (a * x.astype(np.float64) + b * y.astype(np.float64)).astype(np.float32)
    assert np.array_equal(z.astype(np.float64), a * x.astype(np.float64) + b * y.astype(np.float64))
    fz = oracle.forward(w, z, widths)
    ref = a * oracle.forward(w, x, widths) + b * oracle.forward(w, y, widths)
    np.testing.assert_allclose(fz, ref, rtol=1e-12, atol=1e-12)


def test_network_by_layers_matches_forward():
    """The network equals the composition of the single layers with ReLU and
    skip-add written out here (topology of Sec. 3.3, random weights)."""
    widths = [8, 16, 16]
    wts = synth.he_weights(widths, seed=11, bias=True)
    layers = synth.unpack_weights(wts.astype(np.float64), widths)
    rng = np.random.default_rng(8)
    x = rng.normal(size=(2, 7, 16, 16)).astype(np.float32)
    e = [x.astype(np.float64)]
    for s in range(3):
        e.append(np.maximum(oracle.conv3x3s2(e[-1], *layers[s]), 0))
    t = e[3]
    for q, s in enumerate([3, 2]):
        t = np.maximum(oracle.convT3x3s2(t, *layers[3 + q]), 0) + e[s - 1]
    ref = oracle.convT3x3s2(t, *layers[5])
    np.testing.assert_allclose(oracle.forward(wts, x, widths), ref, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(oracle.forward(wts, x, widths, out_relu=True), np.maximum(ref, 0),
                               rtol=1e-13, atol=1e-13)


def test_encode_decode():
    widths = [8]
    wts = synth.he_weights(widths, seed=12, bias=True)
    rng = np.random.default_rng(9)
    L = rng.uniform(0.0, 50.0, size=(2, 7, 4, 4)).astype(np.float32)
    s = 0.5
    enc = L.astype(np.float64).copy()
    enc[:, :3] = np.log1p(s * enc[:, :3])
    y = oracle.forward(wts, enc.astype(np.float32), widths)
    # the oracle encodes in double, the reference above rounds the encoded
    # input to float32 first: compare at float32 input precision
    y_enc = oracle.forward(wts, L, widths, exposure=s, flags=oracle.F_ENCODE_INPUT)
    np.testing.assert_allclose(y_enc, y, rtol=0, atol=1e-5)
    y_dec = oracle.forward(wts, L, widths, exposure=s, flags=oracle.F_ENCODE_INPUT | oracle.F_DECODE_OUTPUT)
    np.testing.assert_allclose(y_dec, np.expm1(y_enc) / s, rtol=1e-14, atol=0)


def test_weight_count_matches_layer_table():
    for widths in ([32, 64, 128], [64, 128, 256], [64, 128, 256, 512], [16]):
        assert oracle.weight_count(widths) == synth.weight_count(widths)
    assert oracle.weight_count([32, 64, 128]) == 187523
    with pytest.raises(ValueError):
        oracle.forward(np.zeros(10, np.float32), np.zeros((1, 7, 8, 8), np.float32), [8])
