"""Pins of the oracle's paper-form network (Sec. 3.3, "Neural network"): a
U-Net of two 3x3 convolutions per stage with batch normalisation and
LeakyReLU, 2x2 max pooling, 2x bilinear upsampling, concatenated skips and a
1x1 head with ReLU.  Each part is pinned against PyTorch's float64
operators or a closed form, and the whole network against the same network
written with PyTorch's functional operators."""
import numpy as np
import pytest

import oracle
from paper_1910_02480_gb300 import synth

torch = pytest.importorskip("torch")
F = torch.nn.functional


def _t(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float64))


def test_conv3x3s1_against_torch_and_concat():
    rng = np.random.default_rng(0)
    x1 = rng.standard_normal((2, 3, 5, 7))
    x2 = rng.standard_normal((2, 2, 5, 7))
    w = rng.standard_normal((4, 5, 3, 3))
    b = rng.standard_normal(4)
    y = oracle.conv3x3s1(x1, w, b, x2=x2)
    ref = F.conv2d(torch.cat([_t(x1), _t(x2)], 1), _t(w), _t(b), padding=1).numpy()
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-12)


def test_convT3x3s1_against_torch_and_adjoint():
    """The transposed convolution is the adjoint of the convolution with the
    same weights: <conv(x), y> = <x, convT(y)>."""
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 6, 4))
    w = rng.standard_normal((3, 5, 3, 3))  # [Cin][Cout] of the transposed conv
    b = rng.standard_normal(5)
    y = oracle.convT3x3s1(x, w, b)
    ref = F.conv_transpose2d(_t(x), _t(w), _t(b), padding=1).numpy()
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-12)
    z = rng.standard_normal((2, 5, 6, 4))
    # conv with the same tensor read as [Cout'=3][Cin'=5]: maps 5 -> 3 channels
    lhs = np.sum(oracle.conv3x3s1(z, w) * x)
    rhs = np.sum(z * oracle.convT3x3s1(x, w))
    assert lhs == pytest.approx(rhs, rel=1e-12)
    # the concatenated form splits the channels
    x2 = rng.standard_normal((2, 2, 6, 4))
    w5 = rng.standard_normal((5, 5, 3, 3))
    np.testing.assert_allclose(oracle.convT3x3s1(x, w5, b, x2=x2),
                               F.conv_transpose2d(torch.cat([_t(x), _t(x2)], 1), _t(w5), _t(b), padding=1).numpy(),
                               rtol=1e-12, atol=1e-12)


def test_maxpool2():
    x = np.array([[1.0, 5.0, -2.0, 0.0], [3.0, 2.0, -1.0, -3.0], [0.0, 0.0, 7.0, 7.0], [-1.0, 0.0, 6.0, 8.0]])
    np.testing.assert_array_equal(oracle.maxpool2(x[None, None])[0, 0], [[5.0, 0.0], [0.0, 8.0]])
    r = np.random.default_rng(2).standard_normal((2, 3, 8, 6))
    np.testing.assert_array_equal(oracle.maxpool2(r), F.max_pool2d(_t(r), 2).numpy())


def test_upsample2_closed_forms_and_torch():
    """A constant map stays constant; a ramp f = i (rows) comes out as the
    half-pixel source coordinate (p + 1/2)/2 - 1/2 away from the borders,
    and as the first / last row at them."""
    H = 6
    ramp = np.tile(np.arange(H, dtype=np.float64)[:, None], (1, 4))[None, None]
    up = oracle.upsample2(ramp)[0, 0]
    for p in range(2 * H):
        s = (p + 0.5) / 2 - 0.5
        np.testing.assert_allclose(up[p], min(max(s, 0.0), H - 1.0), rtol=0, atol=1e-15)
    np.testing.assert_allclose(oracle.upsample2(np.full((1, 2, 3, 5), 2.5)), 2.5, rtol=0, atol=1e-15)
    r = np.random.default_rng(3).standard_normal((2, 3, 4, 7))
    ref = F.interpolate(_t(r), scale_factor=2, mode="bilinear", align_corners=False).numpy()
    np.testing.assert_allclose(oracle.upsample2(r), ref, rtol=1e-12, atol=1e-13)


def _torch_unet(params, x, base, levels, cin=7, cout=3):
    """The same network from PyTorch's functional operators, reading the
    packed parameters in order (and checking that it reads all of them)."""
    p = _t(params)
    off = [0]

    def take(*shape):
        n = int(np.prod(shape))
        t = p[off[0]:off[0] + n].reshape(shape)
        off[0] += n
        return t

    def act(z, c, bn):
        if bn:
            g, be, mu, var = take(c), take(c), take(c), take(c)
            z = F.batch_norm(z, mu, var, g, be, training=False, eps=1e-5)
        return F.leaky_relu(z, 0.01)

    z = _t(x)
    enc = []
    for lvl in range(levels + 1):
        c = base << lvl
        if lvl > 0:
            z = F.max_pool2d(z, 2)
        for _ in range(2):
            w = take(c, z.shape[1], 3, 3)
            z = act(F.conv2d(z, w, take(c), padding=1), c, True)
        enc.append(z)
    d = enc[levels]
    for lvl in range(levels - 1, -1, -1):
        c = base << lvl
        z = torch.cat([F.interpolate(d, scale_factor=2, mode="bilinear", align_corners=False), enc[lvl]], 1)
        for _ in range(2):
            w = take(z.shape[1], c, 3, 3)
            z = act(F.conv_transpose2d(z, w, take(c), padding=1), c, lvl > 0)
        d = z
    out = F.relu(F.conv2d(d, take(cout, base, 1, 1), take(cout)))
    assert off[0] == p.numel()
    return out.numpy()


@pytest.mark.parametrize("base,levels,S", [(8, 2, 16), (4, 3, 32), (4, 1, 8)])
def test_unet_forward_against_torch(base, levels, S):
    params = synth.unet_params(base, levels, seed=base + levels)
    assert params.size == oracle.unet_param_count(base, levels)
    rng = np.random.default_rng(S)
    x = rng.standard_normal((2, 7, S, S)).astype(np.float32)
    y = oracle.unet_forward(params, x, base, levels)
    ref = _torch_unet(params.astype(np.float64), x.astype(np.float64), base, levels)
    np.testing.assert_allclose(y, ref, rtol=1e-10, atol=1e-12)
    assert (y >= 0).all() and (y > 0).any()


def test_unet_shape_errors():
    params = synth.unet_params(4, 2)
    with pytest.raises(ValueError):
        oracle.unet_forward(params, np.zeros((1, 7, 6, 8), np.float32), 4, 2)  # 6 not a multiple of 4
    with pytest.raises(ValueError):
        oracle.unet_forward(params[:-1], np.zeros((1, 7, 8, 8), np.float32), 4, 2)
