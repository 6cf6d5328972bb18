"""Pins of the oracle's L1 loss and gradient (Sec. 3.3 and Sec. 4 training;
Eq. 7) against central finite differences in double precision, exact zero
loss, and linearity of the vector-Jacobian product in the output gradient."""
import numpy as np
import pytest

import oracle
from paper_1910_02480_gb300 import synth

WIDTHS = [8, 16]


def _case(seed=0, N=2, H=8):
    rng = np.random.default_rng(seed)
    w = synth.he_weights(WIDTHS, seed=seed + 1, bias=True)
    x = rng.uniform(0.0, 2.0, size=(N, 7, H, H)).astype(np.float32)
    y = rng.normal(size=(N, 3, H, H)).astype(np.float32)
    return w, x, y


def _fd_check(w, x, y, which, idx, flags=0, exposure=1.0, out_relu=False, h=2.0 ** -12):
    """Central difference with a perturbation h that is exact in float32 at
    the chosen elements, compared with the analytic gradient."""
    loss, dw, dx = oracle.l1_backward(w, x, y, WIDTHS, flags=flags, exposure=exposure, out_relu=out_relu)
    grads = dw if which == "w" else dx.ravel()
    base = w if which == "w" else x.ravel()
    checked = 0
    for i in idx:
        plus, minus = base.copy(), base.copy()
        plus[i] += h
        minus[i] -= h
        if plus[i] - base[i] != h or base[i] - minus[i] != h:
            continue  # perturbation not exact in float32 at this element
        if which == "w":
            lp = oracle.l1_backward(plus, x, y, WIDTHS, flags=flags, exposure=exposure, out_relu=out_relu)[0]
            lm = oracle.l1_backward(minus, x, y, WIDTHS, flags=flags, exposure=exposure, out_relu=out_relu)[0]
        else:
            lp = oracle.l1_backward(w, plus.reshape(x.shape), y, WIDTHS, flags=flags, exposure=exposure,
                                    out_relu=out_relu)[0]
            lm = oracle.l1_backward(w, minus.reshape(x.shape), y, WIDTHS, flags=flags, exposure=exposure,
                                    out_relu=out_relu)[0]
        fd = (lp - lm) / (2 * h)
        # a kink (|out - y| or a ReLU input crossing 0 inside +-h) makes the
        # central difference differ from both one-sided slopes; detect it by
        # comparing the one-sided differences
        fwd = (lp - loss) / h
        bwd = (loss - lm) / h
        if abs(fwd - bwd) > 1e-6 * max(1.0, abs(fd)) + 1e-9:
            continue
        assert abs(fd - grads[i]) <= 1e-6 * max(abs(fd), 1e-3) + 1e-10, (which, i, fd, grads[i])
        checked += 1
    return checked


@pytest.mark.parametrize("flags,out_relu", [(0, False), (oracle.F_ENCODE_INPUT, True)])
def test_weight_gradient_matches_finite_differences(flags, out_relu):
    w, x, y = _case(1)
    rng = np.random.default_rng(2)
    idx = rng.choice(w.size, size=60, replace=False)
    # include every bias and a few first / last layer taps
    layers = synth.layer_shapes(WIDTHS)
    off = 0
    for _, wshape, blen in layers:
        n = int(np.prod(wshape))
        idx = np.concatenate([idx, [off, off + n - 1, off + n]])
        off += n + blen
    checked = _fd_check(w, x, y, "w", idx, flags=flags, exposure=0.5, out_relu=out_relu)
    assert checked >= 40


def test_input_gradient_matches_finite_differences():
    w, x, y = _case(3)
    rng = np.random.default_rng(4)
    idx = rng.choice(x.size, size=50, replace=False)
    assert _fd_check(w, x, y, "x", idx, flags=oracle.F_ENCODE_INPUT, exposure=2.0) >= 35
    assert _fd_check(w, x, y, "x", idx) >= 35


def test_zero_loss_at_own_prediction():
    w, x, _ = _case(5)
    out = oracle.forward(w, x, WIDTHS)
    loss, dw, dx = oracle.l1_backward(w, x, out.astype(np.float32), WIDTHS)
    # out rounded to float32 differs from the double output by < 1 ulp
    assert 0.0 <= loss < 1e-7
    loss2, _, _ = oracle.l1_backward(w, x, out.astype(np.float32) + 10.0, WIDTHS)
    assert loss2 > 9.0


def test_grad_out_mode_is_linear_and_matches_l1():
    """mode GRAD_OUT returns J^T g, linear in g; feeding g = sign(out - y)/n
    reproduces the L1 gradient."""
    w, x, y = _case(6)
    rng = np.random.default_rng(7)
    g1 = rng.normal(size=y.shape).astype(np.float32)
    g2 = rng.normal(size=y.shape).astype(np.float32)
    _, a1, x1 = oracle.l1_backward(w, x, g1, WIDTHS, grad_out=True)
    _, a2, x2 = oracle.l1_backward(w, x, g2, WIDTHS, grad_out=True)
    _, a3, x3 = oracle.l1_backward(w, x, (g1 + g2).astype(np.float32), WIDTHS, grad_out=True)
    exact = np.array_equal((g1 + g2).astype(np.float64), g1.astype(np.float64) + g2.astype(np.float64))
    tol = 1e-12 if exact else 1e-6
    np.testing.assert_allclose(a3, a1 + a2, rtol=tol, atol=tol)
    np.testing.assert_allclose(x3, x1 + x2, rtol=tol, atol=tol)
    out = oracle.forward(w, x, WIDTHS)
    g = (np.sign(out - y.astype(np.float64)) / out.size).astype(np.float32)
    _, al, xl = oracle.l1_backward(w, x, y, WIDTHS)
    _, ag, xg = oracle.l1_backward(w, x, g, WIDTHS, grad_out=True)
    np.testing.assert_allclose(ag, al, rtol=1e-6, atol=1e-12)


@pytest.mark.parametrize("transposed", [False, True])
def test_layer_weight_gradient_is_the_adjoint_of_the_layer(transposed):
    """A layer without bias is linear in its weights, so the weight gradient
    of <g, layer(x; D)> is exactly the tensor G with <G, D> = <g, layer(x; D)>
    for every D: checked for random D against the (separately pinned)
    conv3x3s2 / convT3x3s2, and on a basis direction per tap (one weight)."""
    rng = np.random.default_rng(11 + transposed)
    N, Cin, Cout, H, W = 3, 5, 4, 6, 10
    x = rng.normal(size=(N, Cin, H, W))
    if transposed:
        g = rng.normal(size=(N, Cout, 2 * H, 2 * W))
        layer, shape = oracle.convT3x3s2, (Cin, Cout, 3, 3)
    else:
        g = rng.normal(size=(N, Cout, H // 2, W // 2))
        layer, shape = oracle.conv3x3s2, (Cout, Cin, 3, 3)
    G = oracle.conv_weight_grad(x, g, transposed=transposed)
    assert G.shape == shape
    for _ in range(3):
        D = rng.normal(size=shape)
        lhs = float(np.sum(G * D))
        rhs = float(np.sum(g * layer(x, D)))
        assert abs(lhs - rhs) <= 1e-12 * (np.sum(np.abs(G * D)) + 1.0)
    for t in range(9):  # each tap (u, v) separately: catches a swapped or shifted tap
        D = np.zeros(shape)
        D[1, 2, t // 3, t % 3] = 1.0
        assert abs(G[1, 2, t // 3, t % 3] - np.sum(g * layer(x, D))) <= 1e-12 * np.sum(np.abs(g)) * np.abs(x).max()


def test_layer_weight_gradient_brute_force():
    """Direct sum from the definition on a tiny conv: dW[o][c][u][v] = sum over
    n, i, j of g[n,o,i,j] x[n,c,2i+u-1,2j+v-1], zero outside the input."""
    rng = np.random.default_rng(5)
    x = rng.normal(size=(2, 2, 4, 6))
    g = rng.normal(size=(2, 3, 2, 3))
    ref = np.zeros((3, 2, 3, 3))
    for n in range(2):
        for o in range(3):
            for c in range(2):
                for u in range(3):
                    for v in range(3):
                        for i in range(2):
                            for j in range(3):
                                y, xx = 2 * i + u - 1, 2 * j + v - 1
                                if 0 <= y < 4 and 0 <= xx < 6:
                                    ref[o, c, u, v] += g[n, o, i, j] * x[n, c, y, xx]
    np.testing.assert_allclose(oracle.conv_weight_grad(x, g), ref, rtol=1e-13, atol=1e-13)
