"""Pins of the oracle's training pieces (Sec. 4): the map augmentation by
rotation and flipping, and the Adam step (Kingma & Ba 2015, Alg. 1)."""
import math

import numpy as np
import pytest

import oracle


def _maps(seed=0, N=8, C=3, H=6):
    return np.random.default_rng(seed).standard_normal((N, C, H, H))


# ---------------------------------------------------------------- augment


@pytest.mark.parametrize("code", range(8))
def test_augment_matches_numpy_rot90_and_flip(code):
    """code = r + 4 f: a column mirror (f), then r counter-clockwise quarter
    turns -- numpy's flip and rot90 of the (H, W) axes."""
    x = _maps(code)
    y = oracle.augment(x, [code] * len(x))
    f, r = divmod(code, 4)
    ref = np.rot90(np.flip(x, axis=-1) if f else x, k=r, axes=(-2, -1))
    np.testing.assert_array_equal(y, ref)


def test_augment_hand_worked_2x2():
    x = np.array([[1.0, 2.0], [3.0, 4.0]])[None, None]
    one_turn = oracle.augment(x, [1])[0, 0]
    mirror = oracle.augment(x, [4])[0, 0]
    np.testing.assert_array_equal(one_turn, [[2.0, 4.0], [1.0, 3.0]])
    np.testing.assert_array_equal(mirror, [[2.0, 1.0], [4.0, 3.0]])


def test_augment_group_identities():
    """Four quarter turns and two mirrors are the identity; a mirror then a
    turn is code 5; the eight images of a generic map are distinct, each a
    permutation of the map; every channel moves alike."""
    x = _maps(1, N=1, C=2, H=5)
    y = x
    for _ in range(4):
        y = oracle.augment(y, [1])
    np.testing.assert_array_equal(y, x)
    np.testing.assert_array_equal(oracle.augment(oracle.augment(x, [4]), [4]), x)
    np.testing.assert_array_equal(oracle.augment(oracle.augment(x, [4]), [1]), oracle.augment(x, [5]))
    imgs = [oracle.augment(x, [c])[0] for c in range(8)]
    for a in range(8):
        np.testing.assert_array_equal(np.sort(imgs[a].ravel()), np.sort(x[0].ravel()))
        for b in range(a):
            assert not np.array_equal(imgs[a], imgs[b])
    idx = np.arange(25.0).reshape(5, 5)
    both = np.stack([idx, idx + 100.0])[None]
    for c in range(8):
        z = oracle.augment(both, [c])[0]
        np.testing.assert_array_equal(z[1], z[0] + 100.0)


def test_augment_codes_per_map_and_errors():
    x = _maps(2, N=3)
    y = oracle.augment(x, [0, 3, 6])
    for n, c in enumerate([0, 3, 6]):
        np.testing.assert_array_equal(y[n], oracle.augment(x[n:n + 1], [c])[0])
    with pytest.raises(ValueError):
        oracle.augment(np.zeros((1, 1, 2, 3)), [0])
    with pytest.raises(ValueError):
        oracle.augment(x, [0, 1, 8])


# ------------------------------------------------------------------- Adam


def test_adam_first_step_closed_form():
    """From m = v = 0, step 1 has m^ = g and v^ = g^2, so the update is
    -lr g / (|g| + eps): about -lr sign(g), exactly 0 for g = 0."""
    g = np.array([0.3, -1e-3, 0.0, 5.0, -7e-9])
    w0 = np.array([1.0, -2.0, 0.5, 0.0, 3.0])
    lr, eps = 6e-5, 1e-8
    w, m, v = oracle.adam_step(w0, g, np.zeros(5), np.zeros(5), 1, lr=lr, eps=eps)
    # w - w0 carries the rounding of w at |w0| <= 3: a few 1e-16
    np.testing.assert_allclose(w - w0, -lr * g / (np.abs(g) + eps), rtol=1e-12, atol=2e-15)
    # 1 - b1 and 1 - b2 are not exactly 0.1 and 0.001 in binary: 1e-15 apart
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-14)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-14)


def test_adam_constant_gradient_keeps_the_step():
    """With a constant gradient the bias corrections are exact: m^ = g and
    v^ = g^2 at every t, so every step moves w by -lr g / (|g| + eps)."""
    g = np.array([0.7, -0.02, 3.0])
    w = np.zeros(3)
    m = np.zeros(3)
    v = np.zeros(3)
    for t in range(1, 7):
        w_prev = w
        w, m, v = oracle.adam_step(w, g, m, v, t, lr=1e-3, eps=1e-8)
        np.testing.assert_allclose(w - w_prev, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-10)


def test_adam_hand_worked_two_steps():
    """Scalar, lr = 0.1, eps = 0, g = 1 then 2.  Step 1: m = 0.1, v = 0.001,
    m^ = v^ / v^ ... = 1, so w -= 0.1.  Step 2: m = 0.9 * 0.1 + 0.1 * 2 = 0.29,
    v = 0.999 * 0.001 + 0.001 * 4 = 0.004999, 1 - 0.9^2 = 0.19,
    1 - 0.999^2 = 0.001999: w -= 0.1 (29/19) / sqrt(4999/1999)."""
    w, m, v = oracle.adam_step([2.0], [1.0], [0.0], [0.0], 1, lr=0.1, eps=0.0)
    assert w[0] == pytest.approx(1.9, abs=1e-15)
    w, m, v = oracle.adam_step(w, [2.0], m, v, 2, lr=0.1, eps=0.0)
    assert m[0] == pytest.approx(0.29, rel=1e-15)
    assert v[0] == pytest.approx(0.004999, rel=1e-14)
    assert w[0] == pytest.approx(1.9 - 0.1 * (29 / 19) / math.sqrt(4999 / 1999), rel=1e-14)


def test_adam_zero_gradient_moves_nothing():
    w0 = np.array([1.0, -1.0])
    w, m, v = oracle.adam_step(w0, np.zeros(2), np.zeros(2), np.zeros(2), 1)
    np.testing.assert_array_equal(w, w0)
    assert not m.any() and not v.any()


def test_adam_update_bound():
    """Kingma & Ba, Sec. 2.1: with (1 - b1) > sqrt(1 - b2) every step is at
    most lr (1 - b1) / sqrt(1 - b2) in size (eps = 0), whatever the
    gradients."""
    rng = np.random.default_rng(3)
    n = 1000
    w, m, v = np.zeros(n), np.zeros(n), np.zeros(n)
    lr = 1e-2
    bound = lr * 0.1 / math.sqrt(0.001)
    for t in range(1, 30):
        g = rng.standard_normal(n) * 10.0 ** rng.uniform(-6, 3, size=n)
        w_prev = w
        w, m, v = oracle.adam_step(w, g, m, v, t, lr=lr, eps=0.0)
        assert np.max(np.abs(w - w_prev)) <= bound * (1 + 1e-12)
