"""Pins of the oracle's indirect-term estimator (Sec. 3.2 with Eq. 3): the
hemisphere integral of f_r cos R over the blended cached maps, estimated by
multiple importance sampling between the maps (as environment maps) and the
BRDF.  The quadrature of its expectation is pinned by closed forms; the
estimator by unbiasedness against that quadrature over many independent
sample sets."""
import math

import numpy as np
import pytest

import oracle

H = W = 16


def _frame_normal(rng, n):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _scene(seed=0, n=3, P=5, zero_frac=0.2):
    """n caches with skewed random radiance (some texels exactly zero), P
    pixels whose normals lie within about 60 degrees of their caches', the k = n
    caches with random normalised weights."""
    rng = np.random.default_rng(seed)
    maps = rng.gamma(0.5, 1.0, size=(n, 3, H, W))
    maps[rng.uniform(size=maps.shape) < zero_frac] = 0.0
    cn = _frame_normal(rng, n)
    base = cn.mean(axis=0)
    base /= np.linalg.norm(base)
    pn = base + 0.5 * rng.standard_normal((P, 3))
    pn /= np.linalg.norm(pn, axis=1, keepdims=True)
    idx = np.tile(np.arange(n, dtype=np.int32), (P, 1))
    w = rng.dirichlet(np.ones(n), size=P)
    alb = rng.uniform(0.2, 0.9, size=(P, 3))
    return {"maps": maps, "nrm": cn}, idx, w, pn, alb


def _one(c_rgb, cache_n, pixel_n):
    maps = np.broadcast_to(np.asarray(c_rgb, dtype=np.float64)[None, :, None, None], (1, 3, H, W)).copy()
    caches = {"maps": maps, "nrm": np.asarray([cache_n], dtype=np.float64)}
    return caches, np.zeros((1, 1), np.int32), np.ones((1, 1)), np.asarray([pixel_n], dtype=np.float64)


def test_expectation_closed_forms():
    """Constant radiance c, one cache: the integral of (albedo / pi) cos c
    over the pixel hemisphere where it meets the cache hemisphere -- all of
    it for equal normals (albedo c; exact, the cosine is linear in the
    quadrature's cos-theta midpoints), none for opposite ones, half of the
    cosine-weighted hemisphere (albedo c / 2) for orthogonal ones."""
    alb = np.array([[0.5, 0.7, 0.9]])
    c = [1.0, 2.0, 3.0]
    for cn, pn, factor, tol in (((0, 0, 1), (0, 0, 1), 1.0, 1e-12), ((0.3, -0.4, 0.866), (0.3, -0.4, 0.866), 1.0, 1e-9),
                                ((0, 0, 1), (0, 0, -1), 0.0, 1e-15), ((1, 0, 0), (0, 0, 1), 0.5, 2e-3)):
        cn = np.asarray(cn) / np.linalg.norm(cn)
        pn = np.asarray(pn) / np.linalg.norm(pn)
        got = oracle.indirect_expected(*_one(c, cn, pn), alb, m=32)
        a32 = alb.astype(np.float32).astype(np.float64)  # the oracle reads float32 inputs
        np.testing.assert_allclose(got, factor * a32 * np.asarray(c), rtol=tol, atol=1e-15)


def test_zero_radiance_gives_zero():
    caches, idx, w, pn = _one([0.0, 0.0, 0.0], (0, 0, 1), (0, 0, 1))
    u = np.random.default_rng(0).uniform(size=(1, 8, 4))
    assert np.all(oracle.mis_indirect(caches, idx, w, pn, np.ones((1, 3)), u) == 0.0)


def _unbiased(caches, idx, w, pn, alb, S, T, seed):
    P = idx.shape[0]
    rep = lambda a: np.repeat(a, T, axis=0)
    u = np.random.default_rng(seed).uniform(size=(P * T, S, 4))
    est = oracle.mis_indirect(caches, rep(idx), rep(w), rep(pn), rep(alb), u).reshape(P, T, 3)
    mean, se = est.mean(axis=1), est.std(axis=1, ddof=1) / math.sqrt(T)
    ref = oracle.indirect_expected(caches, idx, w, pn, alb, m=16)
    assert np.all(se > 0)
    assert np.all(np.abs(mean - ref) <= 5.0 * se + 2e-3 * np.abs(ref)), (mean, ref, se)
    return mean, ref, se


@pytest.mark.parametrize("S", [8, 3, 1])
def test_estimator_is_unbiased(S):
    """Alternating environment / BRDF samples (S = 8, and an odd count whose
    environment samples outnumber the BRDF ones), and environment samples
    alone (S = 1): the mean of 4000 independent estimates per pixel is the
    quadrature within five standard errors."""
    _unbiased(*_scene(seed=S), S=S, T=4000, seed=100 + S)


def test_estimator_with_dark_and_bright_texels():
    """Maps whose radiance sits in a few bright texels (most exactly zero):
    the environment technique only draws lit texels, the BRDF technique
    covers the rest; still unbiased."""
    caches, idx, w, pn, alb = _scene(seed=11, zero_frac=0.9)
    _unbiased(caches, idx, w, pn, alb, S=4, T=6000, seed=12)


def test_argument_errors():
    caches, idx, w, pn, alb = _scene()
    with pytest.raises(ValueError):
        oracle.mis_indirect(caches, idx, w[:, :2], pn, alb, np.zeros((5, 2, 4)))
    with pytest.raises(ValueError):
        oracle.mis_indirect(caches, idx, w, pn, alb, np.zeros((5, 2, 3)))


def test_texel_geometry_closed_forms():
    """Aligned normals, light in one texel row or column only: row 0 (polar
    angle below pi / 2H) gives albedo c sin^2(pi / 2H), the cosine-weighted
    solid angle of the polar cap over pi; one column gives albedo c / W (the
    cosine is symmetric in azimuth).  This fixes the rows' order and the
    columns' width, which constant maps cannot see."""
    alb = np.array([[1.0, 1.0, 1.0]])
    row = np.zeros((1, 3, H, W))
    row[0, :, 0, :] = 2.0
    col = np.zeros((1, 3, H, W))
    col[0, :, :, 5] = 2.0
    one = lambda m: ({"maps": m, "nrm": np.array([[0.0, 0.0, 1.0]])}, np.zeros((1, 1), np.int32), np.ones((1, 1)),
                     np.array([[0.0, 0.0, 1.0]]), alb)
    np.testing.assert_allclose(oracle.indirect_expected(*one(row)), 2.0 * math.sin(math.pi / (2 * H)) ** 2, rtol=1e-12)
    np.testing.assert_allclose(oracle.indirect_expected(*one(col)), 2.0 / W, rtol=1e-12)
    # and the estimator agrees (4000 independent estimates of one pixel)
    T = 4000
    caches = one(row)[0]
    u = np.random.default_rng(5).uniform(size=(T, 4, 4))
    est = oracle.mis_indirect(caches, np.zeros((T, 1), np.int32), np.ones((T, 1)), np.tile([[0.0, 0.0, 1.0]], (T, 1)),
                              np.ones((T, 3)), u)
    mean, se = est.mean(axis=0), est.std(axis=0, ddof=1) / math.sqrt(T)
    assert np.all(np.abs(mean - 2.0 * math.sin(math.pi / (2 * H)) ** 2) <= 5 * se + 1e-12)


def test_decision_margin_leaves_the_estimate_alone_and_flags_a_grazing_direction():
    """The margin output reports, in units of float32 error, how close a
    sample's continuous-valued decisions come to changing; asking for it does
    not change the estimate, and a BRDF sample that grazes the pixel's
    horizon (cosine 0) gives a margin below 1."""
    caches, idx, w, pn, alb = _scene(seed=3, n=3, P=4)
    u = np.random.default_rng(4).uniform(0.0, 1.0, size=(4, 6, 4))
    a = oracle.mis_indirect(caches, idx, w, pn, alb, u)
    b, m = oracle.mis_indirect(caches, idx, w, pn, alb, u, want_margin=True)
    np.testing.assert_array_equal(a, b)
    assert np.all(m >= 0.0)
    u2 = u.copy()
    u2[1, 1, 1] = 1.0  # odd sample: BRDF, sqrt(1 - u1) = 0, the direction lies in the tangent plane
    _, m2 = oracle.mis_indirect(caches, idx, w, pn, alb, u2, want_margin=True)
    assert m2[1] < 1.0
    np.testing.assert_array_equal(m2[[0, 2, 3]], m[[0, 2, 3]])


def test_choices_taken_in_float32_keep_the_estimate_unbiased():
    """The map and texel choices, taken from float32 running sums, follow
    the same distributions: the estimate over many independent sample sets
    still averages to the quadrature of its expectation."""
    caches, idx, w, pn, alb = _scene(seed=5, n=3, P=2)
    exp = oracle.indirect_expected(caches, idx, w, pn, alb, m=16)
    reps, S = 3000, 4
    rng = np.random.default_rng(6)
    u = rng.uniform(0.0, 1.0, size=(reps, 2, S, 4)).astype(np.float32).astype(np.float64)
    est = np.stack([oracle.mis_indirect(caches, idx, w, pn, alb, u[r]) for r in range(reps)])
    mean, se = est.mean(0), est.std(0) / np.sqrt(reps)
    assert np.all(np.abs(mean - exp) <= 5 * se + 1e-12)
