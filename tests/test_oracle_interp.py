"""Pins of the oracle's hemisphere integral (Eq. 2, Sec. 3.3) and cache
interpolation (Sec. 3.2) against closed forms, invariants, library sorts and
hand-worked lookups."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1910_02480_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- payload --

def test_payload_constant_map_is_exact():
    """E/pi of a constant map L is L: the band weights telescope to 1/2 and
    the azimuth sums to 2 pi."""
    for H, W in [(1, 1), (8, 8), (32, 32), (16, 24)]:
        L = np.full((2, 3, H, W), 1.0)
        L[1] *= 3.25
        p = oracle.payload(L)
        np.testing.assert_allclose(p, [[1, 1, 1], [3.25, 3.25, 3.25]], rtol=1e-14)


def test_payload_cosine_map_converges_to_two_thirds():
    """L = cos(theta) at texel centres: (1/pi) int cos^2 dOmega = 2/3, with the
    midpoint-rule error shrinking as 1/H^2."""
    errs = []
    for H in (8, 16, 32, 64, 128, 256):
        th = (np.arange(H) + 0.5) * (np.pi / 2) / H
        L = np.broadcast_to(np.cos(th)[:, None], (H, 16))[None, None]
        e = abs(oracle.payload(L)[0, 0] - 2.0 / 3.0)
        assert e < 0.5 / H ** 2
        errs.append(e)
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(ratios > 3.5) and np.all(ratios < 4.5)


def test_payload_azimuthal_harmonic_vanishes():
    """A map 1 + cos(phi) at column centres integrates to exactly 1 (the
    cosine sums to zero over a full turn of evenly spaced columns)."""
    W = 16
    ph = (np.arange(W) + 0.5) * 2 * np.pi / W
    L = np.broadcast_to(1 + np.cos(ph)[None, :], (8, W))[None, None]
    assert abs(oracle.payload(L)[0, 0] - 1.0) < 1e-14


# ----------------------------------------------------------- interpolation --

def _small_scene(width=24, height=16, gx=6, gy=4, seed=2):
    g = synth.gbuffer(width, height, seed=seed)
    c = synth.cache_grid(g, gx, gy)
    rng = np.random.default_rng(seed + 100)
    c["payload"] = rng.uniform(0.0, 2.0, size=(gx * gy, 3)).astype(np.float32)
    return g, c


@pytest.mark.parametrize("metric", [oracle.METRIC_IMAGE, oracle.METRIC_WORLD])
@pytest.mark.parametrize("k", [1, 4, 8])
def test_knn_matches_library_sort(metric, k):
    g, c = _small_scene()
    r = 4.0 if metric == oracle.METRIC_IMAGE else 0.3
    _, idx, d2 = oracle.interpolate(c, g, k, metric, oracle.WP_INVERSE, oracle.INTERP_IRRADIANCE,
                                    r, want_neighbors=True)
    P = g["width"] * g["height"]
    n = c["pos"].shape[0]
    px, py = np.arange(P) % g["width"], np.arange(P) // g["width"]
    if metric == oracle.METRIC_IMAGE:
        D = ((px[:, None] - c["pix"][None, :, 0]) ** 2 + (py[:, None] - c["pix"][None, :, 1]) ** 2).astype(np.float64)
    else:
        D = np.sum((g["pos"][:, None, :].astype(np.float64) - c["pos"][None].astype(np.float64)) ** 2, axis=2)
    for p in range(P):
        order = np.lexsort((np.arange(n), D[p]))  # by distance, then index
        np.testing.assert_array_equal(idx[p], order[:k])
        np.testing.assert_array_equal(d2[p, :k + 1], D[p, order[:k + 1]])


def test_weights_normalised_and_constant_reproduced():
    g, c = _small_scene()
    for metric, r in [(oracle.METRIC_IMAGE, 4.0), (oracle.METRIC_WORLD, 0.3)]:
        for wp in (oracle.WP_INVERSE, oracle.WP_LINEAR):
            ones = dict(c, payload=np.ones_like(c["payload"]))
            out = oracle.interpolate(ones, g, 8, metric, wp, oracle.INTERP_IRRADIANCE, r)
            np.testing.assert_allclose(out, 1.0, rtol=0, atol=2e-15)
            const = dict(c, payload=np.tile(np.float32([0.5, 2.0, 7.25]), (c["pos"].shape[0], 1)))
            out = oracle.interpolate(const, g, 8, metric, wp, oracle.INTERP_IRRADIANCE, r)
            np.testing.assert_allclose(out, np.tile([0.5, 2.0, 7.25], (out.shape[0], 1)), rtol=2e-15)


def test_k1_returns_nearest_cache():
    g, c = _small_scene()
    out, idx, _ = oracle.interpolate(c, g, 1, oracle.METRIC_WORLD, oracle.WP_INVERSE,
                                     oracle.INTERP_IRRADIANCE, 0.3, want_neighbors=True)
    np.testing.assert_allclose(out, c["payload"][idx[:, 0]].astype(np.float64), rtol=1e-15)


def _idw(D, p, idx, payload, r, delta_rel, scale):
    """Shepard inverse-distance weighting of the chosen caches, weights
    scale_j / (d_j + delta)."""
    d = np.sqrt(D[p, idx])
    w = scale / (d + delta_rel * r)
    return (w[:, None] * payload[idx].astype(np.float64)).sum(0) / w.sum()


def test_aligned_and_opposed_normals_reduce_to_inverse_distance():
    """With cache normals equal to (w_n = 1) or opposite to (w_n = 0) the
    pixel normal and eps = 0, the weights are 2 w_p or w_p: inverse-distance
    weighting with a factor 2 on aligned caches.  A flipped normal weight
    (1 - max(0, cos)) would swap the factors."""
    g, c = _small_scene()
    P = g["width"] * g["height"]
    n = c["pos"].shape[0]
    g = dict(g, nrm=np.tile(np.float32([0, 0, 1]), (P, 1)))
    sign = np.where(np.arange(n) % 3 == 0, -1.0, 1.0).astype(np.float32)
    c = dict(c, nrm=np.float32([0, 0, 1])[None, :] * sign[:, None])
    r, dr, k = 4.0, 1e-3, 6
    out, idx, _ = oracle.interpolate(c, g, k, oracle.METRIC_IMAGE, oracle.WP_INVERSE,
                                     oracle.INTERP_IRRADIANCE, r, eps=0.0, delta_rel=dr,
                                     want_neighbors=True)
    px, py = np.arange(P) % g["width"], np.arange(P) // g["width"]
    D = ((px[:, None] - c["pix"][None, :, 0]) ** 2 + (py[:, None] - c["pix"][None, :, 1]) ** 2).astype(np.float64)
    for p in range(P):
        scale = np.where(sign[idx[p]] > 0, 2.0, 1.0)
        np.testing.assert_allclose(out[p], _idw(D, p, idx[p], c["payload"], r, dr, scale), rtol=1e-13)


def test_linear_weights_beyond_radius_give_plain_average():
    """LINEAR w_p vanishes beyond r, so with every neighbour farther than r
    only eps is left and the blend is the plain mean of the k payloads."""
    g, c = _small_scene()
    k = 5
    out, idx, _ = oracle.interpolate(c, g, k, oracle.METRIC_IMAGE, oracle.WP_LINEAR,
                                     oracle.INTERP_IRRADIANCE, 1e-3, want_neighbors=True)
    at_cache = set((c["pix"][:, 1] * g["width"] + c["pix"][:, 0]).tolist())
    for p in range(out.shape[0]):
        if p in at_cache:
            continue
        np.testing.assert_allclose(out[p], c["payload"][idx[p]].astype(np.float64).mean(0), rtol=1e-13)


def test_inverse_weight_concentrates_at_own_pixel():
    """At a cache's own pixel d = 0 and w >= w_p = 1/delta_rel, while each of
    the other k-1 caches (d >= 1 pixel) has w <= 2 r/d + eps: the blend sits
    within (k-1)(2r + eps) delta_rel * max|payload| of the cache's own value."""
    g, c = _small_scene()
    k, r, dr = 8, 4.0, 1e-6
    out = oracle.interpolate(c, g, k, oracle.METRIC_IMAGE, oracle.WP_INVERSE,
                             oracle.INTERP_IRRADIANCE, r, delta_rel=dr)
    bound = (k - 1) * (2 * r + 1e-6) * dr * 2.0
    for j in range(c["pos"].shape[0]):
        p = c["pix"][j, 1] * g["width"] + c["pix"][j, 0]
        np.testing.assert_allclose(out[p], c["payload"][j], rtol=0, atol=bound)


def test_lookup_handworked():
    gold = json.load(open(os.path.join(GOLD, "lookup_handworked.json")))
    H, W = gold["H"], gold["W"]
    i, j = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    R = np.stack([i + 10 * j + 100 * c for c in range(3)]).astype(np.float32)[None]
    for case in gold["cases"]:
        caches = {"pos": np.zeros((1, 3), np.float32), "nrm": np.float32([case["normal"]]),
                  "pix": np.zeros((1, 2), np.int32), "maps": R, "payload": None}
        gb = {"width": 1, "height": 1, "pos": np.zeros((1, 3), np.float32),
              "nrm": np.float32([case["normal"]]), "dir": np.float32([case["dir"]])}
        out = oracle.interpolate(caches, gb, 1, oracle.METRIC_WORLD, oracle.WP_INVERSE,
                                 oracle.INTERP_LOOKUP, 1.0)
        np.testing.assert_allclose(out[0], case["out"], rtol=0, atol=1e-5)


def test_lookup_constant_map_and_horizon():
    """A constant map returns its value for every direction above a cache's
    horizon and nothing below it; with one cache the blend is that value."""
    rng = np.random.default_rng(5)
    n = 40
    nrm = rng.normal(size=(n, 3)).astype(np.float32)
    dirs = rng.normal(size=(n, 3)).astype(np.float32)
    maps = np.full((1, 3, 8, 8), 2.5, np.float32)
    for q in range(n):
        caches = {"pos": np.zeros((1, 3), np.float32), "nrm": nrm[q:q + 1],
                  "pix": np.zeros((1, 2), np.int32), "maps": maps}
        gb = {"width": 1, "height": 1, "pos": np.zeros((1, 3), np.float32),
              "nrm": nrm[q:q + 1], "dir": dirs[q:q + 1]}
        out = oracle.interpolate(caches, gb, 1, oracle.METRIC_WORLD, oracle.WP_INVERSE,
                                 oracle.INTERP_LOOKUP, 1.0)
        above = float(np.dot(nrm[q].astype(np.float64), dirs[q].astype(np.float64))) > 0
        np.testing.assert_allclose(out[0], 2.5 if above else 0.0, rtol=1e-14)


def test_lookup_row_linear_map_pins_polar_angle():
    """A map linear in the row index, R[i, j] = i, is reproduced exactly by
    bilinear interpolation away from the clamped edge rows, so the lookup
    returns theta/(pi/2) H - 0.5 with theta the angle between the direction
    and the cache normal -- whatever the frame's azimuth."""
    rng = np.random.default_rng(6)
    H, W = 16, 8
    R = np.broadcast_to(np.arange(H, dtype=np.float32)[:, None], (H, W))
    maps = np.broadcast_to(R, (1, 3, H, W)).copy()
    for _ in range(60):
        nrm = rng.normal(size=3)
        nrm /= np.linalg.norm(nrm)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        nf, df = nrm.astype(np.float32), d.astype(np.float32)
        theta = np.arccos(np.clip(np.dot(nf.astype(np.float64) / np.linalg.norm(nf.astype(np.float64)),
                                         df.astype(np.float64) / np.linalg.norm(df.astype(np.float64))), -1, 1))
        ti = theta / (np.pi / 2) * H - 0.5
        if not (0.0 <= ti <= H - 1):
            continue
        caches = {"pos": np.zeros((1, 3), np.float32), "nrm": nf[None], "pix": np.zeros((1, 2), np.int32),
                  "maps": maps}
        gb = {"width": 1, "height": 1, "pos": np.zeros((1, 3), np.float32), "nrm": nf[None], "dir": df[None]}
        out = oracle.interpolate(caches, gb, 1, oracle.METRIC_WORLD, oracle.WP_INVERSE,
                                 oracle.INTERP_LOOKUP, 1.0)
        np.testing.assert_allclose(out[0], ti, rtol=0, atol=1e-9)


def _two_cache_row(width=8):
    """A one-row image with two caches at pixels x = 2 and x = 6 (IMAGE
    metric), all normals +Z, payloads a = (1, 2, 4) and b = (8, 16, 32)."""
    gb = {"width": width, "height": 1, "pos": np.zeros((width, 3), np.float32),
          "nrm": np.tile(np.float32([0, 0, 1]), (width, 1)), "dir": None}
    caches = {"pos": np.zeros((2, 3), np.float32), "nrm": np.tile(np.float32([0, 0, 1]), (2, 1)),
              "pix": np.int32([[2, 0], [6, 0]]),
              "payload": np.float32([[1, 2, 4], [8, 16, 32]]), "maps": None}
    return gb, caches


def test_linear_weight_inside_radius_handworked():
    """LINEAR w_p = max(0, 1 - d/r) for d < r, worked by hand at r = 4,
    eps = 0: pixel 3 is 1 and 3 pixels from the caches, so w_p = 3/4 and 1/4
    and, with aligned normals (w = 2 w_p), the blend is 3/4 a + 1/4 b.
    Pixel 4 sits half way (1/2, 1/2); pixel 2 is on cache a with b at
    d = r (w_p = 1 and 0); pixel 7 is 5 and 1 away (0 and 3/4).
    1 - d^2/r^2 would give 15/16 and 7/16 at pixel 3, and 1/(d + delta)
    would give 1/(1+delta) and 1/(3+delta): neither matches."""
    gb, caches = _two_cache_row()
    a, b = np.float64([1, 2, 4]), np.float64([8, 16, 32])
    expect = {0: a, 1: a, 2: a, 3: 0.75 * a + 0.25 * b, 4: 0.5 * a + 0.5 * b,
              5: 0.25 * a + 0.75 * b, 6: b, 7: b}
    out = oracle.interpolate(caches, gb, 2, oracle.METRIC_IMAGE, oracle.WP_LINEAR,
                             oracle.INTERP_IRRADIANCE, 4.0, eps=0.0)
    for x, e in expect.items():
        np.testing.assert_allclose(out[x], e, rtol=1e-15, atol=0)
    # the normal term on a LINEAR weight: cache b facing away (w_n = 0) keeps
    # w = w_p, cache a aligned keeps w = 2 w_p; at pixel 3: (1.5 a + 0.25 b) / 1.75
    caches["nrm"] = np.float32([[0, 0, 1], [0, 0, -1]])
    out = oracle.interpolate(caches, gb, 2, oracle.METRIC_IMAGE, oracle.WP_LINEAR,
                             oracle.INTERP_IRRADIANCE, 4.0, eps=0.0)
    np.testing.assert_allclose(out[3], (1.5 * a + 0.25 * b) / 1.75, rtol=1e-15, atol=0)
    np.testing.assert_allclose(out[5], (0.5 * a + 0.75 * b) / 1.25, rtol=1e-15, atol=0)


def test_inverse_weight_radius_factor_with_eps_handworked():
    """INVERSE w_p = r/(d + delta_rel r): at r = 4, delta_rel = 1/4 (delta = 1)
    pixel 3 has d = 1 and 3, so w_p = 4/2 = 2 and 4/4 = 1; aligned normals and
    eps = 1 give w = 2 w_p + eps = 5 and 3, so the blend is (5 a + 3 b)/8.
    Without the factor r (w_p = 1/2, 1/4) it would be (2 a + 1.5 b)/3.5, and
    with delta = delta_rel rather than delta_rel r it would differ again, so
    eps > 0 makes the r factor visible."""
    gb, caches = _two_cache_row()
    a, b = np.float64([1, 2, 4]), np.float64([8, 16, 32])
    out = oracle.interpolate(caches, gb, 2, oracle.METRIC_IMAGE, oracle.WP_INVERSE,
                             oracle.INTERP_IRRADIANCE, 4.0, eps=1.0, delta_rel=0.25)
    np.testing.assert_allclose(out[3], (5 * a + 3 * b) / 8, rtol=1e-15, atol=0)
    # pixel 4: d = 2, 2 -> equal weights; pixel 2: d = 0, 4 -> w_p = 4, 4/5,
    # w = 9 and 2.6
    np.testing.assert_allclose(out[4], 0.5 * (a + b), rtol=1e-15, atol=0)
    np.testing.assert_allclose(out[2], (9 * a + 2.6 * b) / 11.6, rtol=1e-14, atol=0)
