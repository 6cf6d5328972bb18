"""Pins of the oracle's input-map generation (a next step: the maps traced
from cache points in an analytic interior -- radiance with the direct light
left out, distance, normal; Sec. 3.2-3.3)."""
import math

import numpy as np
import pytest

import oracle

WHITE = np.full((6, 3), 0.5)


def test_distances_and_normals_from_the_box_centre():
    """From the centre looking up (+z), a ray at polar angle theta <= 45
    degrees meets the ceiling: distance 0.5 / cos(theta), normal (0, 0, -1),
    in every column whatever the azimuth frame."""
    H = W = 16
    m = oracle.gen_maps([[0.5, 0.5, 0.5]], [[0.0, 0.0, 1.0]], H, W, WHITE, D=0)[0]
    for a in range(H):
        th = (a + 0.5) * math.pi / (2 * H)
        if th <= math.pi / 4:
            np.testing.assert_allclose(m[3, a], 0.5 / math.cos(th), rtol=1e-12)
            np.testing.assert_array_equal(m[4:7, a].T, np.tile([0.0, 0.0, -1.0], (W, 1)))
    # every hit lies on a wall and every normal is a unit axis vector pointing inward
    n = m[4:7].reshape(3, -1).T
    assert np.all(np.abs(n).sum(axis=1) == 1.0)
    assert np.all((m[3] >= 0.5 - 1e-12) & (m[3] <= 0.5 * math.sqrt(3) + 1e-12))


def test_sphere_distance():
    """A sphere of radius r on the axis of the cache normal at distance d:
    a ray at polar angle theta meets it at d cos(theta) - sqrt(r^2 - d^2
    sin^2(theta)), with the outward normal facing back toward the cache."""
    H = W = 32
    sph = [[0.5, 0.5, 0.75, 0.2, 0.3, 0.3, 0.3]]  # cache point and centre exact in float32
    m = oracle.gen_maps([[0.5, 0.5, 0.25]], [[0.0, 0.0, 1.0]], H, W, WHITE, spheres=sph, D=0)[0]
    d, r = 0.5, 0.2
    for a in range(3):
        th = (a + 0.5) * math.pi / (2 * H)
        np.testing.assert_allclose(m[3, a], d * math.cos(th) - math.sqrt(r * r - d * d * math.sin(th) ** 2),
                                   rtol=1e-12)
        assert np.all(m[6, a] < 0.0)
        np.testing.assert_allclose(np.linalg.norm(m[4:7, a], axis=0), 1.0, rtol=1e-12)


def test_furnace():
    """Every wall emits Le and reflects with albedo rho: whatever the random
    directions, a path of D bounces brings rho Le + rho^2 Le + ... + rho^D Le
    (the first hit's own emission is left out)."""
    rng = np.random.default_rng(0)
    le = np.array([1.0, 0.5, 0.25])
    rho = np.array([0.5, 0.3, 0.7])
    pos = rng.uniform(0.1, 0.9, size=(3, 3))
    nrm = rng.standard_normal((3, 3))
    H, W, D = 6, 8, 4
    u = rng.uniform(size=(3, H, W, D, 2))
    m = oracle.gen_maps(pos, nrm, H, W, np.tile(rho, (6, 1)), np.tile(le, (6, 1)), D=D, u=u)
    expect = sum(rho ** i * le for i in range(1, D + 1))
    np.testing.assert_allclose(np.moveaxis(m[:, :3], 1, -1), np.broadcast_to(expect, (3, H, W, 3)), rtol=1e-12)


def test_direct_light_left_out():
    """Black walls and a bright ceiling light in view: the radiance channels
    are zero (the light is seen directly, and nothing reflects it)."""
    light = [0.2, 0.8, 0.2, 0.8, 10.0, 10.0, 10.0]
    m = oracle.gen_maps([[0.5, 0.5, 0.3]], [[0.0, 0.0, 1.0]], 8, 8, np.zeros((6, 3)), light=light, D=3,
                        u=np.random.default_rng(1).uniform(size=(1, 8, 8, 3, 2)))
    assert np.all(m[0, :3] == 0.0) and np.all(m[0, 3] > 0.0)


def _corner_form_factor(A, B):
    """Point-to-rectangle form factor for a point above one corner of a
    parallel A x B rectangle at unit height (the standard closed form)."""
    a, b = math.sqrt(1 + A * A), math.sqrt(1 + B * B)
    return (A / a * math.atan(B / a) + B / b * math.atan(A / b)) / (2 * math.pi)


def test_one_bounce_sees_the_floor_by_its_form_factor():
    """Only the floor emits (Le); from near the ceiling's centre the polar
    rays hit the ceiling (albedo rho), whose one cosine-sampled bounce brings
    Le when it lands on the floor: the expectation is rho Le F, F the form
    factor from the ceiling centre to the unit floor one unit below (four
    0.5 x 0.5 corner rectangles)."""
    rho, le = 0.6, 2.0
    alb = np.full((6, 3), rho)
    em = np.zeros((6, 3))
    em[4] = le  # -z: the floor
    T, H = 20000, 8
    us = np.random.default_rng(4).uniform(size=(T, H, 1, 1, 2))
    # row 0 (polar angle 5.6 degrees) from 0.05 below the ceiling centre hits
    # the ceiling within 0.005 of its centre
    pos = np.tile([[0.5, 0.5, 0.95]], (T, 1))
    m = oracle.gen_maps(pos, np.tile([[0.0, 0.0, 1.0]], (T, 1)), H, 1, alb, em, D=1, u=us)
    assert np.all(m[:, 6, 0, 0] == -1.0)  # the first hit is the ceiling
    F = 4 * _corner_form_factor(0.5, 0.5)
    vals = m[:, 0, 0, 0]
    mean, se = vals.mean(), vals.std(ddof=1) / math.sqrt(T)
    assert abs(mean - rho * le * F) <= 4 * se + 1e-3 * rho * le * F


def test_argument_errors():
    with pytest.raises(ValueError):
        oracle.gen_maps([[0.5, 0.5, 1.5]], [[0.0, 0.0, 1.0]], 4, 4, WHITE)
    with pytest.raises(ValueError):
        oracle.gen_maps([[0.5, 0.5, 0.5]], [[0.0, 0.0, 0.0]], 4, 4, WHITE)


def test_margin_flags_rays_into_a_box_edge_and_leaves_the_maps_alone():
    """The margin output: asking for it changes no map value.  From the box
    centre with normal +z and W = 4 columns, every column's azimuth is a
    diagonal (pi/4 + j pi/2), so its rays meet two side walls at the same
    distance; for the rows below 54.7 degrees from the horizon (polar angle
    above atan(sqrt 2)) those walls are the nearest surfaces: a tie, margin
    below 1.  The two upper rows meet the ceiling well before either wall."""
    H = W = 4
    light = [0.25, 0.75, 0.25, 0.75, 5.0, 5.0, 5.0]
    u = np.random.default_rng(7).uniform(size=(1, H, W, 2, 2))
    a = oracle.gen_maps([[0.5, 0.5, 0.5]], [[0.0, 0.0, 1.0]], H, W, WHITE, light=light, D=2, u=u)
    b, m = oracle.gen_maps([[0.5, 0.5, 0.5]], [[0.0, 0.0, 1.0]], H, W, WHITE, light=light, D=2, u=u,
                           want_margin=True)
    np.testing.assert_array_equal(a, b)
    _, m0 = oracle.gen_maps([[0.5, 0.5, 0.5]], [[0.0, 0.0, 1.0]], H, W, WHITE, D=0, want_margin=True)
    assert np.all(m0[0, 2:] < 1.0)   # polar angles 56.25 and 78.75 degrees
    assert np.all(m0[0, :2] > 100.0)  # 11.25 and 33.75 degrees: the ceiling first
    assert np.all(m <= m0)            # longer paths only add decisions
