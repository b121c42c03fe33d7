"""Pins of the oracle's light-time and sky projection (paper sec. 3: the
object's location at the time of every image, transformed to pixels by the
WCS TAN projection of the image header, Calabretta & Greisen 2002)."""
import math

import numpy as np
import pytest

import oracle as O

EPS = O.obliquity()
C = O.c_light()


def _ecl_from_radec(ra_deg, dec_deg):
    """Unit vector of (RA, Dec) in ecliptic coordinates (inverse of a rotation about x by eps)."""
    a, d = math.radians(ra_deg), math.radians(dec_deg)
    q = np.array([math.cos(d) * math.cos(a), math.cos(d) * math.sin(a), math.sin(d)])
    ce, se = math.cos(EPS), math.sin(EPS)
    return np.array([q[0], ce * q[1] + se * q[2], -se * q[1] + ce * q[2]])


def _inverse_gnomonic(x, y, crval, crpix, cd):
    """Pixel -> (RA, Dec) by the inverse gnomonic projection (Snyder 1987,
    Map Projections - A Working Manual, eqs. 20-14 and 22-16)."""
    xi, eta = np.asarray(cd).reshape(2, 2) @ np.array([x - crpix[0], y - crpix[1]])
    xi, eta = math.radians(xi), math.radians(eta)
    a0, d0 = math.radians(crval[0]), math.radians(crval[1])
    rho = math.hypot(xi, eta)
    if rho == 0:
        return crval[0], crval[1]
    c = math.atan(rho)
    dec = math.asin(math.cos(c) * math.sin(d0) + eta * math.sin(c) * math.cos(d0) / rho)
    ra = a0 + math.atan2(xi * math.sin(c), rho * math.cos(d0) * math.cos(c) - eta * math.sin(d0) * math.sin(c))
    return math.degrees(ra), math.degrees(dec)


def test_ecliptic_to_equatorial_rotation():
    cd = [[-1e-4, 0], [0, 1e-4]]
    for vec, ra, dec in [((1, 0, 0), 0.0, 0.0),
                         ((0, 1, 0), 90.0, math.degrees(EPS)),
                         ((0, 0, 1), 270.0, 90.0 - math.degrees(EPS))]:
        ok, x, y, r, d = O.project(np.array(vec, float), [ra, dec], [0, 0], cd)
        assert ok
        assert abs(math.degrees(r) % 360.0 - ra) < 1e-12
        assert abs(math.degrees(d) - dec) < 1e-12
        assert abs(x) < 1e-9 and abs(y) < 1e-9


def test_crval_maps_to_crpix():
    rng = np.random.default_rng(1)
    for _ in range(50):
        crval = [rng.uniform(0, 360), rng.uniform(-89, 89)]
        crpix = rng.uniform(0, 4000, 2)
        th = rng.uniform(0, 2 * math.pi)
        cd = 1e-4 * np.array([[-math.cos(th), math.sin(th)], [math.sin(th), math.cos(th)]])
        u = _ecl_from_radec(*crval) * rng.uniform(0.1, 50)
        ok, x, y, _, _ = O.project(u, crval, crpix, cd)
        assert ok and abs(x - crpix[0]) < 1e-9 and abs(y - crpix[1]) < 1e-9


def test_inverse_gnomonic_round_trip():
    rng = np.random.default_rng(2)
    for _ in range(200):
        crval = [rng.uniform(0, 360), rng.uniform(-85, 85)]
        crpix = rng.uniform(0, 4000, 2)
        s = rng.uniform(0.1, 30) / 3600
        th = rng.uniform(0, 2 * math.pi)
        cd = s * np.array([[-math.cos(th), math.sin(th)], [math.sin(th), math.cos(th)]])
        cd = cd + rng.normal(size=(2, 2)) * 0.05 * s   # skew
        x, y = rng.uniform(-500, 4500, 2)
        ra, dec = _inverse_gnomonic(x, y, crval, crpix, cd)
        ok, xo, yo, _, _ = O.project(_ecl_from_radec(ra, dec) * 2.7, crval, crpix, cd)
        assert ok
        assert abs(xo - x) < 1e-8 and abs(yo - y) < 1e-8


def test_small_offset_limit():
    crval = [123.0, 41.0]
    d_ra = 1e-6  # deg
    u = _ecl_from_radec(crval[0] + d_ra, crval[1])
    ok, x, y, _, _ = O.project(u, crval, [0, 0], [[1, 0], [0, 1]])
    assert ok
    # 1e-7 relative: the input RA itself carries ~1e-14 deg of rounding
    assert abs(x - d_ra * math.cos(math.radians(41.0))) < 1e-7 * d_ra
    assert abs(y) < 1e-12


def test_points_ninety_degrees_away_are_invalid():
    crval = [10.0, 20.0]
    base = _ecl_from_radec(*crval)
    other = np.cross(base, np.array([0.3, -0.2, 0.9]))
    assert not O.project(other, crval, [0, 0], [[1e-4, 0], [0, 1e-4]])[0]
    assert not O.project(-base, crval, [0, 0], [[1e-4, 0], [0, 1e-4]])[0]


def test_light_time_stationary_object():
    state = np.array([2.0, -1.0, 0.3, 0.0, 0.0, 0.0])
    obs = np.array([0.6, 0.8, 0.0])
    rho, tau = O.apparent(state, 100.0, 130.0, obs, mu=0.0)
    assert tau == pytest.approx(np.linalg.norm(state[:3] - obs) / C, rel=1e-15)
    np.testing.assert_allclose(rho, state[:3] - obs, atol=1e-15)


def test_light_time_linear_motion_closed_form():
    """Force-free motion: |d - v tau| = c tau with d = r0 + v (t - t0) - obs is a
    quadratic in tau; its positive root is the exact light time."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        r0 = rng.normal(size=3) * 3
        v = rng.normal(size=3) * 0.02
        obs = rng.normal(size=3)
        t0, t = 10.0, 10.0 + rng.uniform(-50, 50)
        d = r0 + v * (t - t0) - obs
        A = v.dot(v) - C * C
        B = -2.0 * d.dot(v)
        Cc = d.dot(d)
        tau_exact = (-B - math.sqrt(B * B - 4 * A * Cc)) / (2 * A)
        rho, tau = O.apparent(np.concatenate([r0, v]), t0, t, obs, mu=0.0)
        assert tau == pytest.approx(tau_exact, rel=1e-13)
        assert np.linalg.norm(rho) == pytest.approx(C * tau, rel=1e-14)


def test_light_time_self_consistent_keplerian():
    rng = np.random.default_rng(4)
    for _ in range(50):
        r = rng.uniform(0.8, 45)
        lon = rng.uniform(0, 2 * math.pi)
        state = np.array([r * math.cos(lon), r * math.sin(lon), 0.05 * r,
                          -math.sin(lon) * 0.0172 / math.sqrt(r), math.cos(lon) * 0.0172 / math.sqrt(r), 0.0])
        obs = np.array([math.cos(lon + 0.3), math.sin(lon + 0.3), 0.0])
        rho, tau = O.apparent(state, 60000.0, 60000.0 + rng.uniform(-300, 300), obs)
        assert np.linalg.norm(rho) == pytest.approx(C * tau, rel=1e-14)
