"""Pins of the oracle's two-body propagation (paper sec. 3: elliptical two-body
motion around the Sun) against closed forms, invariants, an independent
textbook solver and a published worked example."""
import math
import os

import numpy as np
import pytest

import oracle as O

MU = O.gm_sun()
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _random_state(rng, kind):
    """Random heliocentric state: 'ell' bound (e < 0.95), 'hyp' unbound."""
    r = rng.uniform(0.5, 40.0)
    rhat = rng.normal(size=3)
    rhat /= np.linalg.norm(rhat)
    vdir = rng.normal(size=3)
    vdir -= vdir.dot(rhat) * rhat * rng.uniform(0.0, 1.0)
    vdir /= np.linalg.norm(vdir)
    vesc = math.sqrt(2 * MU / r)
    speed = vesc * (rng.uniform(0.2, 0.97) if kind == "ell" else rng.uniform(1.05, 2.0))
    return r * rhat, speed * vdir


def _kepler_E_bisect(r0, v0, dt, mu):
    """Independent solver: classical elements, Kepler's equation E - e sin E = M
    (or e sinh H - H = M) solved by bisection, perifocal position and velocity."""
    r0, v0 = np.asarray(r0, float), np.asarray(v0, float)
    rn = np.linalg.norm(r0)
    h = np.cross(r0, v0)
    evec = np.cross(v0, h) / mu - r0 / rn
    e = np.linalg.norm(evec)
    a = 1.0 / (2.0 / rn - v0.dot(v0) / mu)
    P = evec / e
    Q = np.cross(h / np.linalg.norm(h), P)
    if a > 0:
        n = math.sqrt(mu / a ** 3)
        E0 = math.atan2(r0.dot(v0) / (e * math.sqrt(mu * a)), (1 - rn / a) / e)
        M = E0 - e * math.sin(E0) + n * dt
        lo, hi = M - e - 1.0, M + e + 1.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if mid - e * math.sin(mid) < M:
                lo = mid
            else:
                hi = mid
        E = 0.5 * (lo + hi)
        r = a * (math.cos(E) - e) * P + a * math.sqrt(1 - e * e) * math.sin(E) * Q
        rr = a * (1 - e * math.cos(E))
        v = math.sqrt(mu * a) / rr * (-math.sin(E) * P + math.sqrt(1 - e * e) * math.cos(E) * Q)
    else:
        aa = -a
        n = math.sqrt(mu / aa ** 3)
        H0 = math.asinh(r0.dot(v0) / (e * math.sqrt(mu * aa)))
        M = e * math.sinh(H0) - H0 + n * dt
        lo, hi = -50.0, 50.0
        for _ in range(300):
            mid = 0.5 * (lo + hi)
            if e * math.sinh(mid) - mid < M:
                lo = mid
            else:
                hi = mid
        H = 0.5 * (lo + hi)
        r = aa * (e - math.cosh(H)) * P + aa * math.sqrt(e * e - 1) * math.sinh(H) * Q
        rr = aa * (e * math.cosh(H) - 1)
        v = math.sqrt(mu * aa) / rr * (-math.sinh(H) * P + math.sqrt(e * e - 1) * math.cosh(H) * Q)
    return r, v


def test_golden_vallado_kepler_problem():
    vals = {}
    with open(os.path.join(GOLDEN, "vallado_ex2_4_kepler.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            k, *v = line.split()
            vals[k] = np.array([float(x) for x in v])
    r, v, _, _ = O.kepler(vals["r0"], vals["v0"], vals["dt_s"][0], mu=vals["mu"][0])
    np.testing.assert_allclose(r, vals["r"], atol=6e-5)      # 4 printed decimals
    np.testing.assert_allclose(v, vals["v"], atol=6e-7)      # 6 printed decimals


@pytest.mark.parametrize("seed", range(5))
def test_circular_orbit_closed_form(seed):
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.3, 60.0)
    rhat = rng.normal(size=3); rhat /= np.linalg.norm(rhat)
    t = rng.normal(size=3); t -= t.dot(rhat) * rhat; t /= np.linalg.norm(t)
    r0, v0 = r * rhat, math.sqrt(MU / r) * t
    n = math.sqrt(MU / r ** 3)
    for dt in (0.01, 3.7, 120.0, -55.0, 2.3 * 2 * math.pi / n):
        rr, vv, _, _ = O.kepler(r0, v0, dt)
        exp_r = math.cos(n * dt) * r0 + math.sin(n * dt) * v0 / n
        exp_v = -n * math.sin(n * dt) * r0 + math.cos(n * dt) * v0
        np.testing.assert_allclose(rr, exp_r, atol=2e-13 * r * max(1, abs(n * dt)))
        np.testing.assert_allclose(vv, exp_v, atol=2e-13 * np.linalg.norm(v0) * max(1, abs(n * dt)))


def test_linear_limit_tiny_mu():
    rng = np.random.default_rng(7)
    for _ in range(20):
        r0 = rng.normal(size=3) * 3
        v0 = rng.normal(size=3) * 0.01
        dt = rng.uniform(-200, 200)
        rr, vv, fg, _ = O.kepler(r0, v0, dt, mu=1e-30)
        np.testing.assert_allclose(rr, r0 + v0 * dt, rtol=0, atol=1e-12 * (1 + np.abs(r0 + v0 * dt).max()))
        np.testing.assert_allclose(vv, v0, atol=1e-14)


@pytest.mark.parametrize("kind", ["ell", "hyp"])
def test_energy_angular_momentum_wronskian(kind):
    rng = np.random.default_rng(11 if kind == "ell" else 12)
    for _ in range(200):
        r0, v0 = _random_state(rng, kind)
        dt = rng.uniform(-2000, 2000)
        rr, vv, (f, g, fd, gd), _ = O.kepler(r0, v0, dt)
        E0 = 0.5 * v0.dot(v0) - MU / np.linalg.norm(r0)
        E1 = 0.5 * vv.dot(vv) - MU / np.linalg.norm(rr)
        assert abs(E1 - E0) <= 1e-12 * abs(E0) * 10
        h0, h1 = np.cross(r0, v0), np.cross(rr, vv)
        assert np.linalg.norm(h1 - h0) <= 1e-12 * np.linalg.norm(h0) * 10
        assert abs(f * gd - fd * g - 1.0) <= 1e-12


@pytest.mark.parametrize("kind", ["ell", "hyp"])
def test_against_eccentric_anomaly_bisection(kind):
    rng = np.random.default_rng(21 if kind == "ell" else 22)
    for _ in range(100):
        r0, v0 = _random_state(rng, kind)
        dt = rng.uniform(-400, 400)
        rr, vv, _, _ = O.kepler(r0, v0, dt)
        re, ve = _kepler_E_bisect(r0, v0, dt, MU)
        scale = max(np.linalg.norm(r0), np.linalg.norm(re))
        assert np.linalg.norm(rr - re) <= 1e-11 * scale, (rr, re)
        assert np.linalg.norm(vv - ve) <= 1e-11 * np.linalg.norm(ve) * 10


def test_round_trip():
    rng = np.random.default_rng(5)
    for kind in ("ell", "hyp"):
        for _ in range(100):
            r0, v0 = _random_state(rng, kind)
            dt = rng.uniform(-1000, 1000)
            r1, v1, _, _ = O.kepler(r0, v0, dt)
            r2, v2, _, _ = O.kepler(r1, v1, -dt)
            assert np.linalg.norm(r2 - r0) <= 1e-11 * np.linalg.norm(r0)


def test_zero_step_is_identity():
    r0, v0 = np.array([1.3, -0.4, 0.2]), np.array([0.002, 0.013, -0.001])
    rr, vv, fg, _ = O.kepler(r0, v0, 0.0)
    np.testing.assert_allclose(rr, r0, atol=1e-15)
    np.testing.assert_allclose(vv, v0, atol=1e-17)
