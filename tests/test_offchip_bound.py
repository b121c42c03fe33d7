"""The mathematics the persistent form's off-chip test relies on, checked
against the oracle's exact two-body propagation and projection (CPU).

1. Second-order Taylor prediction p = r + v dt + a dt^2/2 of a two-body
   trajectory misses the true position by at most (4 GM v_q / q^3) |dt|^3 / 6,
   q the perihelion distance and v_q the perihelion speed: |d^3r/dt^3| =
   GM |v/r^3 - 3 r (r.v)/r^5| <= 4 GM |v| / r^3 <= 4 GM v_q / q^3.
2. Within 45 degrees of the tangent point the gnomonic projection moves a
   point by at most sec^2(45 deg) = 2 times the pixel scale per radian of
   angular displacement (radial stretch sec^2, tangential sec).
"""
import math

import numpy as np
import pytest

import oracle as O


def _conic(rng, kind):
    gm = O.gm_sun()
    if kind == "elliptic":
        a = rng.uniform(0.6, 40.0)
        e = rng.uniform(0.0, 0.9)
        p = a * (1 - e * e)
    else:
        e = rng.uniform(1.05, 3.0)
        q = rng.uniform(0.3, 5.0)
        p = q * (1 + e)
    nu = rng.uniform(-2.0, 2.0) if kind == "hyperbolic" else rng.uniform(-math.pi, math.pi)
    if kind == "hyperbolic":                      # stay on the real branch
        nu = np.clip(nu, -0.95 * math.acos(-1 / e), 0.95 * math.acos(-1 / e))
    r = p / (1 + e * math.cos(nu))
    h = math.sqrt(gm * p)
    pos = np.array([r * math.cos(nu), r * math.sin(nu), 0.0])
    vel = np.array([-gm / h * math.sin(nu), gm / h * (e + math.cos(nu)), 0.0])
    # random orientation
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    return Q @ pos, Q @ vel, p, e


def _jerk6(r, v):
    gm = O.gm_sun()
    h = np.cross(r, v)
    p = h @ h / gm
    alpha = 2 / np.linalg.norm(r) - v @ v / gm
    e = math.sqrt(max(0.0, 1 - p * alpha))
    q = p / (1 + e)
    vq = math.sqrt(gm * (2 / q - alpha))
    return 4 * gm * vq / q ** 3 / 6


@pytest.mark.parametrize("kind", ["elliptic", "hyperbolic"])
def test_taylor_remainder_bound(kind):
    rng = np.random.default_rng(11 if kind == "elliptic" else 12)
    gm = O.gm_sun()
    worst = 0.0
    for _ in range(200):
        r, v, _, _ = _conic(rng, kind)
        j6 = _jerk6(r, v)
        a = -gm * r / np.linalg.norm(r) ** 3
        for dt in (0.01, 0.3, 1.0, 5.0, -7.0, 30.0, -90.0):
            rt, _, _, _ = O.kepler(r, v, dt)
            pred = r + v * dt + 0.5 * a * dt * dt
            err = np.linalg.norm(rt - pred)
            bound = j6 * abs(dt) ** 3
            assert err <= bound * (1 + 1e-9) + 1e-13, (kind, dt, err, bound)
            if bound > 1e-10:
                worst = max(worst, err / bound)
    assert worst > 0.05          # the bound is not vacuous on these conics


def test_gnomonic_stretch_within_45_degrees():
    rng = np.random.default_rng(13)
    s_deg = 10.0 / 3600.0                          # 10 arcsec pixels
    cd = np.array([[-s_deg, 0.0], [0.0, s_deg]])
    crval = np.array([rng.uniform(0, 360), rng.uniform(-60, 60)])
    crpix = np.array([0.0, 0.0])
    ppr = (180.0 / math.pi) / s_deg                # px per radian at the tangent point
    a0, d0 = np.radians(crval)
    axis = np.array([math.cos(d0) * math.cos(a0), math.cos(d0) * math.sin(a0), math.sin(d0)])
    eps = math.radians(84381.406 / 3600.0)
    # ecliptic vectors whose equatorial direction is the given unit vector
    Rx = np.array([[1, 0, 0], [0, math.cos(eps), math.sin(eps)], [0, -math.sin(eps), math.cos(eps)]])
    worst = 0.0
    for _ in range(400):
        th = math.radians(rng.uniform(0.0, 44.0))
        u = rng.normal(size=3)
        u -= (u @ axis) * axis
        u /= np.linalg.norm(u)
        d1 = math.cos(th) * axis + math.sin(th) * u
        w = rng.normal(size=3)
        w -= (w @ d1) * d1
        w /= np.linalg.norm(w)
        ang = 1e-6
        d2 = math.cos(ang) * d1 + math.sin(ang) * w
        ok1, x1, y1, _, _ = O.project(Rx @ d1 * 2.0, crval, crpix, cd)
        ok2, x2, y2, _, _ = O.project(Rx @ d2 * 2.0, crval, crpix, cd)
        assert ok1 and ok2
        stretch = math.hypot(x2 - x1, y2 - y1) / (ang * ppr)
        worst = max(worst, stretch)
        assert stretch <= 1.0 / math.cos(math.radians(45.0)) ** 2 + 1e-6
    assert worst > 1.5                             # near 45 degrees the bound is nearly reached


def _block_radius(r, v, tf, tm, h, obs_mid, d_obs, gm, inv_c):
    """The persistent form's block cone (block_direction): predicted unit
    direction at tm from the middle observer and its angular radius, in
    FP32 where the kernel computes in FP32."""
    f = np.float32
    r32, v32 = r.astype(f), v.astype(f)
    dt = f(tm - tf)
    r2 = f(r32 @ r32)
    ir = f(1.0) / np.sqrt(r2)
    k = f(-gm) * ir * ir * ir
    rho = (r32 + v32 * dt + f(0.5) * k * r32 * dt * dt - obs_mid.astype(f)).astype(f)
    rr = f(np.sqrt(rho @ rho))
    tau = (rr * f(1.01) + f(1e-3)) * f(inv_c)
    hvec = np.cross(r, v)
    p = hvec @ hvec / gm
    alpha = 2 / np.linalg.norm(r) - v @ v / gm
    e = math.sqrt(max(0.0, 1 - p * alpha))
    q = p / (1 + e)
    vq = math.sqrt(gm * (2 / q - alpha))
    jerk6, half_acc = 4 * gm * vq / q ** 3 / 6, 0.5 * gm / q ** 2
    adt = abs(float(dt)) + h
    err = (jerk6 * adt ** 3 + half_acc * tau ** 2 + 1e-6 * (math.sqrt(r2) + rr) +
           vq * (1e-6 * adt + 1e-4) + vq * (h + tau) + d_obs)
    u = rho / rr
    return u, (1.6 * err / (rr - err) if rr > 2 * err else math.inf)


@pytest.mark.parametrize("kind", ["mba", "neo"])
def test_block_cone_contains_every_sample_direction(kind):
    """Every sample of a block (epochs within h of the middle one, observers
    on the circular 1 AU orbit) lies inside the block cone: the angle between
    the oracle's light-time corrected topocentric direction at t_j from o_j
    and the predicted direction is at most the cone radius."""
    rng = np.random.default_rng(21 if kind == "mba" else 22)
    gm, c = O.gm_sun(), O.c_light()
    worst = 0.0
    for _ in range(120):
        a = rng.uniform(2.1, 3.3) if kind == "mba" else rng.uniform(1.0, 2.0)
        e = rng.uniform(0.0, 0.2) if kind == "mba" else rng.uniform(0.3, 0.6)
        nu = rng.uniform(-math.pi, math.pi)
        p = a * (1 - e * e)
        rad = p / (1 + e * math.cos(nu))
        hh = math.sqrt(gm * p)
        pos = np.array([rad * math.cos(nu), rad * math.sin(nu), 0.0])
        vel = np.array([-gm / hh * math.sin(nu), gm / hh * (e + math.cos(nu)), 0.0])
        inc = math.radians(rng.uniform(0, 15))
        R = np.array([[1, 0, 0], [0, math.cos(inc), -math.sin(inc)], [0, math.sin(inc), math.cos(inc)]])
        r0, v0 = R @ pos, R @ vel
        tf = 0.0
        gap = rng.uniform(0.0, 12.0) * rng.choice([-1, 1])      # last FP64 state to block middle
        h = rng.uniform(0.0, 1.0)
        tm = tf + gap
        ts = np.sort(np.concatenate([[tm - h, tm, tm + h], rng.uniform(tm - h, tm + h, 5)]))
        th0 = rng.uniform(0, 2 * math.pi)
        obs = np.stack([np.cos(th0 + 0.0172 * ts), np.sin(th0 + 0.0172 * ts), np.zeros_like(ts)], 1)
        om = np.array([math.cos(th0 + 0.0172 * tm), math.sin(th0 + 0.0172 * tm), 0.0])
        d_obs = float(np.max(np.linalg.norm(obs - om, axis=1))) * 1.0001 + 1e-7
        u, radius = _block_radius(r0, v0, tf, tm, h, om, d_obs, gm, 1.0 / c)
        if not math.isfinite(radius):
            continue
        for t, o in zip(ts, obs):
            rho, _ = O.apparent(np.concatenate([r0, v0]), tf, t, o)
            d = rho / np.linalg.norm(rho)
            ang = 2 * math.asin(min(1.0, np.linalg.norm(d - u) / 2))
            assert ang <= radius, (kind, gap, h, ang, radius)
            worst = max(worst, ang / radius)
    assert worst > 0.05                        # the radius is not vacuous


def test_chord_angle_bound():
    """2 asin(c / 2) <= 1.05 c for chords c <= 0.5 (the warp cone's radius)."""
    c = np.linspace(1e-9, 0.5, 100001)
    assert np.all(2 * np.arcsin(c / 2) <= 1.05 * c)
