"""The precision split of the stacking kernel, checked on the CPU against
40-digit arithmetic (mpmath): the kernel's formulas are evaluated here with
FP32 intermediates where the kernel uses FP32 (numpy float32, each operation
rounded) and FP64 with exact fused multiply-adds where it uses FP64.

* The two short-step tiers of the f/g series (Bate, Mueller & White 1971,
  sec. 4.5; Danby 1988, sec. 6.9) against the universal-variable solution of
  the two-body step, on NEO, main-belt, Kuiper-belt and hyperbolic conics at
  and below each tier's bound dt^2 K: position, velocity and 1/|r| to FP64
  rounding.
* The light-time model (third-order expansion of r(t - tau), tau to second
  order in v/c and first in the acceleration) against the oracle's iterated
  light time with exact propagation: within 1e-7 px at 0.2 arcsec pixels,
  where the second-order model without the cubic terms misses by more than
  1e-6 px near a close perihelion.

These check the design (formulas and where each precision is used); the GPU
tests check the compiled kernel against the oracle."""
import math

import numpy as np
import pytest

import oracle as O

mp = pytest.importorskip("mpmath")
mp.mp.dps = 40
GM = O.gm_sun()
f32 = np.float32


def _exact_step(r, v, t):
    """Two-body step in 40 digits: universal variable, Newton to 1e-38."""
    r = [mp.mpf(x) for x in r]
    v = [mp.mpf(x) for x in v]
    gm = mp.mpf(GM)
    r0 = mp.sqrt(sum(x * x for x in r))
    alpha = 2 / r0 - sum(x * x for x in v) / gm
    sig0 = sum(a * b for a, b in zip(r, v)) / mp.sqrt(gm)
    sdt = mp.sqrt(gm) * mp.mpf(t)

    def cs(z):
        if abs(z) < mp.mpf("1e-3"):
            c = s = mp.mpf(0)
            tc, ts = mp.mpf(1) / 2, mp.mpf(1) / 6
            for k in range(40):
                c += tc
                s += ts
                tc *= -z / ((2 * k + 3) * (2 * k + 4))
                ts *= -z / ((2 * k + 4) * (2 * k + 5))
            return c, s
        if z > 0:
            q = mp.sqrt(z)
            return (1 - mp.cos(q)) / z, (q - mp.sin(q)) / q ** 3
        q = mp.sqrt(-z)
        return (mp.cosh(q) - 1) / (-z), (mp.sinh(q) - q) / q ** 3

    chi = sdt / r0
    for _ in range(200):
        z = alpha * chi * chi
        c, s = cs(z)
        f = sig0 * chi * chi * c + (1 - alpha * r0) * chi ** 3 * s + r0 * chi - sdt
        df = sig0 * chi * (1 - z * s) + (1 - alpha * r0) * chi * chi * c + r0
        d = f / df
        chi -= d
        if abs(d) < mp.mpf("1e-38") * (1 + abs(chi)):
            break
    z = alpha * chi * chi
    c, s = cs(z)
    fl = 1 - chi * chi * c / r0
    gl = mp.mpf(t) - chi ** 3 * s / mp.sqrt(gm)
    rr = [fl * a + gl * b for a, b in zip(r, v)]
    rn = mp.sqrt(sum(x * x for x in rr))
    fd = mp.sqrt(gm) / (rn * r0) * chi * (z * s - 1)
    gd = 1 - chi * chi * c / rn
    return rr, [fd * a + gd * b for a, b in zip(r, v)]


def _fma(a, b, c):
    return float(mp.mpf(a) * mp.mpf(b) + mp.mpf(c))


def _series(r, v, t, inv_r, alpha):
    """The f/g series step of Delta t^2 K <= 1e-7 as the kernel forms it."""
    ir2 = inv_r * inv_r
    u = GM * ir2 * inv_r
    p = (r[0] * v[0] + r[1] * v[1] + r[2] * v[2]) * ir2
    t2 = t * t
    a = u * (-0.5 * t2)
    tf, uf, pf = f32(t), f32(u), f32(p)
    wf = uf * (f32(1.0) - f32(alpha) * f32(1.0 / inv_r))
    c4 = uf * (f32(3.0) * wf + (f32(-15.0) * pf) * pf + uf)
    upf = uf * pf
    t2f, t3f = tf * tf, tf * tf * tf
    t4f = t2f * t2f
    bf = f32(0.5) * upf * t3f + c4 * f32(1 / 24) * t4f
    gf = -uf * f32(1 / 6) * t3f + f32(0.25) * upf * t4f
    kf = c4 * f32(1 / 6) * t3f
    lf = upf * t3f
    fm1 = a + float(bf)
    g = t + float(gf)
    fdot = _fma(-u, t, _fma(1.5 * (u * p), t2, float(kf)))
    gdm1 = a + float(lf)
    rr = [_fma(fm1, r[i], _fma(g, v[i], r[i])) for i in range(3)]
    vv = [_fma(fdot, r[i], _fma(gdm1, v[i], v[i])) for i in range(3)]
    x = sum(q * q for q in rr)
    y0 = inv_r * _fma(-p, t, 1.0)
    e = _fma(-x, y0 * y0, 1.0)
    ef = f32(e)
    y = _fma(y0, _fma(0.5, e, float(f32(0.375) * ef * ef)), y0)
    return rr, vv, y


def _tiny(r, v, t, inv_r, alpha):
    """The shortest-step series (Delta t^2 K <= 3e-10) as the kernel forms it."""
    ir2 = inv_r * inv_r
    u = GM * ir2 * inv_r
    tf, uf, irf = f32(t), f32(u), f32(inv_r)
    rvf = f32(r[0]) * f32(v[0]) + f32(r[1]) * f32(v[1]) + f32(r[2]) * f32(v[2])
    pf = rvf * irf * irf
    upf = uf * pf
    t2f, t3f = tf * tf, tf * tf * tf
    af = f32(-0.5) * uf * t2f
    wf = uf * (f32(1.0) - f32(alpha) * f32(1.0 / inv_r))
    c4 = uf * (f32(3.0) * wf + (f32(-15.0) * pf) * pf + uf)
    fm1 = float(f32(0.5) * upf * t3f + af)
    g = t + float(-uf * f32(1 / 6) * t3f)
    fdot = _fma(-u, t, float(f32(1.5) * upf * t2f + c4 * f32(1 / 6) * t3f))
    gdm1 = float(upf * t3f + af)
    rr = [_fma(fm1, r[i], _fma(g, v[i], r[i])) for i in range(3)]
    vv = [_fma(fdot, r[i], _fma(gdm1, v[i], v[i])) for i in range(3)]
    x = sum(q * q for q in rr)
    y0 = _fma(inv_r, float(-pf * tf), inv_r)
    e = _fma(-x, y0 * y0, 1.0)
    return rr, vv, _fma(0.5 * y0, e, y0)


def _series_df(r, v, t, inv_r, alpha):
    """The double-float state's series step (Delta t^2 K <= 1e-6, one order
    more than _series) with its double-float parts exact (40 digits: their
    2^-48 rounding is the state's, bounded separately) and its FP32 parts in
    FP32, as the kernel forms them."""
    R = [mp.mpf(x) for x in r]
    V = [mp.mpf(x) for x in v]
    T = mp.mpf(t)
    ir = mp.mpf(inv_r)
    ir2 = ir * ir
    u = mp.mpf(GM) * ir2 * ir
    p = sum(R[i] * V[i] for i in range(3)) * ir2
    a = -u * T * T / 2
    tf, uf, pf = f32(t), f32(float(u)), f32(float(p))
    wf = uf * (f32(1.0) - f32(alpha) * f32(1.0 / inv_r))
    c4 = uf * (f32(3.0) * wf + (f32(-15.0) * pf) * pf + uf)
    upf = uf * pf
    p2 = pf * pf
    t2f = tf * tf
    t3f, t4f = t2f * tf, t2f * t2f
    t5f = t4f * tf
    f5 = f32(15.0) * upf * (f32(7.0) * p2 - f32(3.0) * wf - uf)
    g5 = -uf * (f32(45.0) * p2 - f32(9.0) * wf - uf)
    f6 = -uf * (p2 * (f32(945.0) * p2 - f32(630.0) * wf - f32(210.0) * uf) + wf * (f32(45.0) * wf + f32(24.0) * uf)
                + uf * uf)
    g6 = f32(30.0) * upf * (f32(14.0) * p2 - f32(6.0) * wf - uf)
    bf = f32(0.5) * upf * t3f + c4 * f32(1 / 24) * t4f + f5 * f32(1 / 120) * t5f
    gf = -uf * f32(1 / 6) * t3f + f32(0.25) * upf * t4f + g5 * f32(1 / 120) * t5f
    kf = c4 * f32(1 / 6) * t3f + f5 * f32(1 / 24) * t4f + f6 * f32(1 / 120) * t5f
    lf = upf * t3f + g5 * f32(1 / 24) * t4f + g6 * f32(1 / 120) * t5f
    fm1 = a + mp.mpf(float(bf))
    g = T + mp.mpf(float(gf))
    fdot = 3 * u * p / 2 * T * T + mp.mpf(float(kf)) - u * T
    gdm1 = a + mp.mpf(float(lf))
    rr = [R[i] + fm1 * R[i] + g * V[i] for i in range(3)]
    vv = [V[i] + gdm1 * V[i] + fdot * R[i] for i in range(3)]
    x = sum(q * q for q in rr)
    y0 = ir - ir * (p * T)
    e = 1 - x * y0 * y0
    y = y0 + y0 * (e / 2 + mp.mpf(float(f32(0.375) * f32(float(e)) * f32(float(e)))))
    return rr, vv, y


def _uv_df(r, v, t, inv_r, alpha):
    """The double-float universal-variable step (|z| <= 1e-2) as the kernel
    forms it: double-float quantities exact (40 digits), FP32 parts FP32.
    Returns None where the kernel hands the step to FP64."""
    R = [mp.mpf(x) for x in r]
    V = [mp.mpf(x) for x in v]
    T = mp.mpf(t)
    ir = mp.mpf(inv_r)
    sgm = mp.sqrt(mp.mpf(GM))
    r0 = sum(x * x for x in R) * ir
    sig0 = sum(R[i] * V[i] for i in range(3)) / sgm
    al = mp.mpf(alpha)
    a1 = 1 - al * r0
    sdt = sgm * T
    irf, alf = f32(inv_r), f32(alpha)
    uf, sif = f32(float(sdt)) * irf, f32(float(sig0)) * irf
    chif = uf * (uf * ((-uf * f32(1 / 6)) * (f32(-3.0) * sif * sif + (irf - alf)) + f32(-0.5) * sif) + f32(1.0))
    if not abs(alf) * chif * chif <= f32(3e-2):
        return None
    chi = mp.mpf(float(chif))
    for _ in range(4):
        chi2 = chi * chi
        z = al * chi2
        zf = f32(float(z))
        if not abs(zf) <= f32(5e-2):
            return None
        z3 = zf * zf * zf
        tc = z3 * (zf * (-zf * f32(1 / 479001600) + f32(1 / 3628800)) + f32(-1 / 40320))
        ts = z3 * (zf * (-zf * f32(1 / 6227020800) + f32(1 / 39916800)) + f32(-1 / 362880))
        C = z * (-mp.mpf(1) / 24 + z / 720) + mp.mpf(float(tc)) + mp.mpf(1) / 2
        S = z * (-mp.mpf(1) / 120 + z / 5040) + mp.mpf(float(ts)) + mp.mpf(1) / 6
        chi2c, chi3s = chi2 * C, chi2 * chi * S
        chi1mzs = chi * (1 - z * S)
        omzcf = f32(1.0) - zf * f32(float(C))
        F = sig0 * chi2c + a1 * chi3s + r0 * chi - sdt
        dF = sig0 * chi1mzs + a1 * chi2c + r0
        d2f = f32(float(sig0)) * omzcf + f32(float(a1)) * f32(float(chi1mzs))
        ff, dff = f32(float(F)), f32(float(dF))
        disc = abs(f32(16.0) * dff * dff - f32(20.0) * ff * d2f)
        delta = f32(5.0) * ff / (dff + np.sqrt(disc))
        if abs(delta) <= f32(1e-7):
            d = mp.mpf(float(delta))
            chi2c_c = chi2c - chi1mzs * d
            fm1 = -chi2c_c * ir
            g = T - (chi3s - chi2c * d) / sgm
            rc = dF + mp.mpf(float(-delta * d2f))
            inv_rc = 1 / rc
            fdot = -sgm * (chi1mzs + mp.mpf(float(-delta * omzcf))) * inv_rc * ir
            gdm1 = -chi2c_c * inv_rc
            rr = [R[i] + fm1 * R[i] + g * V[i] for i in range(3)]
            vv = [V[i] + gdm1 * V[i] + fdot * R[i] for i in range(3)]
            return rr, vv, inv_rc
        chi -= mp.mpf(float(delta))
    return None


def test_double_float_universal_variable_step():
    """The double-float universal-variable step on NEO, main-belt and Kuiper-
    belt conics, steps from the end of the series' range (dt^2 K = 1e-6) to
    |z| near 3e-2: position to 2e-15 and velocity to 5e-15 relative (the
    first-order correction at chi - delta leaves (delta^2/2) |f''| r0 with
    delta <= 1e-7), and every step accepted for |z| <= 2.5e-2."""
    rng = np.random.default_rng(29)
    worst = dict(pos=0.0, vel=0.0, inv_r=0.0)
    n = 0
    for kind in ("neo", "mba", "tno"):
        for _ in range(8):
            r, v = _conic(rng, kind)
            k, alpha = _bound_k(r, v)
            rn = float(np.linalg.norm(r))
            t_lo = math.sqrt(1e-6 / k)
            t_hi = 0.18 * rn ** 1.5 / math.sqrt(GM) / math.sqrt(max(abs(alpha) * rn, 1e-3))
            for t in (t_lo * 1.01, math.sqrt(t_lo * t_hi), t_hi):
                t *= rng.choice([-1.0, 1.0])
                inv_r = float(1 / mp.sqrt(sum(mp.mpf(x) ** 2 for x in r)))
                got = _uv_df(list(r), list(v), t, inv_r, alpha)
                z_est = abs(alpha) * (math.sqrt(GM) * t / rn) ** 2
                if got is None:
                    assert z_est > 2.5e-2, (kind, t, z_est)
                    continue
                n += 1
                rr, vv, y = got
                re, ve = _exact_step(r, v, t)
                rabs = float(mp.sqrt(sum(x * x for x in re)))
                vabs = float(mp.sqrt(sum(x * x for x in ve)))
                worst["pos"] = max(worst["pos"], max(abs(float(rr[i] - re[i])) for i in range(3)) / rabs)
                worst["vel"] = max(worst["vel"], max(abs(float(vv[i] - ve[i])) for i in range(3)) / vabs)
                rnew = mp.sqrt(sum(mp.mpf(x) ** 2 for x in re))
                worst["inv_r"] = max(worst["inv_r"], abs(float(y * rnew - 1)))
    print("uv_df", n, {k: f"{w:.2e}" for k, w in worst.items()})
    assert n >= 40
    assert worst["pos"] <= 2e-15 and worst["vel"] <= 5e-15 and worst["inv_r"] <= 1e-15


def _conic(rng, kind):
    rmag, ecc = {"neo": (rng.uniform(0.7, 1.5), rng.uniform(0.2, 0.9)),
                 "mba": (rng.uniform(2.0, 3.5), rng.uniform(0.0, 0.3)),
                 "tno": (rng.uniform(30, 60), rng.uniform(0.0, 0.3)),
                 "hyp": (rng.uniform(0.5, 5), rng.uniform(0.95, 3.0))}[kind]
    vmag = math.sqrt(GM / rmag) * math.sqrt(1 + ecc) * rng.uniform(0.8, 1.2)
    rd, vd = rng.normal(size=3), rng.normal(size=3)
    return rd / np.linalg.norm(rd) * rmag, vd / np.linalg.norm(vd) * vmag


def _bound_k(r, v):
    """K = GM/q^3 + v_q^2/q^2 (q perihelion distance, v_q the speed there)."""
    rn = np.linalg.norm(r)
    alpha = 2 / rn - v @ v / GM
    h = np.cross(r, v)
    semi = h @ h / GM
    q = semi / (1 + math.sqrt(max(0.0, 1 - semi * alpha)))
    return GM / q ** 3 + GM * (2 / q - alpha) / q ** 2, alpha


# velocity bounds: the series tier's own truncation at its bound is ~5e-16;
# the shortest tier is at rounding (without its c4 t^3/6 term in fdot,
# whose one-sided error would drift the velocity, it reaches ~4.4e-16)
@pytest.mark.parametrize("tier,bound,step,vel_tol", [("series", 1e-7, _series, 8e-16),
                                                     ("tiny", 3e-10, _tiny, 3e-16),
                                                     ("series_df", 1e-6, _series_df, 1e-16)])
def test_short_step_tiers_at_fp64_rounding(tier, bound, step, vel_tol):
    rng = np.random.default_rng({"series": 17, "tiny": 5, "series_df": 23}[tier])
    worst = dict(pos=0.0, vel=0.0, inv_r=0.0)
    for kind in ("neo", "mba", "tno", "hyp"):
        for frac in (1.0, 0.3):
            for _ in range(6):
                r, v = _conic(rng, kind)
                k, alpha = _bound_k(r, v)
                t = math.sqrt(bound / k) * frac * rng.choice([-1.0, 1.0])
                re, ve = _exact_step(r, v, t)
                inv_r = float(1 / mp.sqrt(sum(mp.mpf(x) ** 2 for x in r)))
                rr, vv, y = step(list(r), list(v), t, inv_r, alpha)
                rabs = float(mp.sqrt(sum(x * x for x in re)))
                vabs = float(mp.sqrt(sum(x * x for x in ve)))
                worst["pos"] = max(worst["pos"], max(abs(float(rr[i] - re[i])) for i in range(3)) / rabs)
                worst["vel"] = max(worst["vel"], max(abs(float(vv[i] - ve[i])) for i in range(3)) / vabs)
                rn = mp.sqrt(sum(mp.mpf(x) ** 2 for x in rr))
                worst["inv_r"] = max(worst["inv_r"], abs(float(mp.mpf(y) * rn - 1)))
    print(tier, {k: f"{w:.2e}" for k, w in worst.items()})
    assert worst["pos"] <= 4e-16 and worst["inv_r"] <= 4e-16
    assert worst["vel"] <= vel_tol


def _light_time_model(r, v, obs, cubic=True):
    """rho of the kernel's light-time model, in 40 digits."""
    R = [mp.mpf(x) for x in r]
    V = [mp.mpf(x) for x in v]
    D = [R[i] - mp.mpf(obs[i]) for i in range(3)]
    c = mp.mpf(O.c_light())
    dn = mp.sqrt(sum(x * x for x in D))
    dv = sum(D[i] * V[i] for i in range(3))
    v2 = sum(x * x for x in V)
    rn = mp.sqrt(sum(x * x for x in R))
    u = mp.mpf(GM) / rn ** 3
    dr = sum(D[i] * R[i] for i in range(3))
    tau = dn / c - dv / c ** 2 + (dn * v2 + dv ** 2 / dn - (u * dn * dr if cubic else 0)) / (2 * c ** 3)
    p = sum(R[i] * V[i] for i in range(3)) / rn ** 2
    rho = [D[i] - tau * V[i] - u / 2 * tau ** 2 * R[i] for i in range(3)]
    if cubic:
        rho = [rho[i] + tau ** 3 * u / 6 * (V[i] - 3 * p * R[i]) for i in range(3)]
    return rho, dn


def test_light_time_model_against_the_oracle():
    from paper_2503_08854_gb300 import synth
    from _orbits import mixed_population
    rng = np.random.default_rng(11)
    states = mixed_population(rng, 24)
    t0 = 60215.0
    mjd = np.array([60200.1, 60210.3, 60229.5])
    obs = synth.observer_position(mjd, t0, 0.3)
    px_rad = 0.2 / 3600 * math.pi / 180
    worst, worst_quadratic = 0.0, 0.0
    for st in states:
        for j in range(len(mjd)):
            r, v, _, _ = O.kepler(st[:3], st[3:], mjd[j] - t0)
            rho_o, _ = O.apparent(st, t0, mjd[j], obs[j])
            for cubic in (True, False):
                rho, dn = _light_time_model(r, v, obs[j], cubic)
                px = max(abs(float(rho[i]) - rho_o[i]) for i in range(3)) / float(dn) / px_rad
                if cubic:
                    worst = max(worst, px)
                else:
                    worst_quadratic = max(worst_quadratic, px)
    print(f"light-time model: {worst:.2e} px; without the cubic terms {worst_quadratic:.2e} px")
    assert worst <= 1e-7
    assert worst_quadratic > 1e-6       # the cubic terms are needed at 0.2 arcsec pixels
