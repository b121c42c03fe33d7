"""Seeded synthetic survey inputs shared by the tests, the smoke check and the benchmark.

This module only draws inputs: exposure epochs and pointings, observer
positions, noise images, candidate-orbit states and the states and fluxes of
injected sources.  It never propagates a candidate orbit, never projects a
position into pixels and never evaluates the matched filter: sources are
rendered at pixel positions that the caller supplies (computed by whichever
implementation is under test, or by the oracle in the tests).

The telescope pointing of each exposure follows a crude survey schedule: the
field centre tracks a reference body on a circular orbit in the ecliptic,
seen from the observer without light-time.  That is how a survey picks where
to look, not part of the method, and nothing checks its accuracy.

Units: AU, days, degrees for the WCS.  Frame: heliocentric ecliptic.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GAUSS_K = 0.01720209895                 # AU^1.5 / day (sampling of circular speeds)
KMS_TO_AUD = 86400.0 / 149597870.7      # km/s -> AU/day
OBLIQUITY_DEG = 84381.406 / 3600.0      # for turning a pointing into RA/Dec


@dataclasses.dataclass
class Exposures:
    mjd: np.ndarray      # (n,)     epoch, days
    obs: np.ndarray      # (n, 3)   observer position, AU
    crval: np.ndarray    # (n, 2)   tangent point RA, Dec, deg
    crpix: np.ndarray    # (n, 2)   0-based pixel of the tangent point
    cd: np.ndarray       # (n, 2, 2) deg / px
    sigma: np.ndarray    # (n,)     PSF sigma, px
    var: np.ndarray      # (n,)     constant per-pixel variance
    width: np.ndarray    # (n,) int32
    height: np.ndarray   # (n,) int32

    @property
    def n(self) -> int:
        return len(self.mjd)

    def subset(self, idx) -> "Exposures":
        idx = np.asarray(idx)
        return Exposures(*[np.asarray(getattr(self, f.name))[idx] for f in dataclasses.fields(self)])


@dataclasses.dataclass
class Sky:
    """A synthetic survey: exposures, candidate orbits and injected sources."""
    name: str
    ex: Exposures
    t0: float                     # epoch of every orbit state
    states: np.ndarray            # (n_o, 6) candidate orbits x, y, z, vx, vy, vz
    inj_states: np.ndarray        # (n_inj, 6) injected sources
    inj_flux: np.ndarray          # (n_inj,) flux (counts) of each injected source
    inj_orbit: np.ndarray         # (n_inj,) candidate index equal to each injected source, or -1
    seed: int
    families: tuple | None = None  # (fam_orb_off int64, fam_exp_off int64, fam_exp_idx int32)
    meta: dict = dataclasses.field(default_factory=dict)


def observer_position(t, t_ref, theta_ref):
    """Massless observer on a circular 1 AU orbit in the ecliptic (angular rate k rad/day)."""
    th = theta_ref + GAUSS_K * (np.asarray(t, dtype=np.float64) - t_ref)
    return np.stack([np.cos(th), np.sin(th), np.zeros_like(th)], axis=-1)


def ecliptic_to_radec_deg(vec):
    """Direction of an ecliptic vector as (RA, Dec) in degrees (pointing only)."""
    e = math.radians(OBLIQUITY_DEG)
    x, y, z = vec[..., 0], vec[..., 1], vec[..., 2]
    qy = math.cos(e) * y - math.sin(e) * z
    qz = math.sin(e) * y + math.cos(e) * z
    ra = np.degrees(np.arctan2(qy, x)) % 360.0
    dec = np.degrees(np.arctan2(qz, np.hypot(x, qy)))
    return np.stack([ra, dec], axis=-1)


def circular_reference(t, t_ref, r, lon_ref):
    """Reference body for pointings: circular ecliptic orbit of radius r."""
    th = lon_ref + GAUSS_K / r ** 1.5 * (np.asarray(t, dtype=np.float64) - t_ref)
    return np.stack([r * np.cos(th), r * np.sin(th), np.zeros_like(th)], axis=-1)


def tracking_pointings(mjd, obs, t_ref, r_ref, lon_ref):
    """Field centres that follow a circular reference body (no light-time)."""
    ref = circular_reference(mjd, t_ref, r_ref, lon_ref)
    return ecliptic_to_radec_deg(ref - obs)


def grid_states(r_values, dv_r_kms, dv_t_kms, lon):
    """Orbit grid of the tiny workloads: every node starts on the heliocentric
    ray at longitude ``lon`` (in the ecliptic) at distance r, with the circular
    prograde speed plus (dv_r, dv_t) km/s along the radial and tangential unit
    vectors.  Index o = (i_r * n_vr + i_vr) * n_vt + i_vt."""
    rh = np.array([math.cos(lon), math.sin(lon), 0.0])
    th = np.array([-math.sin(lon), math.cos(lon), 0.0])
    R, VR, VT = np.meshgrid(np.asarray(r_values, dtype=np.float64),
                            np.asarray(dv_r_kms, dtype=np.float64) * KMS_TO_AUD,
                            np.asarray(dv_t_kms, dtype=np.float64) * KMS_TO_AUD, indexing="ij")
    R, VR, VT = R.ravel(), VR.ravel(), VT.ravel()
    vc = GAUSS_K / np.sqrt(R)
    pos = R[:, None] * rh[None, :]
    vel = VR[:, None] * rh[None, :] + (vc + VT)[:, None] * th[None, :]
    return np.concatenate([pos, vel], axis=1)


def half_open_linspace(a, b, n):
    return a + (b - a) * np.arange(n, dtype=np.float64) / n


def flux_for_snr(snr, sigma_px, var):
    """Flux giving a per-image matched-filter SNR of about ``snr`` (continuous
    Gaussian approximation sum P^2 ~ 1 / (4 pi sigma^2))."""
    return np.asarray(snr) * np.sqrt(var) * np.sqrt(4.0 * math.pi) * sigma_px


def render_sources(images, xy, flux, sigma, radius=6.0):
    """Add point sources to ``images`` (n_exp, H, W) in place.  ``xy`` is
    (n_src, n_exp, 2) pixel coordinates (NaN = not visible), ``flux`` (n_src,),
    ``sigma`` (n_exp,) PSF sigma.  Each source is a unit-integral sampled
    Gaussian times its flux, drawn within ``radius`` sigma."""
    n_exp, H, W = images.shape
    for s in range(xy.shape[0]):
        for j in range(n_exp):
            x, y = xy[s, j]
            if not (np.isfinite(x) and np.isfinite(y)):
                continue
            sg = float(sigma[j])
            rad = int(math.ceil(radius * sg))
            x0, x1 = max(int(math.floor(x)) - rad, 0), min(int(math.floor(x)) + rad + 2, W)
            y0, y1 = max(int(math.floor(y)) - rad, 0), min(int(math.floor(y)) + rad + 2, H)
            if x0 >= x1 or y0 >= y1:
                continue
            gx = np.exp(-0.5 * ((np.arange(x0, x1) - x) / sg) ** 2)
            gy = np.exp(-0.5 * ((np.arange(y0, y1) - y) / sg) ** 2)
            images[j, y0:y1, x0:x1] += (flux[s] / (2.0 * math.pi * sg * sg)
                                        * np.outer(gy, gx)).astype(images.dtype)
    return images


# --------------------------------------------------------------------------
# Tiny grid sky (the plain-method workload and its scaled-down test cases)
# --------------------------------------------------------------------------

def grid_sky(*, name="tiny", n_exp=10, nights=20.0, size=512, scale_arcsec=0.2,
             n_r=16, n_v=64, r_range=(2.0, 3.0), v_kms=5.0, sigma_px=1.5, var=1.0,
             inj_snr=2.0, n_inj=5, seed=1, mjd_start=60000.0, lon=0.7) -> Sky:
    """Plain-method grid workload.  Epochs: one per ``nights / n_exp`` nights,
    each jittered by U(-0.1, 0.1) d.  Observer on a circular 1 AU orbit, at
    opposition to the grid's reference body at the epoch t0 (mid-span).
    Pointings track the central node (r = 2.5 AU circular) along the ecliptic.
    Orbit grid: n_r distances x n_v radial x n_v tangential velocity offsets
    (half-open grids, so the circular central node is a grid point).
    Injected sources: ``n_inj`` grid nodes at the central distance with zero
    tangential offset and the smallest radial offsets; those stay in the
    tracked field, so their on-sky tracks stay near the field centre."""
    rng = np.random.default_rng(seed)
    step = nights / n_exp
    mjd = mjd_start + 0.5 + step * np.arange(n_exp) + rng.uniform(-0.1, 0.1, n_exp)
    t0 = float(mjd_start + 0.5 + step * (n_exp - 1) / 2.0)
    obs = observer_position(mjd, t0, lon)
    r_c = 0.5 * (r_range[0] + r_range[1])
    crval = tracking_pointings(mjd, obs, t0, r_c, lon)
    s = scale_arcsec / 3600.0
    ex = Exposures(
        mjd=mjd, obs=obs, crval=crval,
        crpix=np.tile(np.array([size / 2.0, size / 2.0]), (n_exp, 1)),
        cd=np.tile(np.array([[-s, 0.0], [0.0, s]]), (n_exp, 1, 1)),
        sigma=np.full(n_exp, sigma_px), var=np.full(n_exp, var),
        width=np.full(n_exp, size, dtype=np.int32), height=np.full(n_exp, size, dtype=np.int32))
    r_vals = half_open_linspace(r_range[0], r_range[1], n_r)
    dv = half_open_linspace(-v_kms, v_kms, n_v)
    states = grid_states(r_vals, dv, dv, lon)
    i_r = int(np.argmin(np.abs(r_vals - r_c)))
    i_t = int(np.argmin(np.abs(dv)))
    order = np.argsort(np.abs(dv), kind="stable")[:n_inj]
    inj_orbit = np.array([(i_r * n_v + i_v) * n_v + i_t for i_v in order], dtype=np.int64)
    flux = flux_for_snr(np.full(n_inj, inj_snr), sigma_px, var)
    return Sky(name=name, ex=ex, t0=t0, states=states, inj_states=states[inj_orbit].copy(),
               inj_flux=flux, inj_orbit=inj_orbit, seed=seed,
               meta=dict(r_values=r_vals, dv_kms=dv, size=size))


def noise_images(ex: Exposures, seed: int, dtype=np.float32):
    """N(0, var_j) noise, one image per exposure (numpy, seeded)."""
    rng = np.random.default_rng(seed + 1000003)
    out = np.empty((ex.n, int(ex.height[0]), int(ex.width[0])), dtype=dtype)
    for j in range(ex.n):
        out[j] = rng.standard_normal((int(ex.height[j]), int(ex.width[j])), dtype=np.float32) \
            * np.float32(math.sqrt(ex.var[j]))
    return out


# --------------------------------------------------------------------------
# MBA-scale survey (dense coverage, irregular cadence)
# --------------------------------------------------------------------------

def state_from_elements(a, e, inc, node, argp, true_anom, gm=GAUSS_K ** 2):
    """Heliocentric ecliptic state from classical elements with the TRUE anomaly
    (the perifocal conic formula; orbit sampling, no time propagation)."""
    a, e, inc, node, argp, nu = (np.asarray(x, dtype=np.float64) for x in
                                 (a, e, inc, node, argp, true_anom))
    p = a * (1.0 - e * e)
    r = p / (1.0 + e * np.cos(nu))
    pf = np.stack([r * np.cos(nu), r * np.sin(nu), np.zeros_like(nu)], -1)
    vf = np.sqrt(gm / p)[..., None] * np.stack([-np.sin(nu), e + np.cos(nu), np.zeros_like(nu)], -1)
    cO, sO, ci, si, cw, sw = np.cos(node), np.sin(node), np.cos(inc), np.sin(inc), np.cos(argp), np.sin(argp)
    R = np.stack([np.stack([cO * cw - sO * sw * ci, -cO * sw - sO * cw * ci, sO * si], -1),
                  np.stack([sO * cw + cO * sw * ci, -sO * sw + cO * cw * ci, -cO * si], -1),
                  np.stack([sw * si, cw * si, ci], -1)], -2)
    pos = np.einsum("...ij,...j->...i", R, pf)
    vel = np.einsum("...ij,...j->...i", R, vf)
    return np.concatenate([pos, vel], -1)


def irregular_cadence(rng, n_exp, nights, mjd_start, visits=(1, 4), gap_min=15.0, snap_s=90.0):
    """Survey cadence: each night has U{visits} visits at least ``gap_min``
    minutes apart inside a 6 h window; the n_exp exposures are spread over the
    visits as evenly as possible, ``snap_s`` seconds apart within a visit."""
    times = []
    for night in range(int(nights)):
        k = int(rng.integers(visits[0], visits[1] + 1))
        while True:
            t = np.sort(rng.uniform(0.0, 0.25, k))
            if k == 1 or np.min(np.diff(t)) >= gap_min / 1440.0:
                break
        times.extend(mjd_start + night + 0.1 + t)
    times = np.asarray(times)
    per = np.full(len(times), n_exp // len(times))
    per[: n_exp - per.sum()] += 1
    mjd = np.concatenate([t + np.arange(m) * snap_s / 86400.0 for t, m in zip(times, per)])
    return np.sort(mjd)[:n_exp]


def mba_sky(*, n_exp=200, nights=30, size=4096, n_true=1000, fam_size=16384, seed=2,
            mjd_start=60100.0, lon=2.0, lon_half=0.055, scale_arcsec=10.5,
            snr_range=(0.5, 3.0), jitter_r=3e-4, jitter_v=1e-5) -> Sky:
    """MBA-scale workload.  1000 main-belt asteroids (a in [2.1, 3.3] AU,
    e < 0.2, i < 20 deg) near opposition at the mid-span epoch t0, each the
    seed of a family of ``fam_size`` candidate orbits (the true state plus
    seeded state jitter), 16.4 M candidates in all.  Exposures follow an
    irregular 1-4 visit/night cadence over ``nights`` nights; pointings track
    a circular reference body at 2.7 AU; each exposure's chip is offset so
    that it covers a random 60-100 % of the population's extent; PSF sigma
    ~ U(1.2, 2.0) px and variance log-uniform in [0.5, 2] per exposure.
    Candidate orbit o of family f is index f * fam_size + (o % fam_size);
    member 0 of every family is the true state."""
    rng = np.random.default_rng(seed)
    mjd = irregular_cadence(rng, n_exp, nights, mjd_start)
    t0 = float(mjd_start + nights / 2.0)
    obs = observer_position(mjd, t0, lon)
    crval = tracking_pointings(mjd, obs, t0, 2.7, lon)
    s = scale_arcsec / 3600.0
    # population extent along x in pixels (geocentric longitude spread near opposition)
    span_px = 2.0 * math.degrees(lon_half) * 1.9 / s
    cover = rng.uniform(0.6, 1.0, n_exp)
    shift = (1.0 - cover) * span_px * rng.choice([-1.0, 1.0], n_exp)
    crpix = np.stack([size / 2.0 + shift, np.full(n_exp, size / 2.0)], -1)
    sigma = rng.uniform(1.2, 2.0, n_exp).astype(np.float32).astype(np.float64)
    var = np.exp(rng.uniform(math.log(0.5), math.log(2.0), n_exp)).astype(np.float32).astype(np.float64)
    ex = Exposures(mjd=mjd, obs=obs, crval=crval, crpix=crpix,
                   cd=np.tile(np.array([[-s, 0.0], [0.0, s]]), (n_exp, 1, 1)), sigma=sigma, var=var,
                   width=np.full(n_exp, size, np.int32), height=np.full(n_exp, size, np.int32))
    a = rng.uniform(2.1, 3.3, n_true)
    e = rng.uniform(0.0, 0.2, n_true)
    inc = np.radians(rng.uniform(0.0, 20.0, n_true))
    u = rng.uniform(-0.05, 0.05, n_true)                  # argument of latitude: near a node
    u = np.where(rng.random(n_true) < 0.5, u, u + math.pi)
    lam = lon + rng.uniform(-lon_half, lon_half, n_true)  # heliocentric longitude at t0
    node = lam - np.arctan2(np.cos(inc) * np.sin(u), np.cos(u))
    argp = rng.uniform(0.0, 2 * math.pi, n_true)
    true_states = state_from_elements(a, e, inc, node, argp, u - argp)
    states = np.repeat(true_states, fam_size, axis=0)
    jit = np.concatenate([rng.normal(0.0, jitter_r, (len(states), 3)),
                          rng.normal(0.0, jitter_v, (len(states), 3))], 1)
    jit[::fam_size] = 0.0
    states += jit
    snr = rng.uniform(*snr_range, n_true)
    flux = flux_for_snr(snr, 1.6, 1.0)
    return Sky(name="mba", ex=ex, t0=t0, states=states, inj_states=true_states, inj_flux=flux,
               inj_orbit=np.arange(n_true, dtype=np.int64) * fam_size, seed=seed,
               meta=dict(fam_size=fam_size, n_true=n_true, cover=cover, inj_snr=snr, size=size))


def noise_images_torch(ex: Exposures, seed: int, device):
    """N(0, var_j) noise images drawn on a torch device (seeded generator)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) + 1000003)
    out = torch.empty((ex.n, int(ex.height[0]), int(ex.width[0])), dtype=torch.float32, device=device)
    for j in range(ex.n):
        out[j].normal_(0.0, math.sqrt(float(ex.var[j])), generator=g)
    return out


def render_sources_torch(images, xy, flux, sigma, radius=6.0):
    """``render_sources`` for a torch image stack: xy (n_src, n_exp, 2) tensor."""
    import torch
    n_exp, H, W = images.shape
    dev = images.device
    rad = int(math.ceil(radius * float(np.max(sigma))))
    off = torch.arange(-rad, rad + 2, device=dev, dtype=torch.float64)
    xy = torch.as_tensor(xy, device=dev, dtype=torch.float64)
    flux = torch.as_tensor(np.asarray(flux), device=dev, dtype=torch.float64)
    sg = torch.as_tensor(np.asarray(sigma), device=dev, dtype=torch.float64)
    for j in range(n_exp):
        p = xy[:, j]
        ok = torch.isfinite(p).all(-1)
        if not bool(ok.any()):
            continue
        p, f = p[ok], flux[ok]
        bx = torch.floor(p[:, 0])[:, None] + off[None, :]      # (m, K)
        by = torch.floor(p[:, 1])[:, None] + off[None, :]
        s2 = sg[j] ** 2
        gx = torch.exp(-0.5 * (bx - p[:, :1]) ** 2 / s2)
        gy = torch.exp(-0.5 * (by - p[:, 1:]) ** 2 / s2)
        val = (f / (2 * math.pi * s2))[:, None, None] * gy[:, :, None] * gx[:, None, :]
        X = bx[:, None, :].expand_as(val)
        Y = by[:, :, None].expand_as(val)
        m = (X >= 0) & (X < W) & (Y >= 0) & (Y < H)
        lin = (Y[m] * W + X[m]).long()
        images[j].view(-1).index_add_(0, lin, val[m].to(images.dtype))
    return images


# --------------------------------------------------------------------------
# Vetting survey (training and evaluation stamps for the learned vetter)
# --------------------------------------------------------------------------

def field_states(rng, n, lon, r_range=(2.3, 2.7), dv_kms=0.4, spread=2e-3):
    """Orbits near a tracked field: heliocentric distance r ~ U(r_range), a
    random angular offset (up to ``spread`` rad in longitude and latitude) from
    the field's reference direction at t0, circular prograde speed plus
    radial/tangential offsets ~ U(-dv, dv) km/s."""
    r = rng.uniform(*r_range, n)
    dl = rng.uniform(-spread, spread, n)
    db = rng.uniform(-spread, spread, n)
    L = lon + dl
    rh = np.stack([np.cos(L) * np.cos(db), np.sin(L) * np.cos(db), np.sin(db)], -1)
    th = np.stack([-np.sin(L), np.cos(L), np.zeros(n)], -1)
    vr = rng.uniform(-dv_kms, dv_kms, n) * KMS_TO_AUD
    vt = rng.uniform(-dv_kms, dv_kms, n) * KMS_TO_AUD
    vc = GAUSS_K / np.sqrt(r)
    pos = r[:, None] * rh
    vel = vr[:, None] * rh + (vc + vt)[:, None] * th
    return np.concatenate([pos, vel], 1)


def vetting_sky(*, seed, n_exp=10, nights=20.0, size=1024, scale_arcsec=2.0, n_src=400,
                n_art=400, n_rand=400, lon=0.7, snr_range=(3.0, 10.0), art_snr=(8.0, 25.0)) -> Sky:
    """Tracked field like the tiny plain-method workload (10 epochs over 20
    nights, pointings following a 2.5 AU circular body), larger and coarser so
    that hundreds of sources stay inside.  Draws: ``n_src`` injected asteroids
    with stacked SNR ~ U(snr_range) over the n_exp exposures (the per-image
    flux is the stacked SNR / sqrt(n_exp)); ``n_art`` single-exposure
    artefacts (an orbit, one exposure index and a per-image SNR ~ U(art_snr));
    ``n_rand`` unrelated random orbits.  meta holds the artefact and random
    orbits."""
    rng = np.random.default_rng(seed)
    step = nights / n_exp
    mjd = 60000.5 + step * np.arange(n_exp) + rng.uniform(-0.1, 0.1, n_exp)
    t0 = float(60000.5 + step * (n_exp - 1) / 2.0)
    obs = observer_position(mjd, t0, lon)
    crval = tracking_pointings(mjd, obs, t0, 2.5, lon)
    s = scale_arcsec / 3600.0
    sigma = rng.uniform(1.3, 1.8, n_exp).astype(np.float32).astype(np.float64)
    ex = Exposures(mjd=mjd, obs=obs, crval=crval,
                   crpix=np.tile(np.array([size / 2.0, size / 2.0]), (n_exp, 1)),
                   cd=np.tile(np.array([[-s, 0.0], [0.0, s]]), (n_exp, 1, 1)), sigma=sigma,
                   var=np.ones(n_exp), width=np.full(n_exp, size, np.int32),
                   height=np.full(n_exp, size, np.int32))
    src = field_states(rng, n_src, lon)
    snr = rng.uniform(*snr_range, n_src)
    flux = flux_for_snr(snr / math.sqrt(n_exp), 1.55, 1.0)
    art = field_states(rng, n_art, lon)
    art_exp = rng.integers(0, n_exp, n_art)
    art_flux = flux_for_snr(rng.uniform(*art_snr, n_art), 1.55, 1.0)
    rand = field_states(rng, n_rand, lon)
    return Sky(name="vetting", ex=ex, t0=t0, states=src, inj_states=src, inj_flux=flux,
               inj_orbit=np.arange(n_src), seed=seed,
               meta=dict(snr=snr, art_states=art, art_exp=art_exp, art_flux=art_flux,
                         rand_states=rand))


# --------------------------------------------------------------------------
# Batched uneven workload (orbit families with uneven exposure coverage)
# --------------------------------------------------------------------------

def batched_sky(*, n_fam=4096, fam_size=16384, n_exp=400, size=2048, days=365.0, seed=4,
                scale_arcsec=60.0, lon=1.2, fam_exp_range=(20, 400)) -> Sky:
    """Orbit families mixing near-Earth (q < 1.3 AU), main-belt and Kuiper-belt
    (30-50 AU) hypotheses, each a seed state near opposition at the mid-year
    epoch t0 plus seeded state jitter; each family is tested against a random
    subset of U[fam_exp_range] of the exposures (the CSR lists).  Exposures:
    pairs 30 min apart on n_exp/2 random nights of a year; pointings follow the
    anti-solar direction (a circular reference body just outside the observer's
    orbit) with a wide field."""
    rng = np.random.default_rng(seed)
    nights = np.sort(rng.choice(int(days), n_exp // 2, replace=False)).astype(np.float64)
    mjd = np.sort(np.concatenate([60000.3 + nights, 60000.3 + nights + 30.0 / 1440.0]))[:n_exp]
    t0 = float(60000.0 + days / 2.0)
    obs = observer_position(mjd, t0, lon)
    crval = tracking_pointings(mjd, obs, t0, 1.0001, lon)
    s = scale_arcsec / 3600.0
    sigma = rng.uniform(1.2, 2.0, n_exp).astype(np.float32).astype(np.float64)
    ex = Exposures(mjd=mjd, obs=obs, crval=crval,
                   crpix=np.tile(np.array([size / 2.0, size / 2.0]), (n_exp, 1)),
                   cd=np.tile(np.array([[-s, 0.0], [0.0, s]]), (n_exp, 1, 1)), sigma=sigma,
                   var=np.ones(n_exp), width=np.full(n_exp, size, np.int32),
                   height=np.full(n_exp, size, np.int32))
    kind = rng.integers(0, 3, n_fam)                         # 0 NEO, 1 MBA, 2 KBO
    a = np.where(kind == 0, rng.uniform(1.0, 2.0, n_fam),
                 np.where(kind == 1, rng.uniform(2.1, 3.3, n_fam), rng.uniform(30.0, 50.0, n_fam)))
    e_max = np.where(kind == 0, 0.6, 0.2)
    e = rng.uniform(0.0, 1.0, n_fam) * e_max
    e = np.where(kind == 0, np.maximum(e, 1.0 - 1.3 / a + 1e-3), e)   # q < 1.3 AU
    inc = np.radians(rng.uniform(0.0, 15.0, n_fam))
    u = rng.uniform(-0.05, 0.05, n_fam)
    lam = lon + rng.uniform(-0.05, 0.05, n_fam)
    node = lam - np.arctan2(np.cos(inc) * np.sin(u), np.cos(u))
    argp = rng.uniform(0.0, 2 * math.pi, n_fam)
    seeds = state_from_elements(a, e, inc, node, argp, u - argp)
    states = np.repeat(seeds, fam_size, axis=0)
    r = np.linalg.norm(seeds[:, :3], axis=1).repeat(fam_size)
    jit = np.concatenate([rng.normal(0.0, 1.0, (len(states), 3)) * (1e-4 * r)[:, None],
                          rng.normal(0.0, 1.0, (len(states), 3)) * (2e-6 / np.sqrt(r))[:, None]], 1)
    jit[::fam_size] = 0.0
    states += jit
    fo = (np.arange(n_fam + 1) * fam_size).astype(np.int64)
    counts = rng.integers(fam_exp_range[0], fam_exp_range[1] + 1, n_fam)
    fe = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    fi = np.concatenate([rng.choice(n_exp, c, replace=False) for c in counts]).astype(np.int32)
    return Sky(name="batched", ex=ex, t0=t0, states=states, inj_states=seeds,
               inj_flux=np.zeros(n_fam), inj_orbit=fo[:-1].copy(), seed=seed,
               families=(fo, fe, fi), meta=dict(kind=kind, fam_size=fam_size))


# --------------------------------------------------------------------------
# Sparse regime (each orbit meets a small fraction of many small exposures)
# --------------------------------------------------------------------------

def sparse_sky(*, n_exp=20000, days=365.0, fields=14, visits=4, size=512, scale_arcsec=10.0, n_fam=256,
               fam_size=4096, n_inj=64, inj_snr=(2.0, 4.0), seed=7, lon=1.2, field_lon=0.12,
               field_lat=0.06, inc_max_deg=4.0) -> Sky:
    """The paper's sparse regime: a year of small exposures (``size``^2 px at
    ``scale_arcsec``).  Each night ``fields`` random fields within
    +-field_lon rad of the anti-solar ecliptic longitude and +-field_lat rad
    of the ecliptic are each visited ``visits`` times 25 minutes apart.
    Candidate orbits: ``n_fam`` families of main-belt hypotheses (a in
    [2.1, 3.3] AU, e < 0.2, i < inc_max_deg) near opposition at the mid-year
    epoch t0, each its seed state plus ``fam_size - 1`` jittered neighbours;
    the seeds of the first ``n_inj`` families are injected with per-image SNR
    ~ U(inj_snr).  An orbit crosses the chips of well under one percent of the
    exposures."""
    rng = np.random.default_rng(seed)
    per_night = fields * visits
    nights = int(math.ceil(n_exp / per_night))
    night = np.repeat(np.arange(nights, dtype=np.float64), per_night)[:n_exp]
    k = np.tile(np.arange(per_night), nights)[:n_exp]
    field, visit = k % fields, k // fields
    mjd = 60000.2 + night * (days / nights) + (field * 1.5 + visit * 25.0) / 1440.0
    t0 = float(60000.0 + days / 2.0)
    obs = observer_position(mjd, t0, lon)
    theta = lon + GAUSS_K * (night * (days / nights) + 60000.2 - t0)   # anti-solar longitude per night
    off_l = rng.uniform(-field_lon, field_lon, (nights, fields))
    off_b = rng.uniform(-field_lat, field_lat, (nights, fields))
    ni = night.astype(np.int64)
    lam = theta + off_l[ni, field]
    beta = off_b[ni, field]
    vec = np.stack([np.cos(beta) * np.cos(lam), np.cos(beta) * np.sin(lam), np.sin(beta)], -1)
    crval = ecliptic_to_radec_deg(vec)
    s = scale_arcsec / 3600.0
    sigma = rng.uniform(1.2, 2.0, n_exp).astype(np.float32).astype(np.float64)
    ex = Exposures(mjd=mjd, obs=obs, crval=crval,
                   crpix=np.tile(np.array([size / 2.0, size / 2.0]), (n_exp, 1)),
                   cd=np.tile(np.array([[-s, 0.0], [0.0, s]]), (n_exp, 1, 1)), sigma=sigma,
                   var=np.ones(n_exp), width=np.full(n_exp, size, np.int32),
                   height=np.full(n_exp, size, np.int32))
    a = rng.uniform(2.1, 3.3, n_fam)
    e = rng.uniform(0.0, 0.2, n_fam)
    inc = np.radians(rng.uniform(0.0, inc_max_deg, n_fam))
    u = rng.uniform(-0.05, 0.05, n_fam)
    u = np.where(rng.random(n_fam) < 0.5, u, u + math.pi)
    lam0 = lon + rng.uniform(-0.1, 0.1, n_fam)
    node = lam0 - np.arctan2(np.cos(inc) * np.sin(u), np.cos(u))
    argp = rng.uniform(0.0, 2 * math.pi, n_fam)
    seeds = state_from_elements(a, e, inc, node, argp, u - argp)
    states = np.repeat(seeds, fam_size, axis=0)
    jit = np.concatenate([rng.normal(0.0, 3e-4, (len(states), 3)), rng.normal(0.0, 1e-5, (len(states), 3))], 1)
    jit[::fam_size] = 0.0
    states += jit
    snr = rng.uniform(*inj_snr, n_inj)
    return Sky(name="sparse", ex=ex, t0=t0, states=states, inj_states=seeds[:n_inj].copy(),
               inj_flux=flux_for_snr(snr, 1.6, 1.0), inj_orbit=np.arange(n_inj, dtype=np.int64) * fam_size,
               seed=seed, meta=dict(fam_size=fam_size, n_fam=n_fam, inj_snr=snr, size=size))
