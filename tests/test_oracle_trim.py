"""Pins of the outlier-trimming oracle (paper sec. 5.2.3) against closed
forms, statistics and the independent C stacking oracle."""
import math

import numpy as np

import oracle as O
from oracle import trim as T
from paper_2503_08854_gb300 import synth


def _phi(rng, n, J):
    return rng.uniform(0.02, 0.2, (n, J))


def test_noise_free_constant_flux_keeps_everything():
    rng = np.random.default_rng(0)
    phi = _phi(rng, 50, 40)
    a = rng.uniform(0.5, 30.0, (50, 1))
    psi = a * phi
    valid = np.ones_like(phi, bool)
    out = T.trim(psi, phi, valid, kappa=3.0)
    assert np.all(out["n"] == 40) and np.all(out["rounds"] == 1)
    np.testing.assert_allclose(out["nu"], a[:, 0] * np.sqrt(phi.sum(1)), rtol=1e-13)


def test_single_spike_is_removed_closed_form():
    """Constant flux a plus a spike of A sigma in exposure m: the first round
    clips m, a_hat becomes a exactly, the second round confirms; the trimmed
    SNR is a sqrt(Phi - phi_m) and the untrimmed one is larger."""
    rng = np.random.default_rng(1)
    J, a, A = 30, 2.0, 25.0
    phi = _phi(rng, 1, J)
    psi = a * phi
    m = 7
    psi[0, m] += A * np.sqrt(phi[0, m])
    valid = np.ones_like(phi, bool)
    out = T.trim(psi, phi, valid, kappa=3.0)
    assert out["n"][0] == J - 1 and out["rounds"][0] == 2
    clean = a * np.sqrt(phi.sum() - phi[0, m])
    assert out["nu"][0] == np.float64(out["Psi"][0] / np.sqrt(out["Phi"][0]))
    assert math.isclose(out["nu"][0], clean, rel_tol=1e-13)
    assert psi.sum() / np.sqrt(phi.sum()) > clean + 3.0


def test_pure_noise_clips_the_upper_three_sigma_tail():
    """Pure noise: each residual is ~N(0, 1) (slightly less: a_hat is fitted),
    so about P(Z > 3) = 0.00135 of the intersections are clipped."""
    rng = np.random.default_rng(2)
    n, J = 4000, 100
    phi = _phi(rng, n, J)
    psi = rng.normal(size=(n, J)) * np.sqrt(phi)
    valid = np.ones_like(phi, bool)
    out = T.trim(psi, phi, valid, kappa=3.0)
    frac = 1.0 - out["n"].sum() / (n * J)
    p = 0.5 * math.erfc(3.0 / math.sqrt(2.0))
    sd = math.sqrt(p / (n * J))
    assert abs(frac - p) < 5 * sd + 2e-4, (frac, p)


def test_infinite_kappa_is_the_plain_stack_and_matches_the_c_oracle():
    """kappa = inf trims nothing, so the sums over valid intersections must
    equal the independent C oracle's stacked Psi, Phi and n_obs."""
    sky = synth.grid_sky(n_r=2)
    imgs = synth.noise_images(sky.ex, sky.seed)
    xy = O.predict(sky.inj_states, sky.t0, sky.ex)
    synth.render_sources(imgs, xy, sky.inj_flux, sky.ex.sigma)
    planes = [O.planes(imgs[j], sky.ex.sigma[j], sky.ex.var[j]) for j in range(sky.ex.n)]
    sel = np.concatenate([sky.inj_orbit, np.arange(0, len(sky.states), 97)])
    xy = O.predict(sky.states[sel], sky.t0, sky.ex)
    psi, phi, valid, amb = T.intersections(xy, planes, sky.ex.width, sky.ex.height)
    out = T.trim(psi, phi, valid, kappa=np.inf)
    ref = O.stack(sky.states[sel], sky.t0, sky.ex, planes=([p[0] for p in planes], [p[1] for p in planes]))
    ok = ref["n_amb"] == 0
    assert ok.sum() > 0.9 * len(sel)
    assert np.array_equal(out["n"][ok], ref["nobs"][ok])
    np.testing.assert_allclose(out["Psi"][ok], ref["Psi"][ok], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(out["Phi"][ok], ref["Phi"][ok], rtol=1e-12, atol=1e-15)
    assert np.all(out["rounds"] == 1)


def test_artefact_in_one_exposure_is_trimmed_on_a_rendered_sky():
    """One injected asteroid (alone: the tiny sky's five sources share a ray at
    t0 and pile up mid-span, which the constant-flux rule rightly clips) plus
    a bright point artefact placed on another orbit's track in one exposure:
    trimming removes the artefact's intersection from that orbit (its SNR
    collapses) and leaves the asteroid's SNR nearly intact."""
    sky = synth.grid_sky(n_r=2)
    imgs = synth.noise_images(sky.ex, sky.seed)
    xy_inj = O.predict(sky.inj_states[:1], sky.t0, sky.ex)
    synth.render_sources(imgs, xy_inj, 2.0 * sky.inj_flux[:1], sky.ex.sigma)
    # a non-injected orbit that stays inside the chip for the most exposures
    rng = np.random.default_rng(3)
    pool = np.setdiff1d(rng.choice(len(sky.states), 2048, replace=False), sky.inj_orbit)
    xy_p = O.predict(sky.states[pool], sky.t0, sky.ex)
    w, h = sky.ex.width[0], sky.ex.height[0]
    inner = (np.isfinite(xy_p[..., 0]) & (xy_p[..., 0] > 10) & (xy_p[..., 0] < w - 10) &
             (xy_p[..., 1] > 10) & (xy_p[..., 1] < h - 10))
    best = int(np.argmax(inner.sum(1)))
    assert inner[best].sum() >= 4
    o = int(pool[best])
    j = int(np.flatnonzero(inner[best])[0])
    art = np.full((1, sky.ex.n, 2), np.nan)
    art[0, j] = xy_p[best, j]
    flux = 40.0 * 2.0 * math.sqrt(4 * math.pi) * sky.ex.sigma[j]     # per-image SNR ~40
    synth.render_sources(imgs, art, np.array([flux]), sky.ex.sigma)
    planes = [O.planes(imgs[k], sky.ex.sigma[k], sky.ex.var[k]) for k in range(sky.ex.n)]
    cand = np.array([sky.inj_orbit[0], o])
    xy = O.predict(sky.states[cand], sky.t0, sky.ex)
    psi, phi, valid, _ = T.intersections(xy, planes, sky.ex.width, sky.ex.height)
    plain = psi.sum(1) / np.sqrt(phi.sum(1))
    out = T.trim(psi, phi, valid, kappa=3.0)
    assert plain[-1] > 8.0 and out["nu"][-1] < 4.0            # the artefact's orbit collapses
    assert valid[-1, j] and not out["kept"][-1, j]            # by losing the artefact's intersection
    assert out["n"][-1] >= valid[-1].sum() - 2
    assert plain[0] > 8.0 and out["nu"][0] > 0.8 * plain[0], (plain[0], out["nu"][0])
