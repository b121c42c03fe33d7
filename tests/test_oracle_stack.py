"""Pins of the oracle's matched filter, constant-flux stacking and ranking
(paper sec. 3: a matched filter for a Gaussian PSF of the header's width,
per-image signals combined under a constant-flux assumption; Algorithm 1,
FindSignificantResults)."""
import math

import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle as O
from paper_2503_08854_gb300 import synth


def _gauss_kernel(sigma):
    R = int(math.ceil(4 * sigma))
    k = np.arange(-R, R + 1)
    w = np.exp(-(k[:, None] ** 2 + k[None, :] ** 2) / (2 * sigma * sigma))
    return w / w.sum(), R


@pytest.mark.parametrize("sigma", [0.8, 1.5, 2.0])
def test_psf_kernel_shape(sigma):
    P = O.psf_kernel(sigma)
    R = int(math.ceil(4 * sigma))
    assert P.shape == (2 * R + 1, 2 * R + 1)
    assert P.sum() == pytest.approx(1.0, abs=1e-14)
    np.testing.assert_allclose(P, P.T, atol=0)
    np.testing.assert_allclose(P, P[::-1, ::-1], atol=0)
    assert P[R, R + 1] / P[R, R] == pytest.approx(math.exp(-1 / (2 * sigma ** 2)), rel=1e-14)
    assert P[R + 1, R + 1] / P[R, R] == pytest.approx(math.exp(-1 / sigma ** 2), rel=1e-14)


def test_planes_of_delta_and_constant_images():
    sigma, V = 1.5, 2.5
    P, R = _gauss_kernel(sigma)
    img = np.zeros((40, 40), np.float32)
    img[20, 20] = 1.0
    psi, phi = O.planes(img, sigma, V)
    np.testing.assert_allclose(psi[20 - R:21 + R, 20 - R:21 + R], P / V, atol=1e-15)
    assert abs(psi).sum() == pytest.approx(1.0 / V, rel=1e-12)
    inner = phi[R:-R, R:-R]
    np.testing.assert_allclose(inner, (P ** 2).sum() / V, rtol=1e-13)
    assert phi[0, 0] < inner[0, 0]           # window truncated by the image edge
    c = np.full((40, 40), 3.25, np.float32)
    psi_c, _ = O.planes(c, sigma, V)
    np.testing.assert_allclose(psi_c[R:-R, R:-R], 3.25 / V, rtol=1e-13)


@pytest.mark.parametrize("per_pixel_var", [False, True])
def test_planes_match_library_correlation(per_pixel_var):
    """psi = (I/V) correlated with P, phi = (1/V) correlated with P^2, zero outside the image."""
    rng = np.random.default_rng(0)
    sigma = 1.3
    img = rng.normal(size=(37, 53)).astype(np.float32)
    if per_pixel_var:
        var = rng.uniform(0.5, 2.0, size=img.shape).astype(np.float32)
        psi, phi = O.planes(img, sigma, var)
        Vd = var.astype(np.float64)
    else:
        psi, phi = O.planes(img, sigma, 1.7)
        Vd = np.full(img.shape, 1.7)
    P, _ = _gauss_kernel(sigma)
    ref_psi = ndi.correlate(img.astype(np.float64) / Vd, P, mode="constant", cval=0.0)
    ref_phi = ndi.correlate(1.0 / Vd, P ** 2, mode="constant", cval=0.0)
    np.testing.assert_allclose(psi, ref_psi, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(phi, ref_phi, rtol=1e-12, atol=1e-16)


@pytest.mark.parametrize("var", [1.0, 2.5])
def test_pure_noise_snr_is_standard_normal(var):
    """For constant V, psi ~ N(0, sum P^2 / V) = N(0, phi): psi / sqrt(phi) has unit variance."""
    rng = np.random.default_rng(42)
    img = (rng.normal(size=(300, 300)) * math.sqrt(var)).astype(np.float32)
    psi, phi = O.planes(img, 1.5, var)
    z = (psi / np.sqrt(phi))[10:-10, 10:-10]
    assert abs(z.mean()) < 0.05
    assert abs(z.std() - 1.0) < 0.05


def _on_centre_exposures(state, t0, mjds, crpix, size, sigma, var):
    """Exposures whose tangent point is the object's apparent direction, so the
    object projects exactly onto the pixel centre ``crpix``."""
    n = len(mjds)
    obs = synth.observer_position(mjds, t0, 0.4)
    crval = np.zeros((n, 2))
    for j in range(n):
        rho, _ = O.apparent(state, t0, mjds[j], obs[j])
        _, _, _, ra, dec = O.project(rho, [0, 0], [0, 0], [[1, 0], [0, 1]])
        crval[j] = [math.degrees(ra), math.degrees(dec)]
    s = 1.0 / 3600
    return synth.Exposures(
        mjd=np.asarray(mjds, float), obs=obs, crval=crval, crpix=np.tile(crpix, (n, 1)),
        cd=np.tile([[-s, 0], [0, s]], (n, 1, 1)), sigma=np.full(n, sigma), var=np.full(n, var),
        width=np.full(n, size, np.int32), height=np.full(n, size, np.int32))


@pytest.mark.parametrize("n_exp", [1, 4, 9])
def test_snr_closed_form_on_pixel_centres(n_exp):
    """Noise-free source of flux F exactly on a pixel centre in N images:
    psi = F sum P^2 / V per image, so nu = F sqrt(N sum P^2 / V)."""
    sigma, V, F, size = 1.5, 2.0, 7.0, 41
    state = np.array([2.3, 0.9, 0.1, -0.004, 0.010, 0.0005])
    t0 = 60000.0
    ex = _on_centre_exposures(state, t0, t0 + np.linspace(-5, 5, n_exp), [20.0, 20.0], size, sigma, V)
    P, R = _gauss_kernel(sigma)
    imgs = np.zeros((n_exp, size, size), np.float32)
    imgs[:, 20 - R:21 + R, 20 - R:21 + R] = (F * P).astype(np.float32)
    xy = O.predict(state[None], t0, ex)
    np.testing.assert_allclose(xy[0], 20.0, atol=1e-8)
    out = O.stack(state[None], t0, ex, images=list(imgs))
    sP2 = (P ** 2).sum()
    fP = (F * P).astype(np.float32).astype(np.float64)   # the FP32 image actually stored
    assert out["nobs"][0] == n_exp
    assert out["Psi"][0] == pytest.approx(n_exp * (fP * P).sum() / V, rel=1e-13)
    assert out["Phi"][0] == pytest.approx(n_exp * sP2 / V, rel=1e-13)
    nu = O.snr(out["Psi"], out["Phi"], out["nobs"])
    assert nu[0] == pytest.approx(F * math.sqrt(n_exp * sP2 / V), rel=1e-6)


def test_ambiguous_edge_sample_is_bracketed():
    sigma, size = 1.5, 30
    state = np.array([2.3, 0.9, 0.1, -0.004, 0.010, 0.0005])
    t0 = 60000.0
    ex = _on_centre_exposures(state, t0, [t0 + 1.0], [10.5 + 1e-8, 12.0], size, sigma, 1.0)
    rng = np.random.default_rng(9)
    img = rng.normal(size=(size, size)).astype(np.float32)
    psi, phi = O.planes(img, sigma, 1.0)
    out = O.stack(state[None], t0, ex, images=[img], amb_px=1e-6)
    assert out["n_amb"][0] == 1 and out["nobs"][0] == 1
    assert out["Psi"][0] == pytest.approx(psi[12, 11], rel=1e-12)
    assert out["psi_lo"][0] == pytest.approx(min(psi[12, 10], psi[12, 11]), rel=1e-12)
    assert out["psi_hi"][0] == pytest.approx(max(psi[12, 10], psi[12, 11]), rel=1e-12)
    # an edge sample at the image border: the alternative lies outside
    ex2 = _on_centre_exposures(state, t0, [t0 + 1.0], [-0.5 + 1e-8, 12.0], size, sigma, 1.0)
    out2 = O.stack(state[None], t0, ex2, images=[img], amb_px=1e-6)
    assert out2["n_lo"][0] == 0 and out2["n_hi"][0] == 1 and out2["nobs"][0] == 1


def test_planes_and_on_demand_evaluation_agree():
    sky = synth.grid_sky(n_exp=4, size=64, n_r=2, n_v=8, scale_arcsec=2.0, seed=3)
    imgs = synth.noise_images(sky.ex, sky.seed)
    pl = [O.planes(imgs[j], sky.ex.sigma[j], sky.ex.var[j]) for j in range(sky.ex.n)]
    a = O.stack(sky.states, sky.t0, sky.ex, images=list(imgs))
    b = O.stack(sky.states, sky.t0, sky.ex, planes=([p[0] for p in pl], [p[1] for p in pl]))
    np.testing.assert_allclose(a["Psi"], b["Psi"], rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(a["nobs"], b["nobs"])
    assert a["nobs"].sum() > 0


def test_families_equal_separate_stacks():
    sky = synth.grid_sky(n_exp=6, size=64, n_r=2, n_v=8, scale_arcsec=2.0, seed=4)
    imgs = synth.noise_images(sky.ex, sky.seed)
    n = len(sky.states)
    fam_o = np.array([0, 40, n], np.int64)
    fam_e = np.array([0, 3, 7], np.int64)
    fam_i = np.array([0, 2, 5, 1, 2, 3, 4], np.int32)
    out = O.stack(sky.states, sky.t0, sky.ex, images=list(imgs), families=(fam_o, fam_e, fam_i))
    for f in range(2):
        sel = fam_i[fam_e[f]:fam_e[f + 1]]
        ref = O.stack(sky.states[fam_o[f]:fam_o[f + 1]], sky.t0, sky.ex.subset(sel),
                      images=list(imgs[sel]))
        np.testing.assert_allclose(out["Psi"][fam_o[f]:fam_o[f + 1]], ref["Psi"], rtol=1e-13, atol=1e-15)
        np.testing.assert_array_equal(out["nobs"][fam_o[f]:fam_o[f + 1]], ref["nobs"])


def _brute_topk(nu, k):
    """Selection by repeated scans: the largest value, lowest index first."""
    taken = np.zeros(len(nu), bool)
    out = []
    for _ in range(min(k, len(nu))):
        best = -1
        for i in range(len(nu)):
            if taken[i]:
                continue
            if best < 0 or nu[i] > nu[best]:
                best = i
        taken[best] = True
        out.append(best)
    return np.array(out, np.int64)


def test_topk_brute_force_with_ties():
    rng = np.random.default_rng(5)
    nu = np.round(rng.normal(size=300), 1)       # many exact ties
    nu[rng.integers(0, 300, 30)] = -np.inf
    for k in (1, 7, 50, 300, 400):
        idx, val = O.topk(nu, k)
        np.testing.assert_array_equal(idx, _brute_topk(nu, k))
        np.testing.assert_array_equal(val, nu[idx])


def test_snr_min_obs_and_empty():
    nu = O.snr([1.0, 2.0, 3.0], [4.0, 0.0, 9.0], [1, 3, 2], min_obs=2)
    assert nu[0] == -np.inf and nu[1] == -np.inf and nu[2] == pytest.approx(1.0)


def test_oracle_recovers_injected_sources():
    """Brute-force injected-source recovery on a tiny grid: sources at per-image
    SNR 4 on grid nodes appear among the top candidates of the stack."""
    sky = synth.grid_sky(n_exp=8, size=96, n_r=4, n_v=16, scale_arcsec=1.0, inj_snr=4.0,
                         n_inj=3, seed=6)
    xy = O.predict(sky.inj_states, sky.t0, sky.ex)
    inb = (xy[..., 0] > 0) & (xy[..., 0] < 95) & (xy[..., 1] > 0) & (xy[..., 1] < 95)
    assert inb.sum(axis=1).min() >= 6
    imgs = synth.noise_images(sky.ex, sky.seed)
    synth.render_sources(imgs, xy, sky.inj_flux, sky.ex.sigma)
    out = O.stack(sky.states, sky.t0, sky.ex, images=list(imgs))
    nu = O.snr(out["Psi"], out["Phi"], out["nobs"], min_obs=3)
    idx, _ = O.topk(nu, 10)
    assert set(sky.inj_orbit.tolist()) <= set(idx.tolist())
