"""GPU parity of outlier trimming (ndt_trim_candidates) against the FP64
oracle of oracle/trim.py, through the C ABI."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from oracle import trim as T
from paper_2503_08854_gb300 import ndt, synth

from _gpu_helpers import Gpu

pytestmark = pytest.mark.gpu


@pytest.fixture
def gpu():
    g = Gpu()
    yield g
    g.close()


def _sky_with_artefacts(n_art=12, seed=7):
    """The tiny sky with one asteroid and bright one-exposure artefacts on the
    tracks of other orbits; returns sky, images, candidate indices, artefact
    candidates' positions in the candidate list and their exposures."""
    sky = synth.grid_sky(n_r=2)
    imgs = synth.noise_images(sky.ex, sky.seed)
    xy_inj = O.predict(sky.inj_states[:1], sky.t0, sky.ex)
    synth.render_sources(imgs, xy_inj, 2.0 * sky.inj_flux[:1], sky.ex.sigma)
    rng = np.random.default_rng(seed)
    pool = np.setdiff1d(rng.choice(len(sky.states), 4096, replace=False), sky.inj_orbit)
    xy_p = O.predict(sky.states[pool], sky.t0, sky.ex)
    w, h = sky.ex.width[0], sky.ex.height[0]
    inner = (np.isfinite(xy_p[..., 0]) & (xy_p[..., 0] > 10) & (xy_p[..., 0] < w - 10) &
             (xy_p[..., 1] > 10) & (xy_p[..., 1] < h - 10))
    # artefacts at least 30 px from the asteroid's image in their exposure
    d_ast = np.hypot(xy_p[..., 0] - xy_inj[0, :, 0], xy_p[..., 1] - xy_inj[0, :, 1])
    inner &= ~(d_ast < 30.0)
    order = np.argsort(-inner.sum(1), kind="stable")[:n_art]
    assert np.all(inner[order].sum(1) >= 1)
    art_xy = np.full((n_art, sky.ex.n, 2), np.nan)
    art_j = np.zeros(n_art, np.int64)
    for a, b in enumerate(order):
        j = int(np.flatnonzero(inner[b])[rng.integers(inner[b].sum())])
        art_xy[a, j] = xy_p[b, j]
        art_j[a] = j
    flux = 40.0 * 2.0 * math.sqrt(4 * math.pi) * float(np.max(sky.ex.sigma))
    synth.render_sources(imgs, art_xy, np.full(n_art, flux), sky.ex.sigma)
    rand = rng.choice(len(sky.states), 300, replace=False)
    cand = np.concatenate([sky.inj_orbit[:1], pool[order], rand]).astype(np.int64)
    return sky, imgs, cand, np.arange(1, 1 + n_art), art_j


def _gpu_trim(gpu, sky, cand, **kw):
    st = gpu.soa(sky.states)
    cd = torch.as_tensor(cand, device=gpu.dev)
    nu = torch.empty(len(cand), device=gpu.dev)
    nk = torch.empty(len(cand), dtype=torch.int32, device=gpu.dev)
    torch.cuda.synchronize()
    ndt.trim_candidates(gpu.ctx, st, sky.t0, len(sky.states), cd, nu, nk, **kw)
    return nu.cpu().numpy().astype(np.float64), nk.cpu().numpy()


def _oracle(sky, imgs, cand, **kw):
    planes = [O.planes(imgs[j], sky.ex.sigma[j], sky.ex.var[j]) for j in range(sky.ex.n)]
    xy = O.predict(sky.states[cand], sky.t0, sky.ex)
    psi, phi, valid, amb = T.intersections(xy, planes, sky.ex.width, sky.ex.height)
    return T.trim(psi, phi, valid, **kw), amb.any(1), psi, phi, valid


@pytest.mark.parametrize("kappa", [3.0, 2.0])
def test_trim_matches_oracle(gpu, kappa):
    sky, imgs, cand, art, art_j = _sky_with_artefacts()
    gpu.load(sky.ex, imgs)
    nu, nk = _gpu_trim(gpu, sky, cand, kappa=kappa)
    ref, amb, _, _, valid = _oracle(sky, imgs, cand, kappa=kappa)
    # decisions within 1e-3 of the threshold may differ between FP32 and FP64
    ok = ~amb & (ref["margin"] > 1e-3)
    assert ok.sum() >= 0.9 * len(cand), ok.sum()
    assert np.array_equal(nk[ok], ref["n"][ok])
    fin = ok & np.isfinite(ref["nu"])
    err = np.abs(nu[fin] - ref["nu"][fin]) / np.maximum(1.0, np.abs(ref["nu"][fin]))
    assert err.max() <= 1e-5, err.max()
    assert np.all(np.isneginf(nu[ok & ~np.isfinite(ref["nu"])]))
    assert np.all(ref["n"][art] < valid[art].sum(1))             # every artefact orbit was trimmed


def test_infinite_kappa_equals_the_stacked_snr(gpu):
    sky, imgs, cand, _, _ = _sky_with_artefacts()
    gpu.load(sky.ex, imgs)
    nu, nk = _gpu_trim(gpu, sky, cand, kappa=float("inf"))
    out = gpu.stack(sky.states, sky.t0)
    np.testing.assert_array_equal(nk, out["nobs"][cand])
    fin = np.isfinite(out["snr"][cand])
    np.testing.assert_allclose(nu[fin], out["snr"][cand][fin], rtol=2e-6, atol=2e-6)


def test_trim_removes_artefacts_and_keeps_the_asteroid(gpu):
    sky, imgs, cand, art, art_j = _sky_with_artefacts()
    gpu.load(sky.ex, imgs)
    plain = gpu.stack(sky.states, sky.t0)["snr"][cand]
    nu, nk = _gpu_trim(gpu, sky, cand, kappa=3.0)
    assert np.all(plain[art] > 8.0)
    assert np.all(nu[art] < 4.0), nu[art]
    assert plain[0] > 8.0 and nu[0] > 0.8 * plain[0]


def test_trim_degenerate_inputs(gpu):
    sky, imgs, cand, _, _ = _sky_with_artefacts(n_art=2)
    gpu.load(sky.ex, imgs)
    bad = np.array([-1, len(sky.states), 0], np.int64)
    nu, nk = _gpu_trim(gpu, sky, bad)
    assert np.isneginf(nu[0]) and np.isneginf(nu[1]) and nk[0] == 0 and nk[1] == 0
    # host pointers give the same result as device pointers
    st = gpu.soa(sky.states, host=True)
    nu_h = np.zeros(len(cand), np.float32)
    nk_h = np.zeros(len(cand), np.int32)
    ndt.trim_candidates(gpu.ctx, st, sky.t0, len(sky.states), cand, nu_h, nk_h)
    nu_d, nk_d = _gpu_trim(gpu, sky, cand)
    np.testing.assert_array_equal(nk_h, nk_d)
    np.testing.assert_array_equal(nu_h.astype(np.float64), nu_d)
    # no candidates: nothing to do; bad parameters are rejected
    ndt.trim_candidates(gpu.ctx, st, sky.t0, len(sky.states), np.zeros(0, np.int64), nu_h)
    for kw in (dict(kappa=0.0), dict(kappa=-1.0), dict(max_iter=0), dict(min_obs=-1)):
        with pytest.raises(ndt.NdtError):
            ndt.trim_candidates(gpu.ctx, st, sky.t0, len(sky.states), cand, nu_h, **kw)
