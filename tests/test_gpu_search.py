"""GPU tests of filter broadening and the coarse-to-fine search (paper
sec. 5.2.4): broadened planes against the oracle's planes for the broadened
Gaussian, and a coarse-to-fine pass that recovers an injected asteroid with
a fraction of the dense grid's orbits."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_08854_gb300 import ndt, search, synth

from _gpu_helpers import Gpu

pytestmark = pytest.mark.gpu


@pytest.fixture
def gpu():
    g = Gpu()
    yield g
    g.close()


@pytest.mark.parametrize("broaden", [1.0, 3.0])
def test_broadened_planes_match_oracle(gpu, broaden):
    sky = synth.grid_sky(n_r=1, n_exp=3, size=200)
    imgs = synth.noise_images(sky.ex, sky.seed)
    imgs[:, 50:60, 70:80] += 20.0
    ndt.set_filter_broadening(gpu.ctx, broaden)
    gpu.load(sky.ex, imgs)
    ndt.set_filter_broadening(gpu.ctx, 0.0)
    H, W = int(sky.ex.height[0]), int(sky.ex.width[0])
    for j in range(sky.ex.n):
        s_eff = math.sqrt(sky.ex.sigma[j] ** 2 + broaden ** 2)
        ref_psi, ref_phi = O.planes(imgs[j], s_eff, sky.ex.var[j])
        psi, phi = gpu.planes(j, H, W)
        scale = np.abs(ref_psi).max()
        np.testing.assert_allclose(psi, ref_psi, rtol=0, atol=1e-5 * scale)
        np.testing.assert_allclose(phi, ref_phi, rtol=1e-5)


def test_broadening_errors(gpu):
    sky = synth.grid_sky(n_r=1, n_exp=2, size=64)
    imgs = synth.noise_images(sky.ex, sky.seed)
    with pytest.raises(ndt.NdtError):
        ndt.set_filter_broadening(gpu.ctx, -1.0)
    ndt.set_filter_broadening(gpu.ctx, 4.0)        # sqrt(1.5^2 + 4^2) > 4 px
    with pytest.raises(ndt.NdtError):
        gpu.load(sky.ex, imgs)
    ndt.set_filter_broadening(gpu.ctx, 0.0)
    gpu.load(sky.ex, imgs)


def _local_grid(sky, n=32, true_at=(6, 6), px_per_step=2.0):
    """n x n grid of velocity offsets (radial, tangential in the ecliptic)
    around the injected asteroid 0; one step moves its track by about
    px_per_step pixels at the ends of the span; the asteroid is node true_at."""
    st = sky.inj_states[0]
    r = st[:3]
    rhat = r / np.linalg.norm(r)
    that = np.cross([0.0, 0.0, 1.0], rhat)
    that /= np.linalg.norm(that)
    # pixel displacement at the span's ends per unit velocity along each axis
    # (the oracle's projection), so that one step moves the track ~px_per_step
    probe = 1e-6
    test = np.array([st, st, st])
    test[1, 3:] += probe * rhat
    test[2, 3:] += probe * that
    xy = O.predict(test, sky.t0, sky.ex)
    ends = [0, sky.ex.n - 1]

    def step_for(i):
        d = np.hypot(*(xy[i, ends] - xy[0, ends]).T).max()
        return px_per_step * probe / d

    a = (np.arange(n) - true_at[0]) * step_for(1)
    b = (np.arange(n) - true_at[1]) * step_for(2)
    grid = np.empty((n, n, 6))
    grid[..., :3] = r
    grid[..., 3:] = st[3:] + a[:, None, None] * rhat + b[None, :, None] * that
    return grid


def test_coarse_to_fine_recovers_the_asteroid(gpu):
    sky = synth.grid_sky()          # its injected asteroids stay in the tracked field
    imgs = synth.noise_images(sky.ex, sky.seed)
    xy = O.predict(sky.inj_states[:1], sky.t0, sky.ex)
    flux = synth.flux_for_snr(np.array([4.0]), float(sky.ex.sigma[0]), float(sky.ex.var[0]))
    synth.render_sources(imgs, xy, flux, sky.ex.sigma)
    grid = _local_grid(sky)
    d_imgs = torch.from_numpy(imgs).to(gpu.dev)
    torch.cuda.synchronize()
    # dense reference: every node
    gpu.load(sky.ex, imgs)
    dense = gpu.stack(grid.reshape(-1, 6), sky.t0)["snr"].reshape(grid.shape[:-1])
    assert np.unravel_index(np.argmax(dense), dense.shape) == (6, 6)
    # the broadened filter gains signal from adjacent orbits: three steps away
    # (~6 px at the span's ends) it keeps more of the peak than the plain one
    ndt.set_filter_broadening(gpu.ctx, 2.0)
    gpu.load(sky.ex, imgs)
    ndt.set_filter_broadening(gpu.ctx, 0.0)
    broad = gpu.stack(grid[[6, 6], [6, 9]], sky.t0)["snr"]
    assert broad[1] / broad[0] > 1.2 * dense[6, 9] / dense[6, 6]
    assert broad[1] > dense[6, 9]
    # coarse (every 4th node, broadened) then fine around the 2 best
    out = search.coarse_to_fine(gpu.ctx, sky.ex, d_imgs, grid, sky.t0, stride=4, broaden_px=2.0,
                                k_coarse=2, radius=4, k=5, device=gpu.dev)
    assert tuple(out["best"][0]) == (6, 6)
    assert out["nu"][0] == pytest.approx(dense[6, 6], rel=1e-5)
    assert out["evaluated"] <= 0.3 * out["dense"]
