"""GPU parity of ndt_dedup_candidates against the oracle (oracle/dedup.py):
clusters of jittered orbits around a few centres, ranked at random, so that
the kept list depends on the rank order, on several cells of the hash grid
and on candidates that fall outside the reference chips."""
import numpy as np
import pytest
import torch

from oracle import dedup as OD
from paper_2503_08854_gb300 import ndt, synth

from _gpu_helpers import Gpu

pytestmark = pytest.mark.gpu


@pytest.fixture
def gpu():
    g = Gpu()
    yield g
    g.close()


def _clusters(seed, n_centres=12, per=120, pos_sig=4e-6, vel_sig=2e-7):
    sky = synth.grid_sky(n_exp=10, size=512, n_r=16, n_v=16, scale_arcsec=0.2, seed=seed)
    rng = np.random.default_rng(seed)
    centres = sky.states[rng.choice(len(sky.states), n_centres, replace=False)]
    states = np.repeat(centres, per, axis=0)
    states[:, :3] += rng.normal(0, pos_sig, (len(states), 3))
    states[:, 3:] += rng.normal(0, vel_sig, (len(states), 3))
    rank = rng.permutation(len(states))      # the candidate list, best first
    return sky, states, rank


@pytest.mark.parametrize("n_ref,radius,windowed", [(3, 4.0, False), (1, 2.5, False), (5, 8.0, False),
                                                   (3, 4.0, True)])
def test_dedup_matches_oracle(gpu, n_ref, radius, windowed):
    sky, states, rank = _clusters(5)
    gpu.load(sky.ex, np.zeros((sky.ex.n, 512, 512), np.float32))
    n = len(rank)
    t = np.sort(sky.ex.mjd)
    window = (0.5 * (t[1] + t[2]), 0.5 * (t[6] + t[7])) if windowed else None
    cand = torch.as_tensor(rank, dtype=torch.int64, device=gpu.dev)
    out = torch.full((n,), -1, dtype=torch.int64, device=gpu.dev)
    nk = ndt.dedup_candidates(gpu.ctx, gpu.soa(states), sky.t0, len(states), cand, n, out,
                              radius_px=radius, n_ref=n_ref, window=window)
    got = out[:nk].cpu().numpy()
    assert bool((out[nk:] == -1).all())
    ref, dist = OD.dedup(states, sky.t0, sky.ex, rank, radius, n_ref, window)
    # each candidate's fate depends only on the distances to those ranked
    # before it: compare every candidate whose decision does not hinge on a
    # distance within 2e-4 px of the radius (FP32 coordinates on the GPU,
    # half an ulp is 3e-5 px at 500 px)
    amb = np.array([np.any(np.abs(dist[i, :i] - radius) < 2e-4) for i in range(n)])
    kept_g = np.isin(rank, got)
    kept_o = np.isin(rank, ref)
    assert amb.sum() <= n // 50
    assert np.array_equal(kept_g[~amb], kept_o[~amb])
    assert np.array_equal(got, rank[kept_g])         # rank order preserved
    assert 12 <= len(ref) < n // 4                   # the clusters collapse, not to nothing


def test_dedup_host_pointers_and_edges(gpu):
    sky, states, rank = _clusters(6, n_centres=3, per=40)
    gpu.load(sky.ex, np.zeros((sky.ex.n, 512, 512), np.float32))
    n = len(rank)
    out = np.full(n, -1, np.int64)
    nk = ndt.dedup_candidates(gpu.ctx, gpu.soa(states, host=True), sky.t0, len(states),
                              np.ascontiguousarray(rank, np.int64), n, out, radius_px=4.0)
    ref, _ = OD.dedup(states, sky.t0, sky.ex, rank, 4.0, 3)
    assert nk == len(ref) and set(out[:nk]) == set(ref)
    assert ndt.dedup_candidates(gpu.ctx, gpu.soa(states), sky.t0, len(states), out, 0, out) == 0
    # a single candidate and an out-of-range index are kept
    one = np.array([len(states) + 5, 0], np.int64)
    o2 = np.zeros(2, np.int64)
    assert ndt.dedup_candidates(gpu.ctx, gpu.soa(states), sky.t0, len(states), one, 2, o2) == 2
    with pytest.raises(ndt.NdtError):
        ndt.dedup_candidates(gpu.ctx, gpu.soa(states), sky.t0, len(states), one, 2, o2, radius_px=0.0)
    with pytest.raises(ndt.NdtError):
        ndt.dedup_candidates(gpu.ctx, gpu.soa(states), sky.t0, len(states), one, 2, o2, n_ref=9)
    with pytest.raises(ndt.NdtError):           # a window without exposures
        ndt.dedup_candidates(gpu.ctx, gpu.soa(states), sky.t0, len(states), one, 2, o2, window=(0.0, 1.0))


def test_count_candidates_matches_oracle_nu(gpu):
    """ndt_count_candidates against the oracle's stacked statistic: the
    number of orbits at or above each threshold, skipping thresholds that
    fall within the SNR tolerance of an oracle value."""
    import oracle as O
    sky = synth.grid_sky(n_exp=6, size=100, n_r=4, n_v=32, scale_arcsec=1.0, inj_snr=4.0, n_inj=3,
                         seed=3)
    imgs = synth.noise_images(sky.ex, sky.seed)
    synth.render_sources(imgs, O.predict(sky.inj_states, sky.t0, sky.ex), sky.inj_flux, sky.ex.sigma)
    gpu.load(sky.ex, imgs)
    n = len(sky.states)
    ndt.stack_orbits(gpu.ctx, gpu.soa(sky.states), sky.t0, n)
    ref = O.stack(sky.states, sky.t0, sky.ex, images=list(imgs))
    nu = O.snr(ref["Psi"], ref["Phi"], ref["nobs"])
    fin = nu[np.isfinite(nu)]
    checked = 0
    for thr in (-1.0, 0.0, 1.5, 3.0, 5.0, 1e9):
        if np.any(np.abs(fin - thr) <= 1e-5 * np.maximum(1.0, np.abs(fin))) or np.any(ref["n_amb"] > 0):
            continue
        assert ndt.count_candidates(gpu.ctx, thr) == int(np.sum(nu >= thr)), thr
        checked += 1
    assert checked >= 4
    with pytest.raises(ndt.NdtError):
        ndt.count_candidates(gpu.ctx, float("nan"))
