"""The sparse regime (each orbit meets well under 1 % of many small
exposures): the persistent form with its block cone test against the FP64
oracle on a reduced survey, and on the full survey (20,000 exposures of
512^2, 1M orbits) the same in-bounds samples for every orbit in every form,
with the block test removing almost all of the per-pair work."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_08854_gb300 import ndt, synth

from _gpu_helpers import Gpu, check_stack

pytestmark = pytest.mark.gpu


@pytest.fixture
def gpu():
    g = Gpu()
    yield g
    g.close()


def _images(gpu, sky):
    imgs = synth.noise_images_torch(sky.ex, sky.seed, gpu.dev)
    xy = O.predict(sky.inj_states, sky.t0, sky.ex, nthreads=0)
    W = float(sky.ex.width[0])
    far = (xy[..., 0] < -20) | (xy[..., 0] > W + 20) | (xy[..., 1] < -20) | (xy[..., 1] > W + 20)
    xy[far] = np.nan                              # render only where a source is near the chip
    synth.render_sources_torch(imgs, xy, sky.inj_flux, sky.ex.sigma)
    torch.cuda.synchronize()
    return imgs


def _stack(gpu, sky, imgs, plane, mode, tiles=(64, 16), block=True):
    ndt.load_exposures(gpu.ctx, sky.ex, imgs, plane_dtype=plane)
    if mode == "persistent":
        ndt.set_launch(gpu.ctx, ndt.LAUNCH_PERSISTENT, tiles[0], tiles[1], use_graph=True)
    else:
        ndt.set_launch(gpu.ctx, ndt.LAUNCH_PLAIN)
    ndt.set_block_test(gpu.ctx, block)
    n = len(sky.states)
    st = torch.from_numpy(np.ascontiguousarray(sky.states.T)).to(gpu.dev)
    out = dict(psi=torch.empty(n, device=gpu.dev), phi=torch.empty(n, device=gpu.dev),
               nobs=torch.empty(n, dtype=torch.int32, device=gpu.dev), snr=torch.empty(n, device=gpu.dev))
    torch.cuda.synchronize()
    ndt.stack_orbits(gpu.ctx, st, sky.t0, n, psi_sum=out["psi"], phi_sum=out["phi"], nobs=out["nobs"],
                     snr=out["snr"])
    ndt.synchronize(gpu.ctx)
    assert gpu.stats()["kepler_failures"] == 0
    return out


@pytest.mark.parametrize("tiles", [(32, 8), (64, 16), (128, 32)])
def test_sparse_block_test_matches_oracle(gpu, tiles):
    sky = synth.sparse_sky(n_exp=3000, n_fam=8, fam_size=128, n_inj=4, seed=11)
    imgs = _images(gpu, sky)
    out = _stack(gpu, sky, imgs, "f32", "persistent", tiles=tiles)
    st = gpu.stats()
    host = imgs.cpu().numpy()
    ref = O.stack(sky.states, sky.t0, sky.ex, images=[host[j] for j in range(sky.ex.n)], nthreads=0)
    check_stack({k: v.cpu().numpy() for k, v in out.items()}, ref)
    assert 0 < st["valid_samples"] < 0.01 * st["samples"]          # the sparse regime
    assert st["block_skipped"] > 0.5 * st["samples"], st


def test_sparse_full_size_forms_count_the_same_samples(gpu, capsys):
    sky = synth.sparse_sky()
    imgs = _images(gpu, sky)
    plain = _stack(gpu, sky, imgs, "f32", "plain")
    st_plain = gpu.stats()
    off = _stack(gpu, sky, imgs, "bf16", "persistent", block=False)
    st_off = gpu.stats()
    on = _stack(gpu, sky, imgs, "bf16", "persistent", block=True)
    st_on = gpu.stats()
    assert torch.equal(plain["nobs"], off["nobs"]) and torch.equal(plain["nobs"], on["nobs"])
    assert st_on["valid_samples"] == st_plain["valid_samples"]
    assert st_plain["valid_samples"] < 0.01 * st_plain["samples"]
    assert st_on["block_skipped"] > 0.9 * st_on["samples"], st_on
    with capsys.disabled():
        print(f"\nsparse survey: {st_on['samples']} pairs, {st_on['valid_samples']} in bounds; "
              f"stack ms plain {st_plain['last_stack_ms']:.1f}, off-chip test "
              f"{st_off['last_stack_ms']:.1f}, + block test {st_on['last_stack_ms']:.1f}; block test "
              f"skipped {st_on['block_skipped'] / st_on['samples']:.4f} of the pairs")


def test_footprint_order_matches_oracle_and_restores_skipping(gpu):
    """The reduced survey's orbits in a random order (families interleaved):
    with the footprint order (ndt_set_footprint_sort) both forms match the
    oracle orbit by orbit, in the caller's order, and the persistent form's
    block test skips at least as many samples as without it."""
    sky = synth.sparse_sky(n_exp=3000, n_fam=8, fam_size=128, n_inj=4, seed=11)
    imgs = _images(gpu, sky)
    sky.states = sky.states[np.random.default_rng(5).permutation(len(sky.states))]
    _stack(gpu, sky, imgs, "f32", "persistent")
    st_shuffled = gpu.stats()
    ndt.set_footprint_sort(gpu.ctx, True)
    ordered = _stack(gpu, sky, imgs, "f32", "persistent")
    st_ordered = gpu.stats()
    plain = _stack(gpu, sky, imgs, "f32", "plain")
    host = imgs.cpu().numpy()
    ref = O.stack(sky.states, sky.t0, sky.ex, images=[host[j] for j in range(sky.ex.n)], nthreads=0)
    check_stack({k: v.cpu().numpy() for k, v in ordered.items()}, ref)
    check_stack({k: v.cpu().numpy() for k, v in plain.items()}, ref)
    assert st_ordered["valid_samples"] == st_shuffled["valid_samples"]
    assert st_ordered["block_skipped"] >= st_shuffled["block_skipped"], (st_ordered, st_shuffled)
    assert st_ordered["block_skipped"] > 0.5 * st_ordered["samples"], st_ordered
