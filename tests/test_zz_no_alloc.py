"""ndt_topk_noalloc, the ranking entry point for callers that cannot let the
library allocate device memory (its scratch is a fixed array inside the
library), gives the same ranking as ndt_topk_candidates on two calls in a row
with different inputs and k, so nothing left in the shared array from one
call leaks into the next.  Runs last (file name) and also alone."""
import numpy as np
import pytest
import torch

from paper_2503_08854_gb300 import ndt, synth

from _gpu_helpers import Gpu

pytestmark = pytest.mark.gpu


def _stacked_snr(g, sky, imgs, states):
    g.load(sky.ex, imgs)
    n = len(states)
    snr = torch.empty(n, device=g.dev)
    ndt.stack_orbits(g.ctx, g.soa(states), sky.t0, n, snr=snr)
    ndt.synchronize(g.ctx)
    return snr


def test_noalloc_topk_matches_context_topk_twice():
    g = Gpu()
    try:
        sky = synth.grid_sky(n_exp=6, size=100, n_r=4, n_v=32, scale_arcsec=1.0, seed=3)
        imgs = synth.noise_images(sky.ex, sky.seed)
        for call, (states, k) in enumerate([(sky.states, 100), (sky.states[::3], 1500)]):
            snr = _stacked_snr(g, sky, imgs, states)
            n = len(states)
            ref_i = torch.empty(k, dtype=torch.int64, device=g.dev)
            ref_v = torch.empty(k, device=g.dev)
            got = ndt.topk_candidates(g.ctx, k, ref_i, ref_v)   # k is clamped to n
            assert got == min(k, n)
            idx = torch.full((k,), -7, dtype=torch.int64, device=g.dev)
            val = torch.full((k,), -7.0, device=g.dev)
            ndt.topk_noalloc(snr, n, k, idx, val, stream=g.stream)
            g.stream.synchronize()
            assert torch.equal(idx[:got], ref_i[:got]), f"call {call}: indices differ"
            assert torch.equal(val[:got], ref_v[:got]), f"call {call}: values differ"
            assert bool((idx[got:] == -7).all())                 # nothing written past n
            assert np.isfinite(val[:10].cpu().numpy()).all()
        with pytest.raises(ndt.NdtError):      # above the stated limit
            ndt.topk_noalloc(snr, len(snr), 8193, idx, val, stream=g.stream)
        with pytest.raises(ndt.NdtError):      # host input
            ndt.topk_noalloc(snr.cpu(), len(snr), 10, idx, val, stream=g.stream)
    finally:
        g.close()
