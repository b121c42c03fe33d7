"""Learned vetting of stacked candidates (paper sec. 5.2.3: a network that
learns to tell stacked images of real detections from stacks of false ones).

Training runs on the GPU through the library's own kernels: ndt_cnn_loss_grad
(forward + backward of the 52,929-parameter CNN) and ndt_cnn_adam_step.  The
training set is synthesised by the pipeline itself: injected asteroids stacked
along their true orbits (positives) against unrelated random orbits,
single-exposure artefacts and the strongest noise peaks of a stack over a
source-free sky (negatives).  The plain SNR threshold stays the fallback and
the yardstick: ``fpr_at_recall`` compares both at the same recall.
"""
from __future__ import annotations

import math

import numpy as np

from . import ndt, synth

N_PARAMS = 52929
STAMP_ELEMS = 2 * 21 * 21


def init_params(seed, device):
    """He-normal conv and linear weights, zero biases, as one flat FP32 tensor
    (layout of ndt_cnn_param_count)."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(int(seed))
    parts = []
    for shape, fan_in in (((32, 2, 5, 5), 50), ((32,), 0), ((32, 32, 5, 5), 800), ((32,), 0),
                          ((32, 32, 5, 5), 800), ((32,), 0), ((32,), 32), ((1,), 0)):
        n = int(np.prod(shape))
        if fan_in:
            gain = 2.0 if len(shape) == 4 else 1.0
            parts.append(torch.randn(n, generator=g, dtype=torch.float64) * math.sqrt(gain / fan_in))
        else:
            parts.append(torch.zeros(n, dtype=torch.float64))
    p = torch.cat(parts).to(torch.float32).to(device)
    assert p.numel() == N_PARAMS == ndt.cnn_param_count()
    return p


def train(ctx, params, x_bf16, labels, *, epochs=4, batch=256, lr=2e-3, seed=0):
    """Adam on the mean BCE; x_bf16 (n, 2, 21, 21) torch.bfloat16 and labels (n,)
    FP32 on the device.  Returns the per-step losses."""
    import torch
    dev = params.device
    n = x_bf16.shape[0]
    grad = torch.zeros_like(params)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    g = torch.Generator(device="cpu").manual_seed(int(seed))
    losses, step = [], 0
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g).to(dev)
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            xb = x_bf16.index_select(0, idx).contiguous()
            yb = labels.index_select(0, idx).contiguous()
            torch.cuda.synchronize(dev)
            losses.append(ndt.cnn_loss_grad(ctx, params, xb, yb, batch, grad))
            step += 1
            ndt.cnn_adam_step(ctx, params, grad, m, v, step, lr=lr)
    ndt.synchronize(ctx)
    return losses


def logits(ctx, params, x_bf16):
    import torch
    out = torch.empty(x_bf16.shape[0], device=params.device)
    torch.cuda.synchronize(params.device)
    ndt.cnn_forward(ctx, params, x_bf16, x_bf16.shape[0], out)
    return out


def fpr_at_recall(score_pos, score_neg, recall):
    """False-positive rate of the threshold that keeps ``recall`` of positives."""
    sp = np.sort(np.asarray(score_pos, np.float64))
    k = int(math.floor((1.0 - recall) * len(sp)))
    thr = sp[min(k, len(sp) - 1)]
    return float(np.mean(np.asarray(score_neg) >= thr)), float(thr)


def make_set(ctx, seed, device, *, n_sky=1, noise_trials=20000, n_peaks=400, trimmed=False, **sky_kw):
    """Stamps and labels from ``n_sky`` vetting skies.  Returns
    (stamps_bf16 (n,2,21,21) torch, labels (n,), kind (n,) numpy: 0 source,
    1 random orbit, 2 artefact, 3 noise peak, centre SNR (n,) numpy), and with
    ``trimmed`` also the outlier-trimmed SNR (n,) numpy."""
    import torch
    xs, ys, kinds, snrs, trims = [], [], [], [], []
    for s in range(n_sky):
        sky = synth.vetting_sky(seed=seed * 1000 + s, **sky_kw)
        ex, n_exp = sky.ex, sky.ex.n
        imgs = synth.noise_images_torch(ex, sky.seed, device)
        torch.cuda.synchronize(device)
        ndt.load_exposures(ctx, ex, imgs)
        pos_src = _predict(ctx, sky.inj_states, sky.t0, n_exp, device)
        synth.render_sources_torch(imgs, pos_src, sky.inj_flux, ex.sigma)
        art = sky.meta["art_states"]
        pos_art = _predict(ctx, art, sky.t0, n_exp, device)
        keep = torch.zeros_like(pos_art)
        keep[:] = float("nan")
        ae = torch.as_tensor(sky.meta["art_exp"], device=device)
        ar = torch.arange(len(art), device=device)
        keep[ar, ae] = pos_art[ar, ae]
        synth.render_sources_torch(imgs, keep, sky.meta["art_flux"], ex.sigma)
        torch.cuda.synchronize(device)
        ndt.load_exposures(ctx, ex, imgs)
        cand_states = np.concatenate([sky.inj_states, sky.meta["rand_states"], art])
        kind = np.concatenate([np.zeros(len(sky.inj_states)), np.ones(len(sky.meta["rand_states"])),
                               np.full(len(art), 2)]).astype(np.int64)
        x, c0, tr = _stamps(ctx, cand_states, sky.t0, device)
        xs.append(x); kinds.append(kind); snrs.append(c0); trims.append(tr)
        # noise peaks: the strongest of many random orbits on a source-free sky
        pure = synth.noise_images_torch(ex, sky.seed + 777, device)
        torch.cuda.synchronize(device)
        ndt.load_exposures(ctx, ex, pure)
        rng = np.random.default_rng(sky.seed + 5)
        trials = synth.field_states(rng, noise_trials, 0.7)
        st = torch.from_numpy(np.ascontiguousarray(trials.T)).to(device)
        torch.cuda.synchronize(device)
        ndt.stack_orbits(ctx, st, sky.t0, noise_trials, min_obs=3)
        idx = torch.empty(n_peaks, dtype=torch.int64, device=device)
        ndt.topk_candidates(ctx, n_peaks, idx)
        peaks = trials[idx.cpu().numpy()]
        x, c0, tr = _stamps(ctx, peaks, sky.t0, device)
        xs.append(x); kinds.append(np.full(len(peaks), 3)); snrs.append(c0); trims.append(tr)
    x = torch.cat(xs)
    kind = np.concatenate(kinds)
    y = torch.as_tensor((kind == 0).astype(np.float32), device=device)
    if trimmed:
        return x, y, kind, np.concatenate(snrs), np.concatenate(trims)
    return x, y, kind, np.concatenate(snrs)


def _predict(ctx, states, t0, n_exp, device):
    import torch
    st = torch.from_numpy(np.ascontiguousarray(np.asarray(states).T)).to(device)
    xy = torch.empty(len(states) * n_exp * 2, dtype=torch.float64, device=device)
    torch.cuda.synchronize(device)
    ndt.predict_positions(ctx, st, t0, len(states), xy)
    return xy.view(len(states), n_exp, 2)


def _stamps(ctx, states, t0, device):
    """BF16 stamps of the given orbits, their FP32 centre SNR and their
    outlier-trimmed SNR (sigma clipping of the intersections, kappa 3)."""
    import torch
    n = len(states)
    st = torch.from_numpy(np.ascontiguousarray(np.asarray(states).T)).to(device)
    cand = torch.arange(n, dtype=torch.int64, device=device)
    f32 = torch.empty((n, 2, 21, 21), device=device)
    bf = torch.empty((n, 2, 21, 21), dtype=torch.bfloat16, device=device)
    trimmed = torch.empty(n, device=device)
    torch.cuda.synchronize(device)
    ndt.stamps(ctx, st, t0, n, cand, f32, bf)
    ndt.trim_candidates(ctx, st, t0, n, cand, trimmed)
    return (bf, f32[:, 0, 10, 10].cpu().numpy().astype(np.float64),
            trimmed.cpu().numpy().astype(np.float64))
