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


def track_rms(ctx, sky, cand, device, chunk=65536):
    """RMS pixel distance (n,) between each candidate's predicted track and
    its family's injected asteroid (family = index // fam_size) over the
    exposures where the asteroid's position lies on the chip, from the
    library's own positions (ndt_predict_positions); infinite for families
    without an injected asteroid."""
    import torch
    fam = sky.meta["fam_size"]
    n_exp = sky.ex.n
    W, H = float(sky.ex.width[0]), float(sky.ex.height[0])
    true_xy = _predict(ctx, sky.inj_states, sky.t0, n_exp, device)
    cover = ((true_xy[..., 0] >= -0.5) & (true_xy[..., 0] < W - 0.5) &
             (true_xy[..., 1] >= -0.5) & (true_xy[..., 1] < H - 0.5))
    cand = np.asarray(cand, np.int64)
    out = np.full(len(cand), np.inf)                 # no injected asteroid: never a match
    has = np.flatnonzero(cand // fam < len(sky.inj_states))
    for s in range(0, len(has), chunk):
        sel = has[s:s + chunk]
        c = cand[sel]
        f = torch.as_tensor(c // fam, device=device)
        xy = _predict(ctx, sky.states[c], sky.t0, n_exp, device)
        d2 = ((xy - true_xy[f]) ** 2).sum(-1)
        cv = cover[f]
        rms = torch.sqrt(torch.where(cv, d2, torch.zeros_like(d2)).sum(1) / cv.sum(1).clamp(min=1))
        out[sel] = rms.cpu().numpy()
    return out


def fpr_at_object_recall(score, match, obj, n_obj, recall):
    """Threshold and false-positive rate of a score on a candidate list: the
    highest threshold at which ``recall`` of the n_obj injected objects have a
    matching entry (match, obj: its object) scoring at least the threshold;
    the FPR is the fraction of non-matching entries at or above it."""
    score = np.asarray(score, np.float64)
    best = np.full(n_obj, -np.inf)
    np.maximum.at(best, np.asarray(obj)[match], score[match])
    k = int(math.ceil(recall * n_obj))
    thr = float(np.sort(best)[::-1][k - 1])
    neg = score[~match]
    return (float(np.mean(neg >= thr)) if len(neg) else None), thr


def make_survey_set(ctx, seed, device, *, n_true=1000, fam_size=512, snr_range=(0.3, 3.0), nu_min=5.0,
                    match_px=2.0, max_pos_per_obj=32, size=4096, n_exp=200):
    """Stamps from an MBA-like survey: the cadence, chips, PSF and noise of
    the MBA workload, with candidate families (each asteroid's true state and
    jittered neighbours).  Positives: orbits with nu >= nu_min whose track
    stays within match_px RMS of their asteroid's (at most max_pos_per_obj
    per asteroid, drawn at random); negatives: as many orbits with nu >=
    nu_min that do not, i.e. tracks that share only part of an asteroid's
    path, and noise peaks.  Returns (stamps_bf16, labels, kind: 0 positive,
    4 negative, nu)."""
    import torch
    sky = synth.mba_sky(n_exp=n_exp, size=size, n_true=n_true, fam_size=fam_size, seed=seed,
                        snr_range=snr_range, scale_arcsec=10.5 * 4096 / size)
    imgs = synth.noise_images_torch(sky.ex, sky.seed, device)
    torch.cuda.synchronize(device)
    ndt.load_exposures(ctx, sky.ex, imgs, plane_dtype="f32")
    pos = _predict(ctx, sky.inj_states, sky.t0, sky.ex.n, device)
    synth.render_sources_torch(imgs, pos, sky.inj_flux, sky.ex.sigma)
    torch.cuda.synchronize(device)
    ndt.load_exposures(ctx, sky.ex, imgs, plane_dtype="bf16")
    del imgs
    n = len(sky.states)
    st = torch.from_numpy(np.ascontiguousarray(sky.states.T)).to(device)
    nu = torch.empty(n, device=device)
    torch.cuda.synchronize(device)
    ndt.stack_orbits(ctx, st, sky.t0, n, snr=nu)
    nu = nu.cpu().numpy()
    cand = np.flatnonzero(nu >= nu_min)
    match = track_rms(ctx, sky, cand, device) < match_px
    rng = np.random.default_rng(seed + 17)
    pos_idx = []
    obj = cand // fam_size
    for o in np.unique(obj[match]):
        m = cand[match & (obj == o)]
        pos_idx.append(rng.choice(m, min(len(m), max_pos_per_obj), replace=False))
    pos_idx = np.concatenate(pos_idx) if pos_idx else np.zeros(0, np.int64)
    negs = cand[~match]
    neg_idx = rng.choice(negs, min(len(negs), len(pos_idx)), replace=False)
    sel = np.concatenate([pos_idx, neg_idx])
    kind = np.concatenate([np.zeros(len(pos_idx)), np.full(len(neg_idx), 4)]).astype(np.int64)
    x, c0, _ = _stamps(ctx, sky.states[sel], sky.t0, device)
    y = torch.as_tensor((kind == 0).astype(np.float32), device=device)
    return x, y, kind, nu[sel]
