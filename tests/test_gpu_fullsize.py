"""Parity at full workload sizes, in the launch forms the benchmark times:
every orbit is stacked on the GPU, a random sample of orbits is recomputed by
the oracle (planes evaluated at the gathered pixels from the same images),
and the precision variant is reported against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_08854_gb300 import ndt, synth

from _gpu_helpers import Gpu, POS_TOL, check_stack

pytestmark = pytest.mark.gpu


@pytest.fixture
def gpu():
    g = Gpu()
    yield g
    g.close()


def _device_sky(gpu, sky):
    """Noise drawn on the device, sources rendered at oracle positions."""
    imgs = synth.noise_images_torch(sky.ex, sky.seed, gpu.dev)
    if np.any(sky.inj_flux > 0):
        xy = O.predict(sky.inj_states, sky.t0, sky.ex, nthreads=0)
        synth.render_sources_torch(imgs, xy, sky.inj_flux, sky.ex.sigma)
    torch.cuda.synchronize()
    return imgs


def _stack_all(gpu, sky, imgs, plane, mode, families=None, df=False):
    ndt.load_exposures(gpu.ctx, sky.ex, imgs, plane_dtype=plane)
    ndt.set_df_state(gpu.ctx, df)
    if mode == "persistent":
        ndt.set_launch(gpu.ctx, ndt.LAUNCH_PERSISTENT, 64, 16, use_graph=True)
    else:
        ndt.set_launch(gpu.ctx, ndt.LAUNCH_PLAIN)
    n = len(sky.states)
    st = torch.from_numpy(np.ascontiguousarray(sky.states.T)).to(gpu.dev)
    out = dict(psi=torch.empty(n, device=gpu.dev), phi=torch.empty(n, device=gpu.dev),
               nobs=torch.empty(n, dtype=torch.int32, device=gpu.dev),
               snr=torch.empty(n, device=gpu.dev))
    fam = None
    if families is not None:
        fam = tuple(torch.from_numpy(np.ascontiguousarray(x)).to(gpu.dev) for x in families)
    torch.cuda.synchronize()
    ndt.stack_orbits(gpu.ctx, st, sky.t0, n, families=fam, psi_sum=out["psi"], phi_sum=out["phi"],
                     nobs=out["nobs"], snr=out["snr"])
    ndt.synchronize(gpu.ctx)
    assert gpu.stats()["kepler_failures"] == 0
    return out


def _sampled(out, sel):
    return {k: v[torch.as_tensor(sel, device=v.device)].cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("form", [("f32", "plain", False), ("bf16", "persistent", False),
                                  ("bf16", "persistent", True)])
def test_mba_full_size_sampled(gpu, form):
    """200 exposures of 4096^2, 16.4 M orbits, as the benchmark runs it (the
    chosen form: persistent, BF16 planes, double-float state)."""
    plane, mode, df = form
    sky = synth.mba_sky()
    imgs = _device_sky(gpu, sky)
    out = _stack_all(gpu, sky, imgs, plane, mode, df=df)
    sel = np.sort(np.random.default_rng(1).choice(len(sky.states), 256, replace=False))
    sel = np.concatenate([sky.inj_orbit[:16], sel])
    host = imgs.cpu().numpy()
    ref = O.stack(sky.states[sel], sky.t0, sky.ex, images=[host[j] for j in range(sky.ex.n)])
    g = _sampled(out, sel)
    if plane == "f32":
        check_stack(g, ref)
    else:
        nu = O.snr(ref["Psi"], ref["Phi"], ref["nobs"])
        ok = (ref["n_amb"] == 0) & np.isfinite(nu)
        assert np.array_equal(g["nobs"][ref["n_amb"] == 0], ref["nobs"][ref["n_amb"] == 0])
        err = np.abs(g["snr"][ok] - nu[ok]) / np.maximum(1.0, np.abs(nu[ok]))
        assert err.max() <= 2.0 ** -8 * (np.sqrt(sky.ex.n) + 1.5), err.max()
    # positions of the sampled orbits through the same device code
    xy = torch.empty(len(sel) * sky.ex.n * 2, dtype=torch.float64, device=gpu.dev)
    st = torch.from_numpy(np.ascontiguousarray(sky.states[sel].T)).to(gpu.dev)
    torch.cuda.synchronize()
    ndt.predict_positions(gpu.ctx, st, sky.t0, len(sel), xy)
    xy = xy.cpu().numpy().reshape(len(sel), sky.ex.n, 2)
    rx = O.predict(sky.states[sel], sky.t0, sky.ex)
    fin = np.isfinite(rx)
    assert np.abs(xy[fin] - rx[fin]).max() <= POS_TOL


@pytest.mark.parametrize("df", [False, True])
@pytest.mark.parametrize("workload", ["mba", "batched"])
def test_full_size_forms_count_the_same_samples(gpu, workload, df):
    """Every orbit of the full workload: the plain form (every sample computed,
    FP64 state) and the persistent form (off-chip test on, BF16 planes, FP64
    or double-float state) find the same in-bounds exposures for every orbit,
    while the persistent form skips the FP64 work of a large share of the
    off-chip samples.  With the double-float state a sample whose position
    lies within its ~1e-9 px (at these pixel scales) of a pixel edge may fall
    on the other side: at most one sample per orbit, on at most 1e-5 of the
    orbits."""
    sky = synth.mba_sky() if workload == "mba" else synth.batched_sky()
    fam = None if workload == "mba" else sky.families
    imgs = _device_sky(gpu, sky)
    plain = _stack_all(gpu, sky, imgs, "f32", "plain", families=fam)
    st_plain = gpu.stats()
    pers = _stack_all(gpu, sky, imgs, "bf16", "persistent", families=fam, df=df)
    st = gpu.stats()
    if df:
        d = (pers["nobs"] - plain["nobs"]).abs()
        assert int(d.max()) <= 1
        assert int((d > 0).sum()) <= 1e-5 * len(sky.states)
        assert abs(st["valid_samples"] - st_plain["valid_samples"]) <= 1e-5 * len(sky.states)
    else:
        assert st["valid_samples"] == st_plain["valid_samples"]
        assert torch.equal(plain["nobs"], pers["nobs"])
    off_chip = st["samples"] - st["valid_samples"]
    assert st["offchip_skipped"] <= off_chip
    assert st["offchip_skipped"] >= 0.5 * off_chip, (st["offchip_skipped"], off_chip)


@pytest.mark.parametrize("df", [False, True])
def test_batched_uneven_full_size_sampled(gpu, df):
    """4,096 families x 16,384 orbits (NEO, MBA, KBO), 20-400 of 400 exposures
    of 2048^2 each, FP32 planes, persistent work queue under a CUDA graph,
    FP64 or double-float state."""
    sky = synth.batched_sky()
    imgs = _device_sky(gpu, sky)
    out = _stack_all(gpu, sky, imgs, "f32", "persistent", families=sky.families, df=df)
    fo, fe, fi = sky.families
    rng = np.random.default_rng(2)
    sel = np.sort(rng.choice(len(sky.states), 256, replace=False))
    fam_of = np.searchsorted(fo, sel, side="right") - 1
    lists = [fi[fe[f]:fe[f + 1]] for f in fam_of]
    mfo = np.arange(len(sel) + 1, dtype=np.int64)
    mfe = np.concatenate([[0], np.cumsum([len(x) for x in lists])]).astype(np.int64)
    host = imgs.cpu().numpy()
    ref = O.stack(sky.states[sel], sky.t0, sky.ex, images=[host[j] for j in range(sky.ex.n)],
                  families=(mfo, mfe, np.concatenate(lists)))
    check_stack(_sampled(out, sel), ref)
    assert gpu.stats()["samples"] == int(np.sum((fo[1:] - fo[:-1]) * (fe[1:] - fe[:-1])))


def test_precision_variant_report(gpu, capsys):
    """The tiny workload refined to 102,400 orbits: BF16/FP16 planes against the
    FP64 oracle (SNR error) and recall of the injected sources against FP32."""
    sky = synth.grid_sky(n_r=25)
    imgs = synth.noise_images(sky.ex, sky.seed)
    xy = O.predict(sky.inj_states, sky.t0, sky.ex)
    synth.render_sources(imgs, xy, sky.inj_flux, sky.ex.sigma)
    pl = [O.planes(imgs[j], sky.ex.sigma[j], sky.ex.var[j]) for j in range(sky.ex.n)]
    ref = O.stack(sky.states, sky.t0, sky.ex, planes=([p[0] for p in pl], [p[1] for p in pl]))
    nu = O.snr(ref["Psi"], ref["Phi"], ref["nobs"])
    ok = (ref["n_amb"] == 0) & np.isfinite(nu)
    report = {}
    for plane in ("f32", "bf16", "f16"):
        gpu.load(sky.ex, imgs, plane=plane)
        out = gpu.stack(sky.states, sky.t0)
        idx, _ = gpu.topk(100)
        err = np.abs(out["snr"][ok] - nu[ok]) / np.maximum(1.0, np.abs(nu[ok]))
        recall = np.isin(sky.inj_orbit, idx).mean()
        report[plane] = (float(err.max()), float(np.median(err)), float(recall))
    with capsys.disabled():
        for k, (mx, md, rc) in report.items():
            print(f"\nprecision {k}: max SNR err {mx:.2e}, median {md:.2e}, recall {rc:.2f}")
    # each stored plane value carries <= u relative rounding error (u = 2^-8
    # BF16, 2^-11 FP16), so |d nu| <= u (sum|psi_j| / sqrt(Phi) + |nu| / 2)
    # <= u (sqrt(n) + 1.5) max(1, |nu|) with n the exposures of the orbit
    n = sky.ex.n
    assert report["f32"][0] <= 1e-5
    assert report["bf16"][0] <= 2.0 ** -8 * (np.sqrt(n) + 1.5)
    assert report["f16"][0] <= 2.0 ** -11 * (np.sqrt(n) + 1.5)
    assert report["bf16"][2] == report["f32"][2] and report["f16"][2] == report["f32"][2]
