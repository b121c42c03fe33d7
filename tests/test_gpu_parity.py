"""GPU parity: every step of the CUDA path against the FP64 oracle, through the C ABI.

Cases span several 32 x 32 plane tiles with ragged tails, the full plain-method
tiny workload (65,536 orbits x 10 exposures of 512 x 512), both launch forms,
orbit families, host and device pointers, reduced-precision planes, force-free
motion and the degenerate inputs of the method."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_08854_gb300 import ndt, synth

from _gpu_helpers import Gpu, POS_TOL, check_stack, check_topk
from _orbits import mixed_population as _mixed_population

pytestmark = pytest.mark.gpu


@pytest.fixture
def gpu():
    g = Gpu()
    yield g
    g.close()


def _ragged_sky(seed=3, n_exp=6, size=100):
    sky = synth.grid_sky(n_exp=n_exp, size=size, n_r=4, n_v=32, scale_arcsec=1.0, inj_snr=4.0,
                         n_inj=3, seed=seed)
    # per-exposure PSF widths and variances (FP32-representable)
    rng = np.random.default_rng(seed)
    sky.ex.sigma = rng.uniform(1.0, 2.2, n_exp).astype(np.float32).astype(np.float64)
    sky.ex.var = rng.uniform(0.5, 2.0, n_exp).astype(np.float32).astype(np.float64)
    return sky


def _images(sky, inject=True):
    imgs = synth.noise_images(sky.ex, sky.seed)
    if inject:
        xy = O.predict(sky.inj_states, sky.t0, sky.ex)
        synth.render_sources(imgs, xy, sky.inj_flux, sky.ex.sigma)
    return imgs


# ---------------------------------------------------------------- planes ----

@pytest.mark.parametrize("per_pixel_var", [False, True])
def test_planes_match_oracle(gpu, per_pixel_var):
    rng = np.random.default_rng(1)
    sky = _ragged_sky()
    ex = sky.ex.subset([0, 1, 2])
    ex.width = np.array([100, 37, 70], np.int32)
    ex.height = np.array([70, 65, 33], np.int32)
    imgs = [rng.normal(size=(ex.height[j], ex.width[j])).astype(np.float32) for j in range(3)]
    var = [rng.uniform(0.5, 2.0, size=im.shape).astype(np.float32) for im in imgs] \
        if per_pixel_var else None
    d = [torch.from_numpy(im).to(gpu.dev) for im in imgs]
    dv = None if var is None else [torch.from_numpy(v).to(gpu.dev) for v in var]
    torch.cuda.synchronize()
    ndt.load_exposures(gpu.ctx, ex, d, variances=dv)
    for j in range(3):
        psi, phi = gpu.planes(j, ex.height[j], ex.width[j])
        rp, rf = O.planes(imgs[j], ex.sigma[j], var[j] if var is not None else ex.var[j])
        np.testing.assert_allclose(psi, rp, rtol=1e-5, atol=2e-6 * np.abs(rp).max())
        np.testing.assert_allclose(phi, rf, rtol=1e-5, atol=1e-7 * np.abs(rf).max())


@pytest.mark.parametrize("plane", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("wide_psf", [False, True])
def test_planes_both_kernel_forms_match_oracle(gpu, plane, wide_psf):
    """Exposures of one load split between the TMA form (widths a multiple of
    4 px) and the general form (other widths), ragged tiles on both axes, a
    one-row image and a 4-pixel-wide one; PSF windows of R <= 8 or, with
    a wide PSF, up to R = 16 (the other compile-time window)."""
    rng = np.random.default_rng(7)
    sky = _ragged_sky(n_exp=6)
    ex = sky.ex.subset(range(6))
    ex.width = np.array([132, 37, 200, 4, 70, 260], np.int32)
    ex.height = np.array([70, 65, 1, 64, 33, 97], np.int32)
    ex.sigma = np.array([1.3, 1.9, 2.0, 0.6, 1.2, 3.9 if wide_psf else 1.7])
    imgs = [rng.normal(size=(ex.height[j], ex.width[j])).astype(np.float32) for j in range(6)]
    d = [torch.from_numpy(im).to(gpu.dev) for im in imgs]
    torch.cuda.synchronize()
    ndt.load_exposures(gpu.ctx, ex, d, plane_dtype=plane)
    rel = {"f32": 0.0, "bf16": 2.0 ** -8, "f16": 2.0 ** -11}[plane]
    for j in range(6):
        psi, phi = gpu.planes(j, ex.height[j], ex.width[j])
        rp, rf = O.planes(imgs[j], ex.sigma[j], ex.var[j])
        s = np.abs(rp).max() / 16384 if plane == "f16" else 0.0
        tol_psi = rel * np.abs(rp) + s * 2.0 ** -14 + 1e-5 * np.abs(rp) + 2e-6 * np.abs(rp).max()
        tol_phi = rel * np.abs(rf) + 1e-5 * np.abs(rf) + 1e-7 * rf.max()
        assert np.all(np.abs(psi - rp) <= tol_psi), (j, np.abs(psi - rp).max())
        assert np.all(np.abs(phi - rf) <= tol_phi), (j, np.abs(phi - rf).max())


@pytest.mark.parametrize("plane", ["f32", "bf16"])
def test_planes_tma_form_many_strips(gpu, plane):
    """The TMA form over 1,156 strips of 20 exposures at once (more CTAs than
    the GPU holds), with different PSF widths, image sizes (ragged strips
    and tiles) and variances per exposure: every plane matches the
    oracle's."""
    rng = np.random.default_rng(11)
    sky = _ragged_sky(n_exp=20)
    ex = sky.ex.subset(range(20))
    ex.width = np.array([1024, 260, 768, 128, 1028] * 4, np.int32)
    ex.height = np.array([512, 200, 420, 330, 140] * 4, np.int32)
    ex.sigma = rng.uniform(1.2, 2.0, 20)
    ex.var = rng.uniform(0.5, 2.0, 20)
    imgs = [rng.normal(size=(ex.height[j], ex.width[j])).astype(np.float32) for j in range(20)]
    d = [torch.from_numpy(im).to(gpu.dev) for im in imgs]
    torch.cuda.synchronize()
    ndt.load_exposures(gpu.ctx, ex, d, plane_dtype=plane)
    rel = {"f32": 0.0, "bf16": 2.0 ** -8}[plane]
    for j in range(20):
        psi, phi = gpu.planes(j, ex.height[j], ex.width[j])
        rp, rf = O.planes(imgs[j], ex.sigma[j], ex.var[j])
        tol_psi = rel * np.abs(rp) + 1e-5 * np.abs(rp) + 2e-6 * np.abs(rp).max()
        tol_phi = rel * np.abs(rf) + 1e-5 * np.abs(rf) + 1e-7 * rf.max()
        assert np.all(np.abs(psi - rp) <= tol_psi), (j, np.abs(psi - rp).max())
        assert np.all(np.abs(phi - rf) <= tol_phi), (j, np.abs(phi - rf).max())


@pytest.mark.parametrize("plane", ["bf16", "f16"])
def test_reduced_precision_planes_error_bound(gpu, plane):
    """RNE of value/scale: |error| <= half an ulp of the stored format (2^-9
    relative for BF16, 2^-12 for FP16 normals) plus the FP32 plane error."""
    sky = _ragged_sky()
    imgs = _images(sky)
    gpu.load(sky.ex, imgs, plane=plane)
    rel = 2.0 ** -8 if plane == "bf16" else 2.0 ** -11
    for j in range(sky.ex.n):
        psi, phi = gpu.planes(j, 100, 100)
        rp, rf = O.planes(imgs[j], sky.ex.sigma[j], sky.ex.var[j])
        s = np.abs(rp).max() / 16384
        assert np.all(np.abs(psi - rp) <= rel * np.abs(rp) + s * 2.0 ** -14 + 2e-6 * np.abs(rp).max())
        assert np.all(np.abs(phi - rf) <= rel * np.abs(rf) + 1e-7 * rf.max())


# ------------------------------------------------------------- positions ----

@pytest.mark.parametrize("df", [False, True])
def test_positions_match_oracle_plain_workload(gpu, df):
    ndt.set_df_state(gpu.ctx, df)
    sky = synth.grid_sky()
    imgs = np.zeros((sky.ex.n, 512, 512), np.float32)
    gpu.load(sky.ex, imgs)
    sel = np.random.default_rng(0).choice(len(sky.states), 4096, replace=False)
    st = sky.states[sel]
    xy = gpu.predict(st, sky.t0, sky.ex.n)
    ref = O.predict(st, sky.t0, sky.ex, nthreads=0)
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(xy))
    err = np.abs(xy[fin] - ref[fin]).max()
    assert err <= POS_TOL, f"max position error {err:.3g} px"


@pytest.mark.parametrize("df", [False, True])
def test_positions_mixed_orbit_classes_long_span(gpu, df):
    """NEO, main-belt, Kuiper-belt and hyperbolic orbits over a year: each
    exposure points at one object, so every object is near the centre of
    several exposures; all finite positions within 1e4 px are compared."""
    ndt.set_df_state(gpu.ctx, df)
    rng = np.random.default_rng(7)
    n_obj, n_exp = 24, 48
    states = _mixed_population(rng, n_obj)
    t0 = 60200.0
    mjd = np.sort(t0 + rng.uniform(-180, 180, n_exp))
    obs = synth.observer_position(mjd, t0, 0.3)
    crval = np.zeros((n_exp, 2))
    for j in range(n_exp):
        rho, _ = O.apparent(states[j % n_obj], t0, mjd[j], obs[j])
        _, _, _, ra, dec = O.project(rho, [0, 0], [0, 0], [[1, 0], [0, 1]])
        crval[j] = [math.degrees(ra) + rng.normal() * 1e-3, math.degrees(dec) + rng.normal() * 1e-3]
    s = 1.0 / 3600
    ex = synth.Exposures(mjd=mjd, obs=obs, crval=crval, crpix=np.tile([1024.0, 1024.0], (n_exp, 1)),
                         cd=np.tile([[-s, 0], [0, s]], (n_exp, 1, 1)), sigma=np.full(n_exp, 1.5),
                         var=np.ones(n_exp), width=np.full(n_exp, 64, np.int32),
                         height=np.full(n_exp, 64, np.int32))
    gpu.load(ex, np.zeros((n_exp, 64, 64), np.float32))
    xy = gpu.predict(states, t0, n_exp)
    ref = O.predict(states, t0, ex)
    near = np.isfinite(ref).all(-1) & (np.abs(ref - 1024).max(-1) < 1e4)
    assert near.sum() >= n_exp
    err = np.abs(xy[near] - ref[near]).max()
    assert err <= POS_TOL, f"max position error {err:.3g} px"
    assert gpu.stats()["kepler_failures"] == 0


# Position bound of the chained-step test: the FP64 state's, and the
# double-float state's (rounding unit 2^-48 instead of 2^-53: over n = 300
# steps ~sqrt(n) 2^-48 (|r| + T |v|) ~ 1e-13 AU of noise, 1e-6 px at 0.2
# arcsec for an object 0.1 AU away, taken with a factor of 10).
CHAINED_TOL = {False: 1e-6, True: 1e-5}


@pytest.mark.parametrize("gap_h", [0.25, 2.5])
@pytest.mark.parametrize("df", [False, True])
@pytest.mark.parametrize("light_time", [False, True])
def test_chained_steps_track_the_oracle_tightly(gpu, light_time, df, gap_h):
    """Hundreds of chained steps of all three kinds: 90 s between the two
    snaps of a visit (the shortest-step series), 15 min or 2.5 h between five
    visits of a night (the f/g series; at 2.5 h the double-float state's
    longer series for main-belt and farther orbits, the universal-variable
    step for NEOs) and a day between nights (the universal-variable step),
    for 30 nights.  NEO, main-belt, Kuiper-belt and hyperbolic positions at
    0.2 arcsec pixels stay within 1e-6 px (FP64 state) or 1e-5 px (double-
    float state) of the oracle's direct FP64 propagation from the epoch,
    without light time and with it (whose light time the oracle iterates to
    convergence).  A term of the series, of 1/|r| or of the light time
    carried at FP32 precision where more is needed shows up here as errors of
    1e-6 px and more (an FP32 light time alone gives ~5e-6 px)."""
    rng = np.random.default_rng(11)
    n_obj = 24
    states = _mixed_population(rng, n_obj)
    nights = np.arange(30.0)
    visit = np.repeat(np.arange(5), 2) * (gap_h / 24.0) + np.tile([0.0, 90.0 / 86400.0], 5)
    mjd = (60200.0 + nights[:, None] + 0.1 + visit[None, :]
           + rng.uniform(0, 20.0 / 86400.0, (30, 1))).ravel()
    n_exp = mjd.size
    t0 = 60215.0
    obs = synth.observer_position(mjd, t0, 0.3)
    crval = np.zeros((n_exp, 2))
    for j in range(n_exp):
        rho, _ = O.apparent(states[j % n_obj], t0, mjd[j], obs[j])
        _, _, _, ra, dec = O.project(rho, [0, 0], [0, 0], [[1, 0], [0, 1]])
        crval[j] = [math.degrees(ra), math.degrees(dec)]
    s = 0.2 / 3600
    ex = synth.Exposures(mjd=mjd, obs=obs, crval=crval, crpix=np.tile([2048.0, 2048.0], (n_exp, 1)),
                         cd=np.tile([[-s, 0], [0, s]], (n_exp, 1, 1)), sigma=np.full(n_exp, 1.5),
                         var=np.ones(n_exp), width=np.full(n_exp, 64, np.int32),
                         height=np.full(n_exp, 64, np.int32))
    if light_time:
        ref = O.predict(states, t0, ex)
    else:
        ndt.set_constants(gpu.ctx, O.gm_sun(), 0.0, O.obliquity())
        # the oracle has no switch for light time: at c = 1e30 AU/day its light
        # time is 1e-30 day, and t_obs - tau rounds to t_obs exactly
        ref = O.predict(states, t0, ex, c=1e30)
    gpu.load(ex, np.zeros((n_exp, 64, 64), np.float32))
    ndt.set_df_state(gpu.ctx, df)
    xy = gpu.predict(states, t0, n_exp)
    near = np.isfinite(ref).all(-1) & (np.abs(ref - 2048).max(-1) < 1e4)
    assert near.sum() >= n_exp
    err = np.abs(xy[near] - ref[near]).max()
    print(f"light time {light_time}, df {df}, gap {gap_h} h: max position error {err:.3g} px "
          f"over {int(near.sum())} positions")
    assert err <= CHAINED_TOL[df], f"max position error {err:.3g} px"
    assert gpu.stats()["kepler_failures"] == 0


@pytest.mark.parametrize("df", [False, True])
def test_force_free_motion_matches_oracle(gpu, df):
    ndt.set_df_state(gpu.ctx, df)
    sky = _ragged_sky()
    imgs = _images(sky, inject=False)
    ndt.set_constants(gpu.ctx, 0.0, O.c_light(), O.obliquity())
    gpu.load(sky.ex, imgs)
    st = sky.states[::7]
    xy = gpu.predict(st, sky.t0, sky.ex.n)
    ref = O.predict(st, sky.t0, sky.ex, mu=0.0)
    fin = np.isfinite(ref)
    assert np.abs(xy[fin] - ref[fin]).max() <= POS_TOL
    out = gpu.stack(st, sky.t0)
    check_stack(out, O.stack(st, sky.t0, sky.ex, images=list(imgs), mu=0.0))


# ------------------------------------------------------------------ stack ----

@pytest.mark.parametrize("df", [False, True])
@pytest.mark.parametrize("plane", ["f32"])
def test_stack_ragged_matches_oracle(gpu, plane, df):
    ndt.set_df_state(gpu.ctx, df)
    sky = _ragged_sky()
    imgs = _images(sky)
    gpu.load(sky.ex, imgs, plane=plane)
    out = gpu.stack(sky.states, sky.t0)
    ref = O.stack(sky.states, sky.t0, sky.ex, images=list(imgs))
    rep = check_stack(out, ref)
    assert rep["n_finite"] > 100
    st = gpu.stats()
    assert st["kepler_failures"] == 0
    assert st["valid_samples"] == int(out["nobs"].sum())
    assert st["samples"] == len(sky.states) * sky.ex.n


def test_plain_workload_stack_and_top100(gpu):
    """The tiny plain-method workload at its full size: 65,536 grid orbits,
    10 exposures of 512 x 512, 5 injected sources, top-100."""
    sky = synth.grid_sky()
    imgs = _images(sky)
    gpu.load(sky.ex, imgs)
    out = gpu.stack(sky.states, sky.t0)
    pl = [O.planes(imgs[j], sky.ex.sigma[j], sky.ex.var[j]) for j in range(sky.ex.n)]
    ref = O.stack(sky.states, sky.t0, sky.ex, planes=([p[0] for p in pl], [p[1] for p in pl]))
    check_stack(out, ref)
    idx, val = gpu.topk(100)
    nu = O.snr(ref["Psi"], ref["Phi"], ref["nobs"])
    check_topk(idx, val, nu, ref["n_amb"] > 0, 100)
    assert set(sky.inj_orbit.tolist()) <= set(idx.tolist())
    # a k larger than the number of finite nu: the tail is the lowest-index -inf orbits
    idx2, val2 = gpu.topk(8192)
    check_topk(idx2, val2, nu, ref["n_amb"] > 0, 8192)
    # large k (multi-block radix sort), up to every orbit of the batch
    for k in (20000, len(sky.states)):
        idx3, val3 = gpu.topk(k)
        check_topk(idx3, val3, nu, ref["n_amb"] > 0, k)


def test_fp64_geometry_form_matches_oracle(gpu):
    """The plain form with FP64 light time and TAN projection (the reference-
    precision variant) on the tiny workload: element-wise parity with the
    oracle, and the same in-bounds samples as the double-float default."""
    sky = synth.grid_sky()
    imgs = _images(sky)
    gpu.load(sky.ex, imgs)
    pl = [O.planes(imgs[j], sky.ex.sigma[j], sky.ex.var[j]) for j in range(sky.ex.n)]
    ref = O.stack(sky.states, sky.t0, sky.ex, planes=([p[0] for p in pl], [p[1] for p in pl]))
    ndt.set_df_state(gpu.ctx, False)     # the FP64 geometry goes with the FP64 state
    ndt.set_fp64_geometry(gpu.ctx, True)
    out64 = gpu.stack(sky.states, sky.t0)
    check_stack(out64, ref)
    ndt.set_fp64_geometry(gpu.ctx, False)
    out = gpu.stack(sky.states, sky.t0)
    clean = ref["n_amb"] == 0
    assert np.array_equal(out64["nobs"][clean], out["nobs"][clean])


def _families(rng, n_orb, n_exp, n_fam):
    cuts = np.sort(rng.choice(np.arange(1, n_orb), n_fam - 1, replace=False))
    fo = np.concatenate([[0], cuts, [n_orb]]).astype(np.int64)
    lists = []
    for f in range(n_fam):
        m = int(rng.integers(1, n_exp + 1))
        lists.append(rng.choice(n_exp, m, replace=False).astype(np.int32))   # unsorted on purpose
    fe = np.concatenate([[0], np.cumsum([len(x) for x in lists])]).astype(np.int64)
    return fo, fe, np.concatenate(lists).astype(np.int32)


@pytest.mark.parametrize("df", [False, True])
@pytest.mark.parametrize("mode", ["plain", "persistent", "graph"])
def test_families_match_oracle(gpu, mode, df):
    ndt.set_df_state(gpu.ctx, df)
    sky = _ragged_sky(n_exp=9)
    imgs = _images(sky)
    gpu.load(sky.ex, imgs)
    fam = _families(np.random.default_rng(2), len(sky.states), sky.ex.n, 37)
    if mode != "plain":
        ndt.set_launch(gpu.ctx, ndt.LAUNCH_PERSISTENT, 64, 8, use_graph=(mode == "graph"))
    ref = O.stack(sky.states, sky.t0, sky.ex, images=list(imgs), families=fam)
    for rep in range(2 if mode == "graph" else 1):   # the second graph call replays
        out = gpu.stack(sky.states, sky.t0, families=fam)
        check_stack(out, ref)
    assert gpu.stats()["samples"] == int(sum((fam[0][f + 1] - fam[0][f]) * (fam[1][f + 1] - fam[1][f])
                                             for f in range(len(fam[0]) - 1)))


@pytest.mark.parametrize("df", [False, True])
@pytest.mark.parametrize("ot", [32, 64, 128])
@pytest.mark.parametrize("et", [8, 16, 32])
def test_every_persistent_tile_shape(gpu, ot, et, df):
    ndt.set_df_state(gpu.ctx, df)
    sky = _ragged_sky(n_exp=11)
    imgs = _images(sky)
    gpu.load(sky.ex, imgs)
    ndt.set_launch(gpu.ctx, ndt.LAUNCH_PERSISTENT, ot, et)
    out = gpu.stack(sky.states, sky.t0)
    check_stack(out, O.stack(sky.states, sky.t0, sky.ex, images=list(imgs)))


@pytest.mark.parametrize("df", [False, True])
def test_offchip_test_changes_no_result(gpu, df):
    """The persistent form's off-chip test removes FP64 work without changing
    what is stacked: on an MBA-shaped sky whose chips cover 60-100 % of the
    population, the sums with the test on equal those with it off, the
    plain form's sample count and the oracle's sums, and samples were
    skipped."""
    sky = synth.mba_sky(n_exp=40, nights=6, size=512, n_true=24, fam_size=256,
                        scale_arcsec=10.5 * 4096 / 512)
    imgs = synth.noise_images(sky.ex, sky.seed)
    gpu.load(sky.ex, imgs)
    ndt.set_df_state(gpu.ctx, df)
    plain = gpu.stack(sky.states, sky.t0)
    valid_plain = gpu.stats()["valid_samples"]
    ndt.set_launch(gpu.ctx, ndt.LAUNCH_PERSISTENT, 64, 16)
    ndt.set_offchip_test(gpu.ctx, False)
    off = gpu.stack(sky.states, sky.t0)
    assert gpu.stats()["offchip_skipped"] == 0
    ndt.set_offchip_test(gpu.ctx, True)
    on = gpu.stack(sky.states, sky.t0)
    st = gpu.stats()
    assert st["valid_samples"] == valid_plain < st["samples"]
    assert st["offchip_skipped"] >= 0.05 * st["samples"], st
    assert st["offchip_skipped"] <= st["samples"] - st["valid_samples"]
    for other in (off, plain):
        assert np.array_equal(on["nobs"], other["nobs"])
        scale = np.sqrt(np.maximum(on["phi"], 1e-30))
        assert np.all(np.abs(on["psi"] - other["psi"]) <= 1e-6 * np.maximum(1.0, scale))
        assert np.allclose(on["phi"], other["phi"], rtol=1e-6, atol=0)
    sel = np.sort(np.random.default_rng(3).choice(len(sky.states), 256, replace=False))
    ref = O.stack(sky.states[sel], sky.t0, sky.ex, images=list(imgs))
    check_stack({k: v[sel] for k, v in on.items()}, ref)


def test_host_pointers_give_device_results(gpu):
    sky = _ragged_sky()
    imgs = _images(sky)
    gpu.load(sky.ex, imgs, host=True)
    h = gpu.stack(sky.states, sky.t0, host=True)
    hi, hv = gpu.topk(50, host=True)
    gpu.load(sky.ex, imgs, host=False)
    d = gpu.stack(sky.states, sky.t0)
    di, dv = gpu.topk(50)
    for k in h:
        np.testing.assert_array_equal(h[k], d[k])
    np.testing.assert_array_equal(hi, di)
    np.testing.assert_array_equal(hv, dv)


def test_per_pixel_variance_stack(gpu):
    sky = _ragged_sky()
    imgs = _images(sky)
    var = np.random.default_rng(4).uniform(0.5, 2.0, imgs.shape).astype(np.float32)
    gpu.load(sky.ex, imgs, variances=var)
    out = gpu.stack(sky.states, sky.t0)
    check_stack(out, O.stack(sky.states, sky.t0, sky.ex, images=list(imgs), var_planes=list(var)))


@pytest.mark.parametrize("plane", ["bf16", "f16"])
def test_reduced_precision_stack_error(gpu, plane):
    """Reduced-precision planes: nu error against the FP64 oracle stays within
    the storage format's rounding, and the injected sources stay on top."""
    sky = _ragged_sky()
    imgs = _images(sky)
    gpu.load(sky.ex, imgs, plane=plane)
    out = gpu.stack(sky.states, sky.t0)
    ref = O.stack(sky.states, sky.t0, sky.ex, images=list(imgs))
    nu = O.snr(ref["Psi"], ref["Phi"], ref["nobs"])
    clean = (ref["n_amb"] == 0) & np.isfinite(nu)
    err = np.abs(out["snr"][clean] - nu[clean]) / np.maximum(1.0, np.abs(nu[clean]))
    # each stored value carries <= u relative rounding (u = 2^-8 BF16, 2^-11
    # FP16): |d nu| <= u (sum|psi_j| / sqrt(Phi) + |nu| / 2) <= u (sqrt(n) + 1.5)
    u = 2.0 ** -8 if plane == "bf16" else 2.0 ** -11
    bound = u * (np.sqrt(sky.ex.n) + 1.5)
    assert err.max() <= bound, f"{plane}: max SNR error {err.max():.3g}"
    idx, _ = gpu.topk(10)
    assert set(sky.inj_orbit.tolist()) <= set(idx.tolist())


# ------------------------------------------------------------ edge cases ----

def test_degenerate_inputs(gpu):
    sky = _ragged_sky()
    imgs = _images(sky, inject=False)
    with pytest.raises(ndt.NdtError) as e:
        ndt.stack_orbits(gpu.ctx, gpu.soa(sky.states), sky.t0, len(sky.states))
    assert e.value.status == ndt.ESTATE
    gpu.load(sky.ex, imgs)
    # empty batch
    ndt.stack_orbits(gpu.ctx, gpu.soa(sky.states[:1]), sky.t0, 0)
    with pytest.raises(ndt.NdtError) as e:
        gpu.topk(5)
    assert e.value.status == ndt.ESTATE
    # an orbit that never lands in an image: nu = -inf, n_obs = 0
    far = sky.states[:1].copy()
    far[0, :3] *= -1.0
    out = gpu.stack(far, sky.t0)
    assert out["nobs"][0] == 0 and out["snr"][0] == -np.inf
    idx, val = gpu.topk(3)
    assert list(idx) == [0] and val[0] == -np.inf
    # min_obs above every count: all -inf, ranking by index
    out = gpu.stack(sky.states[:50], sky.t0, min_obs=1000)
    assert np.all(out["snr"] == -np.inf)
    idx, _ = gpu.topk(7)
    assert list(idx) == list(range(7))
    # bad arguments
    bad = sky.ex.subset([0])
    bad.sigma = np.array([0.0])
    with pytest.raises(ndt.NdtError) as e:
        gpu.load(bad, imgs[:1])
    assert e.value.status == ndt.EINVAL
    with pytest.raises(ndt.NdtError):
        ndt.set_launch(gpu.ctx, ndt.LAUNCH_PERSISTENT, 48, 8)
    fo = np.array([0, 10], np.int64)   # does not span the batch
    with pytest.raises(ndt.NdtError) as e:
        gpu.stack(sky.states[:20], sky.t0, families=(fo, np.array([0, 1], np.int64),
                                                     np.array([0], np.int32)))
    assert e.value.status == ndt.EINVAL


def test_single_exposure_single_orbit(gpu):
    sky = _ragged_sky()
    imgs = _images(sky)
    ex = sky.ex.subset([2])
    gpu.load(ex, imgs[2:3])
    st = sky.states[sky.inj_orbit[:1]]
    out = gpu.stack(st, sky.t0)
    check_stack(out, O.stack(st, sky.t0, ex, images=[imgs[2]]))
