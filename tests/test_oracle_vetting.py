"""Pins of the vetting oracle (stamps and CNN; paper sec. 5.2.3 names the
stage, the definitions are in oracle/vetting.py): a library correlation,
central finite differences, closed forms and a separable toy problem."""
import math

import numpy as np
import pytest
import scipy.signal

import oracle as O
from oracle import vetting as V
from paper_2503_08854_gb300 import synth


def test_parameter_count():
    assert V.N_PARAMS == 52929
    theta = V.init_params(0)
    assert theta.shape == (V.N_PARAMS,)
    np.testing.assert_array_equal(V.pack(V.unpack(theta)), theta)


def test_conv_matches_library_correlation():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 3, 21, 21))
    w = rng.normal(size=(4, 3, 5, 5))
    b = rng.normal(size=4)
    y = V.conv2d(x, w, b)
    for bi in range(2):
        for o in range(4):
            ref = b[o] + sum(scipy.signal.correlate(x[bi, c], w[o, c], mode="same") for c in range(3))
            np.testing.assert_allclose(y[bi, o], ref, rtol=1e-12, atol=1e-12)


def test_bce_special_values():
    assert V.bce_with_logits([0.0], [1.0]) == pytest.approx(math.log(2.0), rel=1e-15)
    assert V.bce_with_logits([0.0], [0.0]) == pytest.approx(math.log(2.0), rel=1e-15)
    assert V.bce_with_logits([40.0], [1.0]) < 1e-17
    assert V.bce_with_logits([-40.0], [1.0]) == pytest.approx(40.0, rel=1e-15)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    theta = V.init_params(3)
    theta += rng.normal(scale=0.01, size=theta.shape)     # biases off zero
    x = rng.normal(size=(3, 2, 21, 21))
    y = np.array([1.0, 0.0, 1.0])
    loss, g = V.loss_and_grad(theta, x, y)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in V.SHAPES])
    picks = np.concatenate([rng.integers(offs[i], offs[i + 1], 8) for i in range(len(V.SHAPES))])
    h = 1e-5
    for i in picks:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (V.bce_with_logits(V.forward(tp, x), y) - V.bce_with_logits(V.forward(tm, x), y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(fd), 1e-4), (i, fd, g[i])


def _on_centre_case(n_exp, F=7.0, sigma=1.5, V_=2.0, size=61):
    state = np.array([2.3, 0.9, 0.1, -0.004, 0.010, 0.0005])
    t0 = 60000.0
    mjd = t0 + np.linspace(-5, 5, n_exp)
    obs = synth.observer_position(mjd, t0, 0.4)
    crval = np.zeros((n_exp, 2))
    for j in range(n_exp):
        rho, _ = O.apparent(state, t0, mjd[j], obs[j])
        _, _, _, ra, dec = O.project(rho, [0, 0], [0, 0], [[1, 0], [0, 1]])
        crval[j] = [math.degrees(ra), math.degrees(dec)]
    s = 1.0 / 3600
    c = size // 2
    ex = synth.Exposures(mjd=mjd, obs=obs, crval=crval, crpix=np.tile([float(c), float(c)], (n_exp, 1)),
                         cd=np.tile([[-s, 0], [0, s]], (n_exp, 1, 1)), sigma=np.full(n_exp, sigma),
                         var=np.full(n_exp, V_), width=np.full(n_exp, size, np.int32),
                         height=np.full(n_exp, size, np.int32))
    P = O.psf_kernel(sigma)
    R = P.shape[0] // 2
    imgs = np.zeros((n_exp, size, size), np.float32)
    imgs[:, c - R:c + R + 1, c - R:c + R + 1] = (F * P).astype(np.float32)
    return state, t0, ex, imgs, P


@pytest.mark.parametrize("n_exp", [2, 5])
def test_stamp_closed_forms_on_pixel_centres(n_exp):
    """Noise-free constant-flux source on pixel centres: the stamp centre holds
    the stacked SNR of the orbit and the constant-flux model fits every
    exposure exactly (chi2 = 0, channel 1 = -sqrt((n-1)/2))."""
    state, t0, ex, imgs, P = _on_centre_case(n_exp)
    xy = O.predict(state[None], t0, ex)
    planes = [O.planes(imgs[j], ex.sigma[j], ex.var[j]) for j in range(n_exp)]
    st = V.stamps(xy, planes, ex.width, ex.height)
    ref = O.stack(state[None], t0, ex, images=list(imgs))
    nu = O.snr(ref["Psi"], ref["Phi"], ref["nobs"])[0]
    c = V.STAMP_HALF
    assert st[0, 0, c, c] == pytest.approx(nu, rel=1e-12)
    np.testing.assert_allclose(st[0, 0], st[0, 0][::-1, ::-1], atol=1e-9)   # symmetric PSF
    np.testing.assert_allclose(st[0, 1], -math.sqrt((n_exp - 1) / 2.0), atol=1e-6)


def test_stamp_flags_a_single_exposure_outlier():
    state, t0, ex, imgs, P = _on_centre_case(6, F=0.0)
    c = imgs.shape[1] // 2
    R = P.shape[0] // 2
    imgs[3, c - R:c + R + 1, c - R:c + R + 1] += (200.0 * P).astype(np.float32)   # one-image artefact
    xy = O.predict(state[None], t0, ex)
    planes = [O.planes(imgs[j], ex.sigma[j], ex.var[j]) for j in range(6)]
    st = V.stamps(xy, planes, ex.width, ex.height)
    h = V.STAMP_HALF
    assert st[0, 0, h, h] > 5.0          # the plain stack is fooled
    assert st[0, 1, h, h] > 20.0         # the consistency channel is not


def test_toy_problem_is_learned():
    """Plain gradient descent with the oracle gradients separates a toy set
    (a centred blob versus pure noise) perfectly."""
    rng = np.random.default_rng(2)
    n = 16
    yy, xx = np.mgrid[-10:11, -10:11]
    blob = np.exp(-(xx ** 2 + yy ** 2) / 4.0)
    x = rng.normal(size=(n, 2, 21, 21)) * 0.5
    y = (np.arange(n) % 2).astype(np.float64)
    x[y == 1, 0] += 3.0 * blob
    theta = V.init_params(1)
    loss0 = V.bce_with_logits(V.forward(theta, x), y)
    for _ in range(40):
        loss, g = V.loss_and_grad(theta, x, y)
        theta -= 0.08 * g
    z = V.forward(theta, x)
    assert V.bce_with_logits(z, y) < 0.5 * loss0
    assert np.all((z > 0) == (y == 1))


def test_bf16_rounding_matches_library():
    """The oracle's BF16 rounding (for the scoring variant) equals torch's
    round-to-nearest-even conversion, ties included."""
    import torch
    rng = np.random.default_rng(4)
    a = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-5, 5, 5000),
                        [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -1.0 - 2.0 ** -8, 0.0, 1e-30]])
    ref = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(V.bf16_round(a), ref)


def _perturbed_logits(theta, x, group, d):
    """Logits with one operand group scaled by (1 + d): a weight tensor of a
    layer or the activations entering layer 2 or 3 (built from the pinned
    conv2d, not from forward())."""
    p = V.unpack(theta)
    w = {k: p[k] * (1 + d) if k == group else p[k] for k in ("w1", "w2", "w3")}
    a1 = np.maximum(V.conv2d(x, w["w1"], p["b1"]), 0)
    if group == "a1":
        a1 = a1 * (1 + d)
    a2 = np.maximum(V.conv2d(a1, w["w2"], p["b2"]), 0)
    if group == "a2":
        a2 = a2 * (1 + d)
    a3 = np.maximum(V.conv2d(a2, w["w3"], p["b3"]), 0)
    return a3.mean(axis=(2, 3)) @ p["wl"] + p["bl"][0]


def _bound_case():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(6, 2, 21, 21))
    x[:, 0, 8:13, 8:13] += 2.0
    theta = V.init_params(2) + np.random.default_rng(3).normal(scale=0.02, size=V.N_PARAMS)
    return theta, x


def test_logit_sensitivities_predict_random_operand_roundings():
    """For each rounded operand group, relative perturbations of +-u with
    random signs move the exact logit by sum_i c_i d_i: its RMS over many
    draws matches u sqrt(sum c_i^2) (a dropped, doubled or misplaced
    sensitivity term fails this)."""
    theta, x = _bound_case()
    x = x[:2]
    z, terms, _ = V.logit_sensitivities(theta, x)
    np.testing.assert_allclose(z, V.forward(theta, x), rtol=1e-13)
    rng = np.random.default_rng(7)
    p = V.unpack(theta)
    shapes = {"w1": p["w1"].shape, "w2": p["w2"].shape, "w3": p["w3"].shape,
              "a1": (2, 32, 21, 21), "a2": (2, 32, 21, 21)}
    for group, t in terms.items():
        pred = V.U_BF16 * np.sqrt((t.reshape(2, -1) ** 2).sum(axis=1))
        errs = []
        for _ in range(60):
            d = V.U_BF16 * rng.choice([-1.0, 1.0], size=shapes[group])
            errs.append(_perturbed_logits(theta, x, group, d) - z)
        rms = np.sqrt(np.mean(np.square(errs), axis=0))
        assert np.all(np.abs(rms / pred - 1) < 0.3), (group, rms, pred)


def test_bf16_bound_covers_a_bf16_rounded_network():
    """The network with its weights and hidden activations rounded to BF16
    (one concrete rounding pattern) stays inside the bound, and the bound is
    a small fraction of the logits' spread (not vacuous)."""
    theta, x = _bound_case()
    bound, z = V.bf16_logit_bound(theta, x)
    zb = V.forward(theta, x, bf16_operands=True)
    assert np.all(np.abs(zb - z) <= bound)
    assert np.median(bound) < 0.15 * np.sqrt(np.mean(z ** 2))
