"""GPU parity of the iterative-MAD noise estimate (ndt_noise_mad and the
variance <= 0 path of ndt_load_exposures) against oracle/mad.py: bit-exact,
since every deciding quantity is an FP32 operation or an exact order
statistic."""
import numpy as np
import pytest
import torch

from oracle import mad as M
from paper_2503_08854_gb300 import ndt, synth

from _gpu_helpers import Gpu

pytestmark = pytest.mark.gpu


@pytest.fixture
def gpu():
    g = Gpu()
    yield g
    g.close()


def _images():
    rng = np.random.default_rng(0)
    out = []
    # noise with bright sources and deep holes, several sizes (ragged chunks)
    for n, s, mu in [(512 * 512, 1.0, 0.0), (1000 * 1001, 2.5, 7.0), (70_001, 0.3, -2.0)]:
        x = (rng.normal(size=n) * s + mu).astype(np.float32)
        idx = rng.choice(n, n // 25, replace=False)
        x[idx[: n // 40]] += rng.uniform(20, 500, n // 40).astype(np.float32)
        x[idx[n // 40:]] -= 60.0
        out.append(x)
    out.append(np.array([1, 2, 3, 4, 100], np.float32))           # the hand-worked case
    out.append(np.array([5.5], np.float32))                       # one pixel
    out.append(np.full(4096, 3.25, np.float32))                   # constant: sigma 0
    out.append(np.array([-0.0, 0.0, 1.0, -1.0, 2.0, 0.5], np.float32))
    out.append((np.random.default_rng(9).integers(-3, 4, 100_000)).astype(np.float32))  # many ties
    # far from zero with infinities: in round 0 the median's bin holds more
    # keys than the selection buffer and is histogrammed again
    x = (np.random.default_rng(3).normal(size=1 << 20) + 100.0).astype(np.float32)
    x[np.random.default_rng(4).choice(x.size, 2000, replace=False)] = np.inf
    out.append(x)
    return out


def _check(med, sig, rnd, imgs):
    for i, x in enumerate(imgs):
        m, s, r = M.iterative_mad(x)
        assert med[i] == m and sig[i] == s and rnd[i] == r, (i, med[i], m, sig[i], s, rnd[i], r)


def test_noise_mad_bit_exact_device(gpu):
    imgs = _images()
    dev = [torch.from_numpy(x).to(gpu.dev) for x in imgs]
    torch.cuda.synchronize()
    med, sig, rnd = ndt.noise_mad(gpu.ctx, dev)
    _check(med, sig, rnd, imgs)


def test_noise_mad_bit_exact_host_and_round_limit(gpu):
    imgs = _images()
    med, sig, rnd = ndt.noise_mad(gpu.ctx, imgs)
    _check(med, sig, rnd, imgs)
    med1, sig1, rnd1 = ndt.noise_mad(gpu.ctx, imgs[:3], max_rounds=1)
    for i in range(3):
        m, s, r = M.iterative_mad(imgs[i], max_rounds=1)
        assert med1[i] == m and sig1[i] == s and rnd1[i] == 1


def test_noise_mad_empty_and_errors(gpu):
    med, sig, rnd = ndt.noise_mad(gpu.ctx, [np.zeros(0, np.float32), np.ones(3, np.float32)])
    assert np.isnan(med[0]) and np.isnan(sig[0]) and med[1] == 1.0 and sig[1] == 0.0
    with pytest.raises(ndt.NdtError):
        ndt.noise_mad(gpu.ctx, [np.ones(3, np.float32)], max_rounds=0)


def test_load_exposures_estimates_missing_variance(gpu):
    """Exposures whose table variance is <= 0 get sigma^2 of the iterative
    MAD: the planes equal those built from that variance given explicitly."""
    sky = synth.grid_sky(n_r=2)
    imgs = synth.noise_images(sky.ex, sky.seed)
    imgs[:, 100:110, 200:210] += 50.0                       # a bright blob
    ex_est = sky.ex.__class__(**{**sky.ex.__dict__, "var": np.where(np.arange(sky.ex.n) % 2 == 0, 0.0, sky.ex.var)})
    sig = np.array([M.iterative_mad(imgs[j])[1] for j in range(sky.ex.n)], np.float32)
    var_exp = np.where(np.arange(sky.ex.n) % 2 == 0, sig.astype(np.float64) ** 2, sky.ex.var)
    ex_given = sky.ex.__class__(**{**sky.ex.__dict__, "var": var_exp})
    H, W = int(sky.ex.height[0]), int(sky.ex.width[0])
    gpu.load(ex_est, imgs)
    a = [gpu.planes(j, H, W) for j in range(sky.ex.n)]
    gpu.load(ex_given, imgs)
    b = [gpu.planes(j, H, W) for j in range(sky.ex.n)]
    for j in range(sky.ex.n):
        np.testing.assert_array_equal(a[j][0], b[j][0])
        np.testing.assert_array_equal(a[j][1], b[j][1])
    assert np.all(np.abs(sig - 1.0) < 0.05)                # unit-variance noise
