"""Pins of the iterative-MAD noise oracle (paper sec. 3) against hand-worked
values, textbook medians and the statistics of normal noise."""
import math

import numpy as np
import pytest

from oracle import mad as M


def test_hand_worked_example():
    """x = [1, 2, 3, 4, 100]: m = 3, |x - m| = [2, 1, 0, 1, 97] -> mad 1, sigma
    1.4826, threshold 4.4478 drops 100; then m = 2 (lower median of 1..4),
    deviations [1, 0, 1, 2] -> mad 1; the third round repeats (2, 1.4826)."""
    m, s, rounds = M.iterative_mad(np.array([1, 2, 3, 4, 100], np.float32))
    assert m == np.float32(2.0) and s == np.float32(1.4826) and rounds == 3


@pytest.mark.parametrize("n", [1, 2, 7, 1000, 1001])
def test_lower_median_against_the_textbook_median(n):
    rng = np.random.default_rng(n)
    v = rng.normal(size=n).astype(np.float32)
    lm = M.lower_median(v)
    if n % 2:
        assert lm == np.median(v)                      # odd: the median itself
    else:
        s = np.sort(v)
        assert lm == s[n // 2 - 1] and lm <= np.median(v) <= s[n // 2]


def test_normal_noise_sigma():
    """For N(mu, s^2) the clipped MAD estimate converges to s times
    Phi^-1(0.5 P(|Z| <= 3)) / Phi^-1(0.75) = 0.9973 s."""
    rng = np.random.default_rng(1)
    s = 2.5
    img = (rng.normal(size=(1024, 1024)) * s + 7.0).astype(np.float32)
    m, sig, rounds = M.iterative_mad(img)
    assert abs(m - 7.0) < 0.01 and rounds <= 10
    assert abs(sig / s - 0.9973) < 0.004, sig / s


def test_robust_to_sources_and_holes():
    """3 % bright point-like outliers and 1 % deep negative holes leave the
    estimate within 2 % of the noise sigma; the plain standard deviation is
    inflated several times."""
    rng = np.random.default_rng(2)
    img = rng.normal(size=(1024, 1024)).astype(np.float32)
    flat = img.ravel()
    idx = rng.choice(flat.size, int(0.04 * flat.size), replace=False)
    flat[idx[: int(0.03 * flat.size)]] += rng.uniform(20, 200, int(0.03 * flat.size)).astype(np.float32)
    flat[idx[int(0.03 * flat.size):]] -= 50.0
    _, sig, _ = M.iterative_mad(img)
    assert abs(sig - 1.0) < 0.02, sig
    assert np.std(img) > 5.0


def test_constant_image_gives_zero_sigma():
    m, s, rounds = M.iterative_mad(np.full((64, 64), 3.25, np.float32))
    assert m == np.float32(3.25) and s == 0.0 and rounds == 2


def test_mad_constant_is_the_normal_quantile():
    """1.4826 ~ 1 / Phi^-1(3/4) (the MAD of a standard normal is 0.67449)."""
    q = math.sqrt(2.0) * 0.4769362762044699        # Phi^-1(3/4) = sqrt(2) erfinv(1/2)
    assert abs(1.0 / q - float(M.MAD_TO_SIGMA)) < 1e-4
