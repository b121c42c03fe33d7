"""Oracle of the iterative median-absolute-deviation noise estimate.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper (sec. 3) derives each image's pixel noise variance from a median
absolute deviation that is iterated, and gives no further detail.  The
reading built to here, per image of FP32 pixels x:

    S_0 = every pixel
    m_i     = lower median of S_i          (the element of rank floor((n-1)/2))
    mad_i   = lower median of { |x - m_i| : x in S_i }
    sigma_i = 1.4826 * mad_i               (1 / Phi^-1(3/4): sigma of a normal)
    S_{i+1} = { x : |x - m_i| <= 3 sigma_i }   over every pixel
    stop when (m_i, sigma_i) equals (m_{i-1}, sigma_{i-1}), or after 10 rounds;
    variance = sigma^2 of the last round.

Every quantity that decides membership or a rank is an FP32 value computed
with FP32 operations in the order written (|x - m| as one FP32 subtraction,
sigma = fl32(1.4826 * mad), the threshold fl32(3 * sigma)), so that an FP32
implementation can reproduce it bit for bit; ranks are exact order
statistics.  numpy's float32 arithmetic rounds to nearest like the GPU's.
"""
import numpy as np

MAD_TO_SIGMA = np.float32(1.4826)
CLIP = np.float32(3.0)


def lower_median(v):
    """The element of rank floor((n - 1) / 2) of v in ascending order."""
    v = np.asarray(v)
    k = (len(v) - 1) // 2
    return np.partition(v, k)[k]


def iterative_mad(img, max_rounds=10):
    """(median, sigma, rounds) of one image (any shape, FP32 values)."""
    x = np.asarray(img, np.float32).ravel()
    keep = np.ones(x.shape, bool)
    prev = None
    m = sigma = np.float32(0.0)
    rounds = 0
    for _ in range(max_rounds):
        rounds += 1
        s = x[keep]
        m = np.float32(lower_median(s))
        dev = np.abs(s - m)                      # FP32 subtraction, exact |.|
        sigma = np.float32(MAD_TO_SIGMA * np.float32(lower_median(dev)))
        if prev is not None and prev == (m, sigma):
            break
        prev = (m, sigma)
        thr = np.float32(CLIP * sigma)
        keep = np.abs(x - m) <= thr
    return m, sigma, rounds


def variance(img, max_rounds=10):
    """Noise variance estimate sigma^2 (FP64 of the FP32 sigma)."""
    _, s, _ = iterative_mad(img, max_rounds)
    return float(s) ** 2
