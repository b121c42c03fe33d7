"""CPU check of the selection scheme of the GPU noise estimate (the
iterative median absolute deviation, paper sec. 3): the scheme written out
in numpy (no code shared with the CUDA path) must reproduce the oracle's
(median, sigma, rounds) bit for bit, whatever the speculation decides.

The scheme selects each order statistic on order-preserving 32-bit keys of
the FP32 values: a histogram of 8192 bins of 2^shift keys laid around a
predicted key (the previous round's result; the whole key range in round 0),
one bin below and one above the window, the bin width set from the key
density the previous round found; the keys of the few bins around the
prediction copied speculatively; the chosen bin selected exactly from those
copies, else copied out by a second pass, else histogrammed again at a finer
width.  Exactness rests on the bins being monotone in the key and on the
final selection being exact among every key of the chosen bin; the images
below push every branch (offset data whose round-0 bin overflows the copy
buffer, one value repeated beyond it, ties, infinities, constant and tiny
images)."""
import numpy as np
import pytest

from oracle import mad as M

INNER = 8192
BINS = INNER + 2
MAX_SHIFT = 19


def keys_of(v):
    u = np.asarray(v, np.float32).view(np.uint32).astype(np.uint64)
    return np.where(u & 0x80000000, (~u) & 0xFFFFFFFF, u | 0x80000000).astype(np.uint64)


def value_of(k):
    k = int(k)
    u = (k & 0x7FFFFFFF) if (k & 0x80000000) else ((~k) & 0xFFFFFFFF)
    return np.array([u], np.uint32).view(np.float32)[0]


def bins_of(k, lo, shift):
    q = k.astype(np.int64) - lo
    return np.where(q < 0, 0, np.minimum((q >> shift) + 1, BINS - 1))


class Sel:
    """The per-image state of the selection (one image)."""

    def __init__(self, cap, max_rounds):
        self.cap, self.max_rounds = cap, max_rounds
        self.done, self.round, self.rounds, self.passes = False, 0, 0, 0
        self.rho, self.kpred = [0.0, 0.0], [0, 0]
        self.trace = []                                    # the branch each pick took
        self.m_prev = self.thr_prev = self.m_cur = self.m_last = self.sigma = np.float32(0)
        self.setup(0)

    def setup(self, w):
        self.what, self.phase, self.level = w, "hist", 0
        self.blo, self.bhi, self.slo, self.shi = 0, 0xFFFFFFFF, 1, 0
        rho = self.rho[w]
        if self.round == 0 or not (rho > 0) or not np.isfinite(rho):
            self.lo, self.shift = (0x80000000, MAX_SHIFT - 1) if w else (0, MAX_SHIFT)
            return
        bw = self.cap / 16.0 / rho
        sft = 0
        while sft < MAX_SHIFT and (1 << sft) < bw:
            sft += 1
        kp = self.kpred[w]
        half = (INNER // 2) << sft
        self.lo, self.shift = (kp - half if kp > half else 0), sft
        bc = 1 + ((kp - self.lo) >> sft)
        hbf = self.cap / 8.0 / (rho * (1 << sft))
        hb = 1 if hbf < 1 else (64 if hbf > 64 else int(hbf))
        b0, b1 = max(1, bc - hb), min(INNER, bc + hb)
        slo, shi = self.lo + ((b0 - 1) << sft), self.lo + (b1 << sft) - 1
        if slo <= 0xFFFFFFFF:
            self.slo, self.shi = slo, min(shi, 0xFFFFFFFF)

    def finish(self, key, bl, bh, cb):
        w = self.what
        self.rho[w], self.kpred[w] = cb / (bh - bl + 1.0), key
        v = value_of(key)
        if w == 0:
            self.m_cur = v
            self.setup(1)
            return
        sigma = np.float32(np.float32(1.4826) * v)
        self.rounds = self.round + 1
        if self.round > 0 and self.m_cur == self.m_last and sigma == self.sigma:
            self.done = True
            return
        self.m_last, self.sigma, self.m_prev = self.m_cur, sigma, self.m_cur
        self.thr_prev = np.float32(np.float32(3.0) * sigma)
        self.round += 1
        if self.round >= self.max_rounds:
            self.done = True
            return
        self.setup(0)

    def step(self, x):
        """One pass over the image, then the pick."""
        member = np.ones(x.shape, bool) if self.round == 0 else np.abs(x - self.m_prev) <= self.thr_prev
        v = x[member] if self.what == 0 else np.abs(x[member] - self.m_cur)
        k = keys_of(v)
        k = k[(k >= self.blo) & (k <= self.bhi)]
        self.passes += 1
        if self.phase == "compact":
            self.trace.append("compacted")
            self.finish(int(np.sort(k)[self.krem]), self.blo, self.bhi, len(k))
            return
        h = np.bincount(bins_of(k, self.lo, self.shift), minlength=BINS)
        copies = k[(k >= self.slo) & (k <= self.shi)]
        total = int(h.sum())
        if total == 0:
            self.m_cur = self.m_last = self.sigma = np.float32(np.nan)
            self.done = True
            return
        r = (total - 1) // 2 if self.level == 0 else self.krem
        c = np.cumsum(h)
        b = int(np.searchsorted(c, r, side="right"))
        r -= int(c[b - 1]) if b > 0 else 0
        if b == 0:
            bl, bh = 0, self.lo - 1
        elif b == BINS - 1:
            bl, bh = self.lo + (INNER << self.shift), 0xFFFFFFFF
        else:
            bl = self.lo + ((b - 1) << self.shift)
            bh = bl + (1 << self.shift) - 1
        bl, bh = max(bl, self.blo), min(bh, self.bhi)
        cb = int(h[b])
        spec = self.slo <= self.shi and bl >= self.slo and bh <= self.shi and len(copies) <= self.cap
        self.trace.append("single" if bl == bh else "spec" if spec else "compact" if cb <= self.cap else "level")
        if bl == bh:
            self.finish(bl, bl, bh, cb)
        elif spec:
            self.finish(int(np.sort(copies[(copies >= bl) & (copies <= bh)])[r]), bl, bh, cb)
        elif cb <= self.cap:
            self.phase, self.level, self.blo, self.bhi, self.krem = "compact", self.level + 1, bl, bh, r
            self.slo, self.shi = 1, 0
        else:
            self.phase, self.level, self.blo, self.bhi, self.krem = "hist", self.level + 1, bl, bh, r
            self.slo, self.shi, self.lo = 1, 0, bl
            sft = 0
            while ((bh - bl) >> sft) >= INNER:
                sft += 1
            self.shift = sft


def estimate(x, cap, max_rounds=10):
    x = np.asarray(x, np.float32).ravel()
    s = Sel(cap, max_rounds)
    for _ in range(10 * max_rounds + 4):
        if s.done:
            break
        s.step(x)
    return s


def _images():
    rng = np.random.default_rng(0)
    out = []
    for n, sg, mu in [(200_000, 1.0, 0.0), (150_000, 2.5, 7.0), (70_001, 0.3, -2.0)]:
        x = (rng.normal(size=n) * sg + mu).astype(np.float32)
        idx = rng.choice(n, n // 25, replace=False)
        x[idx[: n // 40]] += rng.uniform(20, 500, n // 40).astype(np.float32)
        x[idx[n // 40:]] -= 60.0
        out.append(x)
    x = (np.random.default_rng(3).normal(size=300_000) + 100.0).astype(np.float32)
    x[np.random.default_rng(4).choice(x.size, 700, replace=False)] = np.inf
    out.append(x)                                          # round 0's bin overflows the buffer
    x = np.zeros(100_000, np.float32)
    x[:20_000] = np.random.default_rng(6).normal(size=20_000).astype(np.float32)
    out.append(x)                                          # one key above the buffer: a single-key end
    out += [np.array([1, 2, 3, 4, 100], np.float32), np.array([5.5], np.float32),
            np.full(4096, 3.25, np.float32), np.array([-0.0, 0.0, 1.0, -1.0, 2.0, 0.5], np.float32),
            np.random.default_rng(9).integers(-3, 4, 100_000).astype(np.float32)]
    return out


@pytest.mark.parametrize("cap", [1 << 16, 4096])
def test_selection_scheme_is_exact(cap):
    imgs = _images()
    for x in imgs:
        m, s, r = M.iterative_mad(x)
        est = estimate(x, min(cap, max(len(x), 1)))
        assert est.m_last == m and est.sigma == s and est.rounds == r, (len(x), est.m_last, m, est.sigma, s)


def test_selection_paths_are_exercised():
    """Every branch of the pick runs on these images (speculative hits, a
    compaction pass, a finer histogram level, a single-key end), and once
    the estimate settles a selection takes one pass: at most two passes for
    each of round 0's selections and the next one, one for every other."""
    seen = set()
    for x in _images():
        seen.update(estimate(x, min(1 << 16, max(len(x), 1))).trace)
    assert {"spec", "compact", "compacted", "level", "single"} <= seen, seen
    x = _images()[0]
    m, s, r = M.iterative_mad(x)
    est = estimate(x, 1 << 16)
    assert est.passes <= 2 * r + 4 < 6 * r                 # a plain 3-digit radix select: 6 a round
