"""FP64 oracle of the learned vetting stage: stacked postage stamps along a
candidate's track and a small CNN that scores them.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper names this stage as future work (sec. 5.2.3: a network
that learns to tell stacked images of real detections from stacks of false
ones) and
fixes neither the stamp nor the network.  The definitions here are the
readings this project builds to:

Stamps.  For candidate orbit o and every exposure j where its predicted
nearest pixel (ix, iy) lies inside the image, take the matched-filter planes
in the (2H+1) x (2H+1) window centred on (ix, iy) (pixels outside the image
contribute nothing) and accumulate over exposures, per window offset q:
  SPsi(q) = sum_j psi_j(p_j + q),   SPhi(q) = sum_j phi_j(p_j + q).
Channel 0 is the stacked SNR SPsi / sqrt(SPhi) (0 where SPhi = 0), i.e. the
constant-flux statistic of sec. 3 evaluated on a grid of shifted tracks.
Channel 1 measures how badly the constant-flux model fits the individual
exposures, the outlier signature of sec. 5.2.3: with
Q(q) = sum_j psi_j(p_j + q)^2 / phi_j(p_j + q) over the n(q) contributing
exposures, the model residual is chi2 = Q - SPsi^2 / SPhi (the minimum over
the flux of sum_j (psi_j - a phi_j)^2 / phi_j), and channel 1 is its
standardised excess (chi2 - (n - 1)) / sqrt(2 (n - 1)) (0 where n < 2).

Network.  x (B, 2, 21, 21) -> conv5x5(2->32) -> ReLU -> conv5x5(32->32) ->
ReLU -> conv5x5(32->32) -> ReLU -> global average pool -> linear(32->1) ->
logit; score = sigmoid(logit); loss = mean binary cross-entropy with logits.
Convolutions are cross-correlations with zero padding 2 and a bias per output
channel.  Parameters are one flat FP64 vector in the order
w1 (32,2,5,5), b1 (32), w2 (32,32,5,5), b2 (32), w3 (32,32,5,5), b3 (32),
wl (32), bl (1): 52,929 values.
"""
import numpy as np

STAMP_HALF = 10
STAMP = 2 * STAMP_HALF + 1
C_IN, C_HID, K = 2, 32, 5
SHAPES = [("w1", (C_HID, C_IN, K, K)), ("b1", (C_HID,)),
          ("w2", (C_HID, C_HID, K, K)), ("b2", (C_HID,)),
          ("w3", (C_HID, C_HID, K, K)), ("b3", (C_HID,)),
          ("wl", (C_HID,)), ("bl", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    theta = np.asarray(theta, np.float64)
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in SHAPES])


def init_params(seed=0):
    """He-normal weights, zero biases (seeded)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in SHAPES:
        if name.startswith("w") and len(shp) == 4:
            fan_in = shp[1] * shp[2] * shp[3]
            p[name] = rng.normal(0.0, np.sqrt(2.0 / fan_in), shp)
        elif name == "wl":
            p[name] = rng.normal(0.0, np.sqrt(1.0 / shp[0]), shp)
        else:
            p[name] = np.zeros(shp)
    return pack(p)


# ------------------------------------------------------------------ stamps --

def stamps(xy, planes, width, height, half=STAMP_HALF):
    """xy: (n_cand, n_exp, 2) predicted pixel coordinates (NaN: not visible);
    planes: list of (psi, phi) FP64 planes per exposure.  Returns
    (n_cand, 2, 2h+1, 2h+1) FP64 stamps by the definition above."""
    n_cand, n_exp, _ = xy.shape
    S = 2 * half + 1
    out = np.zeros((n_cand, 2, S, S))
    for o in range(n_cand):
        spsi = np.zeros((S, S))
        sphi = np.zeros((S, S))
        sq = np.zeros((S, S))
        cnt = np.zeros((S, S), np.int64)
        for j in range(n_exp):
            x, y = xy[o, j]
            if not (np.isfinite(x) and np.isfinite(y)):
                continue
            ix, iy = int(np.floor(x + 0.5)), int(np.floor(y + 0.5))
            W, H = int(width[j]), int(height[j])
            if not (0 <= ix < W and 0 <= iy < H):
                continue
            psi, phi = planes[j]
            for dy in range(-half, half + 1):
                for dx in range(-half, half + 1):
                    px, py = ix + dx, iy + dy
                    if not (0 <= px < W and 0 <= py < H):
                        continue
                    a, b = psi[py, px], phi[py, px]
                    if not b > 0:
                        continue
                    q = (dy + half, dx + half)
                    spsi[q] += a
                    sphi[q] += b
                    sq[q] += a * a / b
                    cnt[q] += 1
        ok = sphi > 0
        ch0 = np.zeros((S, S))
        ch0[ok] = spsi[ok] / np.sqrt(sphi[ok])
        m = cnt >= 2
        ch1 = np.zeros((S, S))
        chi2 = sq[m] - spsi[m] ** 2 / sphi[m]
        ch1[m] = (chi2 - (cnt[m] - 1)) / np.sqrt(2.0 * (cnt[m] - 1))
        out[o, 0] = ch0
        out[o, 1] = ch1
    return out


# --------------------------------------------------------------------- CNN --

def _cols(x, KK):
    """im2col: (B, C, H, W) -> (B, C*KK*KK, H*W), zero padding KK//2; row index
    c*KK*KK + u*KK + v holds x[c, h+u-KK//2, w+v-KK//2]."""
    B, C, H, W = x.shape
    p = KK // 2
    xp = np.zeros((B, C, H + 2 * p, W + 2 * p))
    xp[:, :, p:p + H, p:p + W] = x
    win = np.lib.stride_tricks.sliding_window_view(xp, (KK, KK), axis=(2, 3))  # B,C,H,W,KK,KK
    return win.transpose(0, 1, 4, 5, 2, 3).reshape(B, C * KK * KK, H * W)


def conv2d(x, w, b):
    """Cross-correlation, zero padding K//2, stride 1: x (B,C,H,W), w (O,C,K,K)."""
    B, C, H, W = x.shape
    O, _, KK, _ = w.shape
    y = np.matmul(w.reshape(O, -1), _cols(x, KK))             # (B, O, H*W)
    return y.reshape(B, O, H, W) + b[None, :, None, None]


def bf16_round(a):
    """Round to BF16 (round-to-nearest-even, through FP32 first), as FP64."""
    u = np.asarray(a, np.float64).astype(np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta, x, keep=False, bf16_operands=False):
    """Logits (B,) of the network; with keep=True also the activations.
    bf16_operands=True gives the scoring variant, whose convolution operands
    are BF16: the weights of all three layers and the activations entering
    layers 2 and 3 are rounded to BF16 (the stamps already are BF16); sums,
    biases, pooling and the head stay exact here."""
    p = unpack(theta)
    x = np.asarray(x, np.float64)
    rnd = bf16_round if bf16_operands else (lambda a: a)
    y1 = conv2d(x, rnd(p["w1"]), p["b1"]); a1 = rnd(np.maximum(y1, 0))
    y2 = conv2d(a1, rnd(p["w2"]), p["b2"]); a2 = rnd(np.maximum(y2, 0))
    y3 = conv2d(a2, rnd(p["w3"]), p["b3"]); a3 = np.maximum(y3, 0)
    g = a3.mean(axis=(2, 3))
    z = g @ p["wl"] + p["bl"][0]
    if keep:
        return z, dict(x=x, y1=y1, a1=a1, y2=y2, a2=a2, y3=y3, a3=a3, g=g)
    return z


def bce_with_logits(z, y):
    """Mean over the batch of -[y log s + (1-y) log(1-s)], s = sigmoid(z)."""
    z, y = np.asarray(z, np.float64), np.asarray(y, np.float64)
    return float(np.mean(np.maximum(z, 0) - z * y + np.log1p(np.exp(-np.abs(z)))))


def _conv_backward(x, w, dy):
    """Gradients of conv2d: (dx, dw, db)."""
    B, C, H, W = x.shape
    O, _, KK, _ = w.shape
    p = KK // 2
    cols = _cols(x, KK)                                        # (B, C*KK*KK, HW)
    dyf = dy.reshape(B, O, H * W)
    dw = np.matmul(dyf, cols.transpose(0, 2, 1)).sum(axis=0).reshape(w.shape)
    dcols = np.matmul(w.reshape(O, -1).T, dyf).reshape(B, C, KK, KK, H, W)
    dxp = np.zeros((B, C, H + 2 * p, W + 2 * p))
    for u in range(KK):
        for v in range(KK):
            dxp[:, :, u:u + H, v:v + W] += dcols[:, :, u, v]
    return dxp[:, :, p:p + H, p:p + W], dw, dy.sum(axis=(0, 2, 3))


def loss_and_grad(theta, x, y):
    """Mean BCE loss and its gradient with respect to the flat parameters."""
    p = unpack(theta)
    z, c = forward(theta, x, keep=True)
    y = np.asarray(y, np.float64)
    B = len(z)
    loss = bce_with_logits(z, y)
    dz = (1.0 / (1.0 + np.exp(-z)) - y) / B                     # (B,)
    grads = {"wl": c["g"].T @ dz, "bl": np.array([dz.sum()])}
    dg = dz[:, None] * p["wl"][None, :]                           # (B,32)
    HW = c["a3"].shape[2] * c["a3"].shape[3]
    da3 = np.broadcast_to(dg[:, :, None, None] / HW, c["a3"].shape)
    dy3 = da3 * (c["y3"] > 0)
    da2, grads["w3"], grads["b3"] = _conv_backward(c["a2"], p["w3"], dy3)
    dy2 = da2 * (c["y2"] > 0)
    da1, grads["w2"], grads["b2"] = _conv_backward(c["a1"], p["w2"], dy2)
    dy1 = da1 * (c["y1"] > 0)
    _, grads["w1"], grads["b1"] = _conv_backward(c["x"], p["w1"], dy1)
    return loss, pack(grads)


# ------------------------------------------- error bound of BF16 scoring --
#
# A scorer that rounds the network's convolution operands to BF16 (unit
# roundoff u = 2^-8 for round-to-nearest-even) and accumulates in FP32
# computes a logit z~ that differs from the exact logit z of forward().  The
# bound below takes that difference in two parts.
#
# BF16 operand rounding.  Every rounded operand v (a weight of w1, w2 or w3,
# an activation of a1 or a2; the stamps are BF16 already) becomes v (1 + d)
# with |d| <= u.  To first order the logit moves by sum_i c_i d_i with
# c_i = (dz/dv_i) v_i, the operand's sensitivity times its value, both from
# the exact network.  Under the probabilistic model of rounding (Higham &
# Mary 2019: the d_i independent, mean zero, |d_i| <= u), Hoeffding's
# inequality gives P(|sum c_i d_i| >= lam u sqrt(sum c_i^2)) <=
# 2 exp(-lam^2 / 2), 4.6e-11 at lam = 7.
#
# FP32 accumulation.  Each output of layer l (K_l = 25 C_in products plus
# the bias) and the pooling (441 terms) and head (33 terms) sums are
# bounded in the worst case, whatever the summation order or rounding mode,
# by 2 n u32 sum_k |term_k| (u32 = 2^-24; the factor 2 admits truncating
# adders), carried to the logit by |dz/dy|.
#
# The bound neglects second-order terms (relative size ~u) and the few
# activations whose sign a perturbation flips (a ReLU kink moves such an
# element by at most its own perturbation).

U_BF16 = 2.0 ** -8
U_FP32 = 2.0 ** -24


def _conv_abs(x, w):
    """|w| correlated with |x| (zero padding), no bias: the sum of the term
    magnitudes under each output."""
    return conv2d(np.abs(x), np.abs(w), np.zeros(w.shape[0]))


def _conv_backward_per_stamp(x, w, dy):
    """Per-stamp gradients of conv2d: dx (B,C,H,W) and dw (B,O,C,K,K)."""
    B, C, H, W = x.shape
    O, _, KK, _ = w.shape
    p = KK // 2
    cols = _cols(x, KK)                                        # (B, C*KK*KK, HW)
    dyf = dy.reshape(B, O, H * W)
    dw = np.matmul(dyf, cols.transpose(0, 2, 1)).reshape((B,) + w.shape)
    dcols = np.matmul(w.reshape(O, -1).T, dyf).reshape(B, C, KK, KK, H, W)
    dxp = np.zeros((B, C, H + 2 * p, W + 2 * p))
    for u in range(KK):
        for v in range(KK):
            dxp[:, :, u:u + H, v:v + W] += dcols[:, :, u, v]
    return dxp[:, :, p:p + H, p:p + W], dw


def logit_sensitivities(theta, x):
    """Per stamp: the exact logits z (B,), the operand terms c = (dz/dv) v of
    every BF16-rounded group {'w1','w2','w3','a1','a2'} (arrays (B, ...)),
    and the FP32-accumulation magnitudes {'y1','y2','y3','pool','head'}
    (B,): sum over the sums' outputs of |dz/dy| times sum |term| and the
    term count n, as (magnitude, n) pairs."""
    p = unpack(theta)
    z, c = forward(theta, x, keep=True)
    B = len(z)
    HW = c["a3"].shape[2] * c["a3"].shape[3]
    da3 = np.broadcast_to(p["wl"][None, :, None, None] / HW, c["a3"].shape)
    dy3 = da3 * (c["y3"] > 0)
    da2, dw3 = _conv_backward_per_stamp(c["a2"], p["w3"], dy3)
    dy2 = da2 * (c["y2"] > 0)
    da1, dw2 = _conv_backward_per_stamp(c["a1"], p["w2"], dy2)
    dy1 = da1 * (c["y1"] > 0)
    _, dw1 = _conv_backward_per_stamp(c["x"], p["w1"], dy1)
    terms = {"w1": dw1 * p["w1"][None], "w2": dw2 * p["w2"][None], "w3": dw3 * p["w3"][None],
             "a1": da1 * c["a1"], "a2": da2 * c["a2"]}
    acc = {}
    for name, dy, a_in, w, b in (("y1", dy1, c["x"], p["w1"], p["b1"]),
                                 ("y2", dy2, c["a1"], p["w2"], p["b2"]),
                                 ("y3", dy3, c["a2"], p["w3"], p["b3"])):
        mag = _conv_abs(a_in, w) + np.abs(b)[None, :, None, None]
        acc[name] = ((np.abs(dy) * mag).sum(axis=(1, 2, 3)), w.shape[1] * w.shape[2] * w.shape[3] + 1)
    acc["pool"] = ((np.abs(p["wl"])[None, :] * c["a3"].mean(axis=(2, 3))).sum(axis=1), HW)
    acc["head"] = (np.abs(c["g"] * p["wl"][None, :]).sum(axis=1) + abs(p["bl"][0]), p["wl"].size + 1)
    return z, terms, acc


def bf16_logit_bound(theta, x, lam=7.0, chunk=32):
    """Per-stamp bound (B,) on |z~ - z| for a scorer with BF16 weights and
    BF16 activations entering layers 2 and 3 and FP32 sums (see above):
      lam u sqrt(sum_groups sum_i c_i^2) + sum_sums 2 n u32 |dz/dy| sum |term|.
    Also returns the exact logits."""
    x = np.asarray(x, np.float64)
    zs, bounds = [], []
    for s in range(0, len(x), chunk):
        z, terms, acc = logit_sensitivities(theta, x[s:s + chunk])
        ss = sum((t.reshape(len(z), -1) ** 2).sum(axis=1) for t in terms.values())
        b32 = sum(2.0 * n * U_FP32 * m for m, n in acc.values())
        zs.append(z)
        bounds.append(lam * U_BF16 * np.sqrt(ss) + b32)
    return np.concatenate(bounds), np.concatenate(zs)
