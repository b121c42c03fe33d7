"""FP64 oracle of outlier trimming of a candidate's intersections.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper (sec. 5.2.3, the outlier figure there) removes false positives
caused by an artefact in a single difference image: an intersection whose
own SNR lies far above what the constant-flux combination of the others
predicts is dropped (sigma clipping) and the stacked SNR is recomputed.  It fixes neither the statistic nor the
threshold; the readings built to here:

For candidate orbit o, the valid intersections j (nearest pixel inside the
image, phi_j > 0) carry psi_j, phi_j from the matched-filter planes.  Under
the constant-flux model psi_j ~ N(a phi_j, phi_j) (sec. 3), so the
intersection's own SNR s_j = psi_j / sqrt(phi_j) has unit noise about
a sqrt(phi_j), and the residual r_j = s_j - a_hat sqrt(phi_j) is standard
normal.  Starting from the kept set K = all valid intersections:
    a_hat = sum_K psi / sum_K phi;
    K'    = { j valid : r_j(a_hat) <= kappa }      (one-sided: artefacts add flux)
    stop when K' == K or after max_iter rounds, else K = K'.
Every valid intersection is re-tested in each round (clipping is a fixed
point of the rule, not a one-way removal).  The trimmed statistic is
nu' = sum_K psi / sqrt(sum_K phi) over the final K, -inf when sum_K phi = 0
or |K| < min_obs.  Defaults: kappa = 3 (the usual sigma-clipping threshold),
max_iter = 10.
"""
import numpy as np

AMB_PX = 1e-6        # a coordinate this close to a pixel edge is ambiguous


def intersections(xy, planes, width, height):
    """psi (n, J), phi (n, J), valid (n, J) and edge-ambiguity (n, J) of n
    candidates over J exposures: xy (n, J, 2) predicted pixel coordinates
    (NaN when the exposure's tangent point is 90 deg or more away), planes a
    list of (psi_j, phi_j) arrays (H, W) per exposure, nearest pixel
    floor(x + 1/2)."""
    xy = np.asarray(xy, np.float64)
    n, J, _ = xy.shape
    psi = np.zeros((n, J))
    phi = np.zeros((n, J))
    valid = np.zeros((n, J), bool)
    amb = np.zeros((n, J), bool)
    for j in range(J):
        x, y = xy[:, j, 0], xy[:, j, 1]
        fin = np.isfinite(x) & np.isfinite(y)
        ix = np.floor(np.where(fin, x, -1e9) + 0.5)
        iy = np.floor(np.where(fin, y, -1e9) + 0.5)
        inside = fin & (ix >= 0) & (ix < width[j]) & (iy >= 0) & (iy < height[j])
        fx = np.where(fin, x + 0.5 - ix, 0.5)
        fy = np.where(fin, y + 0.5 - iy, 0.5)
        near_edge = fin & ((np.minimum(fx, 1 - fx) < AMB_PX) | (np.minimum(fy, 1 - fy) < AMB_PX))
        ii = np.where(inside, iy, 0).astype(np.int64)
        jj = np.where(inside, ix, 0).astype(np.int64)
        p, f = planes[j]
        psi[:, j] = np.where(inside, p[ii, jj], 0.0)
        phi[:, j] = np.where(inside, f[ii, jj], 0.0)
        valid[:, j] = inside & (phi[:, j] > 0)
        amb[:, j] = near_edge & (fin & (ix >= -1) & (ix <= width[j]) & (iy >= -1) & (iy <= height[j]))
    return psi, phi, valid, amb


def trim(psi, phi, valid, kappa=3.0, max_iter=10, min_obs=1):
    """Sigma-clip each candidate's intersections (rule in the module
    docstring).  Returns a dict of arrays over candidates: Psi, Phi, n (kept
    sums and count), nu (trimmed SNR), rounds (rule evaluations made) and
    margin (the smallest |r_j - kappa| met in any round: a clipping decision
    this close to the threshold may go either way at lower precision) and
    kept, the final kept mask (n, J)."""
    psi = np.atleast_2d(np.asarray(psi, np.float64))
    phi = np.atleast_2d(np.asarray(phi, np.float64))
    valid = np.atleast_2d(np.asarray(valid, bool))
    n_c = psi.shape[0]
    out = {k: np.zeros(n_c) for k in ("Psi", "Phi", "nu", "margin")}
    out["n"] = np.zeros(n_c, np.int64)
    out["rounds"] = np.zeros(n_c, np.int64)
    out["kept"] = np.zeros(psi.shape, bool)
    for c in range(n_c):
        v = valid[c]
        s = np.zeros_like(psi[c])
        w = np.sqrt(np.where(v, phi[c], 0.0))
        s[v] = psi[c][v] / w[v]
        keep = v.copy()
        margin = np.inf
        rounds = 0
        for _ in range(max_iter):
            rounds += 1
            F = phi[c][keep].sum()
            a_hat = psi[c][keep].sum() / F if F > 0 else 0.0
            r = s - a_hat * w
            if v.any():
                margin = min(margin, float(np.min(np.abs(r[v] - kappa))))
            new = v & (r <= kappa)
            if np.array_equal(new, keep):
                break
            keep = new
        P, F, k = psi[c][keep].sum(), phi[c][keep].sum(), int(keep.sum())
        out["Psi"][c], out["Phi"][c], out["n"][c] = P, F, k
        out["nu"][c] = P / np.sqrt(F) if (F > 0 and k >= min_obs) else -np.inf
        out["rounds"][c] = rounds
        out["margin"][c] = margin
        out["kept"][c] = keep
    return out
