"""Oracle of duplicate suppression of a ranked candidate list.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper reports detections orbit by orbit (Algorithm 1,
FindSignificantResults) and says nothing about candidates that are the same
object found through neighbouring orbits.  The reading built to here: the
candidates come in rank order; n_ref reference exposures are spread evenly
over the epoch-sorted exposures (those with epochs in a given window, when
one is given), at positions round(k (m - 1) / (n_ref - 1)) among those m
(the middle one, (m - 1) // 2, when n_ref = 1), repeated positions dropped; candidate i is a duplicate when some candidate ranked before it has
predicted pixel coordinates within distance r of i's at every reference
exposure (Euclidean distance in that exposure's pixel grid; an undefined
position is never within r); duplicates are removed, the rest keep their
order.  Positions are the oracle's FP64 predictions (two-body propagation,
iterated light time, TAN projection).  Brute force over every pair.
"""
import numpy as np

from .oracle import predict


def reference_positions(ex, n_ref, window=None):
    """Table indices of the reference exposures (epoch order), spread over
    the exposures with epochs in window = (t_lo, t_hi) (all without one)."""
    order = np.argsort(np.asarray(ex.mjd), kind="stable")
    if window is not None:
        t = np.asarray(ex.mjd)[order]
        order = order[(t >= window[0]) & (t <= window[1])]
    n = len(order)
    if n_ref == 1:
        pos = [(n - 1) // 2]
    else:
        pos = []
        for k in range(n_ref):
            p = int(np.floor(k * (n - 1) / (n_ref - 1) + 0.5))
            if not pos or p > pos[-1]:
                pos.append(p)
    return order[np.asarray(pos)]


def track_distances(states, t0, ex, cand, n_ref, window=None):
    """Pixel positions [n_cand, n_ref', 2] of the candidates at the reference
    exposures and the matrix D[i, j] = max over references of the distance
    (inf where a position is undefined)."""
    refs = reference_positions(ex, n_ref, window)
    xy = predict(np.asarray(states)[np.asarray(cand)], t0, ex.subset(refs))
    d = np.sqrt(((xy[:, None, :, :] - xy[None, :, :, :]) ** 2).sum(axis=-1))   # (n, n, n_ref)
    d = np.where(np.isfinite(d), d, np.inf)
    return xy, d.max(axis=-1)


def dedup(states, t0, ex, cand, radius, n_ref=3, window=None):
    """Kept candidates (rank order) and the distance matrix."""
    cand = np.asarray(cand, np.int64)
    _, D = track_distances(states, t0, ex, cand, n_ref, window)
    n = len(cand)
    keep = np.ones(n, bool)
    for i in range(n):
        if np.any(D[i, :i] < radius):
            keep[i] = False
    return cand[keep], D
