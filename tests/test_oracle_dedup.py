"""Pins of the duplicate-suppression oracle (oracle/dedup.py): reference
exposures by hand-worked positions, identical orbits, far-apart orbits and
the rank-order rule on a chain of three tracks."""
import numpy as np

import oracle as O
from oracle import dedup as D
from paper_2503_08854_gb300 import synth


def test_reference_positions_hand_worked():
    ex = synth.grid_sky(n_exp=10, size=64, n_r=1, n_v=2, seed=1).ex
    order = np.argsort(ex.mjd, kind="stable")
    # 10 exposures, 3 references: positions 0, round(4.5) = 5, 9
    assert list(D.reference_positions(ex, 3)) == list(order[[0, 5, 9]])
    # 1 reference: the middle position (10 - 1) // 2 = 4
    assert list(D.reference_positions(ex, 1)) == [order[4]]
    # 4 references: 0, 3, 6, 9
    assert list(D.reference_positions(ex, 4)) == list(order[[0, 3, 6, 9]])
    # 2 exposures, 3 references: 0, round(0.5) = 1, 1 -> the repeat is dropped
    assert list(D.reference_positions(ex.subset([3, 1]), 3)) == [1, 0]


def test_reference_positions_in_a_window():
    ex = synth.grid_sky(n_exp=10, size=64, n_r=1, n_v=2, seed=1).ex
    order = np.argsort(ex.mjd, kind="stable")
    t = ex.mjd[order]
    # a window holding sorted positions 3..7 (m = 5): 3, 3 + round(2) = 5, 7
    w = (0.5 * (t[2] + t[3]), 0.5 * (t[7] + t[8]))
    assert list(D.reference_positions(ex, 3, w)) == list(order[[3, 5, 7]])
    assert list(D.reference_positions(ex, 1, w)) == [order[5]]


def test_reference_positions_follow_epoch_order():
    ex = synth.grid_sky(n_exp=5, size=64, n_r=1, n_v=2, seed=1).ex
    perm = np.array([3, 0, 4, 1, 2])
    sub = ex.subset(perm)                    # table out of epoch order
    refs = D.reference_positions(sub, 3)
    assert list(sub.mjd[refs]) == [ex.mjd.min(), np.sort(ex.mjd)[2], ex.mjd.max()]


def _chain(sky, step):
    """Three orbits: a base state and two offsets of 1 and 2 steps (AU)
    perpendicular to the base's line of sight at t0, in the ecliptic."""
    s0 = sky.states[len(sky.states) // 2].copy()
    los = s0[:3] - sky.ex.obs[np.argmin(np.abs(sky.ex.mjd - sky.t0))]
    perp = np.cross(los, [0.0, 0.0, 1.0])
    perp /= np.linalg.norm(perp)
    out = np.array([s0, s0, s0])
    out[1, :3] += step * perp
    out[2, :3] += 2 * step * perp
    return out


def test_identical_and_far_orbits():
    sky = synth.grid_sky(n_exp=8, size=200, n_r=4, n_v=8, scale_arcsec=1.0, seed=2)
    st = sky.states
    far = np.argmax(np.linalg.norm(st[:, 3:] - st[0, 3:], axis=1))
    states = np.array([st[0], st[0], st[far], st[0]])
    kept, dist = D.dedup(states, sky.t0, sky.ex, np.arange(4), radius=1.0)
    assert list(kept) == [0, 2]               # copies of candidate 0 go, the far orbit stays
    assert dist[1, 0] == 0.0 and dist[3, 0] == 0.0
    assert dist[2, 0] > 100.0


def test_local_maximum_rule_on_a_chain():
    sky = synth.grid_sky(n_exp=8, size=200, n_r=4, n_v=8, scale_arcsec=1.0, seed=2)
    states = _chain(sky, 2e-6)
    _, dist = D.dedup(states, sky.t0, sky.ex, np.arange(3), radius=1e9)
    dab, dac, dbc = dist[1, 0], dist[2, 0], dist[2, 1]
    assert 0 < dab < dac and 0 < dbc < dac    # a chain: B between A and C
    r = 0.5 * (max(dab, dbc) + dac) if max(dab, dbc) < dac else None
    assert r is not None
    # rank A, B, C: B lies within r of A, C within r of B -> only A survives,
    # although C is farther than r from A (a candidate falls to any better
    # neighbour, kept or not)
    kept, _ = D.dedup(states, sky.t0, sky.ex, np.arange(3), radius=r)
    assert list(kept) == [0]
    # rank A, C, B: C is farther than r from A and stays; B falls to A
    kept, _ = D.dedup(states, sky.t0, sky.ex, np.array([0, 2, 1]), radius=r)
    assert list(kept) == [0, 2]
    # the distance is the largest over the references of the per-exposure
    # distance between the oracle's own predicted positions
    refs = D.reference_positions(sky.ex, 3)
    xy = O.predict(states, sky.t0, sky.ex.subset(refs))
    assert np.isclose(dab, np.max(np.hypot(*(xy[1] - xy[0]).T)), rtol=1e-12)
