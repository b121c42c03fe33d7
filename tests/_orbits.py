"""Seeded orbit populations shared by tests (no GPU needed)."""
import math

import numpy as np

import oracle as O


def mixed_population(rng, n):
    """NEO-like (q < 1.3 AU, e up to 0.8), main belt, Kuiper belt (30-50 AU) and
    hyperbolic states at random orientations."""
    mu = O.gm_sun()
    out = []
    for i in range(n):
        kind = i % 4
        if kind == 0:
            a, e = rng.uniform(0.8, 2.5), rng.uniform(0.3, 0.8)
        elif kind == 1:
            a, e = rng.uniform(2.1, 3.3), rng.uniform(0.0, 0.2)
        elif kind == 2:
            a, e = rng.uniform(30.0, 50.0), rng.uniform(0.0, 0.2)
        else:
            a, e = -rng.uniform(1.0, 5.0), rng.uniform(1.1, 2.0)
        nu = rng.uniform(-2.0, 2.0) if kind == 3 else rng.uniform(0, 2 * math.pi)
        p = a * (1 - e * e)
        r = p / (1 + e * math.cos(nu))
        pos = np.array([r * math.cos(nu), r * math.sin(nu), 0.0])
        vel = math.sqrt(mu / p) * np.array([-math.sin(nu), e + math.cos(nu), 0.0])
        inc, node, argp = rng.uniform(0, 0.5), rng.uniform(0, 2 * math.pi), rng.uniform(0, 2 * math.pi)
        def rot(v):
            c, s = math.cos(argp), math.sin(argp)
            v = np.array([c * v[0] - s * v[1], s * v[0] + c * v[1], v[2]])
            c, s = math.cos(inc), math.sin(inc)
            v = np.array([v[0], c * v[1] - s * v[2], s * v[1] + c * v[2]])
            c, s = math.cos(node), math.sin(node)
            return np.array([c * v[0] - s * v[1], s * v[0] + c * v[1], v[2]])
        out.append(np.concatenate([rot(pos), rot(vel)]))
    return np.array(out)
