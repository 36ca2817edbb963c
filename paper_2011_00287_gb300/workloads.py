"""Seeded synthetic workload descriptions (shapes and parameter draws only; none of the
method's arithmetic).  Both the library's users (bench, tests) and the oracle build their
parameters from these tuples."""
from __future__ import annotations

import numpy as np


def droplet_box(n: int):
    """One droplet in an n^3 box: R = n/4, pitch p0 = n/4 (the 128^3 workload has R = 32,
    pitch 32).  Returns (grid, R, p0)."""
    return (n, n, n), n / 4.0, n / 4.0


def batch_uneven(seed: int = 7, count: int = 64, edges=(48, 64, 80, 96)):
    """`count` independent droplets: each box edge drawn uniformly from `edges`, R = (min
    edge)/4, zeta ~ U[0.001, 0.01], pitch p0 ~ U[12, 40], all from numpy's PCG64 seeded
    with `seed`.  Returns a list of dicts with grid, R, p0, zeta."""
    rng = np.random.default_rng(seed)
    e = rng.choice(np.asarray(edges), size=(count, 3))
    zeta = rng.uniform(0.001, 0.01, size=count)
    p0 = rng.uniform(12.0, 40.0, size=count)
    out = []
    for i in range(count):
        g = tuple(int(v) for v in e[i])
        out.append(dict(grid=g, R=min(g) / 4.0, p0=float(p0[i]), zeta=float(zeta[i])))
    return out


def shard(count: int, rank: int, world: int):
    """Contiguous share of `count` independent units for `rank` of `world`."""
    lo = (count * rank) // world
    hi = (count * (rank + 1)) // world
    return list(range(lo, hi))
