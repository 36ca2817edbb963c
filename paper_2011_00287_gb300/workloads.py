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


def bulk_order(shape, S0: float = 0.5, q0: float = 0.0, noise: float = 1e-3, seed: int = 1):
    """Bulk liquid crystal with no droplet (psi = 1 everywhere): Q = S0 (n n - I/3) with the
    director n = (cos q0 z, sin q0 z, 0) (q0 = 0: a uniform nematic along x; q0 != 0: a
    cholesteric helix about z), plus noise * U[-1, 1) on each stored component from numpy's
    PCG64 seeded with `seed`.  Returns {"q": (5, nz, ny, nx), "psi": (nz, ny, nx)}; the
    populations and the velocity keep the fluid at rest as created."""
    nx, ny, nz = shape
    z = np.arange(nz, dtype=np.float64).reshape(nz, 1, 1) * np.ones((nz, ny, nx))
    n0, n1 = np.cos(q0 * z), np.sin(q0 * z)
    q = np.array([S0 * (n0 * n0 - 1.0 / 3.0), S0 * n0 * n1, 0.0 * z, S0 * (n1 * n1 - 1.0 / 3.0), 0.0 * z])
    rng = np.random.default_rng(seed)
    q += noise * rng.uniform(-1.0, 1.0, size=q.shape)
    return {"q": np.ascontiguousarray(q), "psi": np.ones((nz, ny, nx))}


def shard(count: int, rank: int, world: int):
    """Contiguous share of `count` independent units for `rank` of `world`."""
    lo = (count * rank) // world
    hi = (count * (rank + 1)) // world
    return list(range(lo, hi))
