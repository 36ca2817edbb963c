"""Host-side analysis of fields read back through the C ABI: scalar order, defect count,
periodic centroid trajectory and droplet speed (the observables of Sec. 4: defects on and
in the droplet, and its drift).  These run on numpy arrays that lbcad_get_fields /
lbcad_observables already produced; nothing here is on the per-step path.
"""
from __future__ import annotations

import numpy as np


def scalar_order(q5: np.ndarray) -> np.ndarray:
    """S = 3/2 lambda_max(Q) per site from the five stored components (5, nz, ny, nx)."""
    xx, xy, xz, yy, yz = q5
    Q = np.empty(q5.shape[1:] + (3, 3))
    Q[..., 0, 0], Q[..., 0, 1], Q[..., 0, 2] = xx, xy, xz
    Q[..., 1, 0], Q[..., 1, 1], Q[..., 1, 2] = xy, yy, yz
    Q[..., 2, 0], Q[..., 2, 1], Q[..., 2, 2] = xz, yz, -xx - yy
    return 1.5 * np.linalg.eigvalsh(Q)[..., -1]


def _periodic_components(mask: np.ndarray):
    """Sizes of the 26-connected components of a boolean (nz, ny, nx) mask on a torus."""
    from scipy import ndimage
    lab, n = ndimage.label(mask, structure=np.ones((3, 3, 3), dtype=bool))
    if n == 0:
        return np.zeros(0, dtype=np.int64)
    parent = np.arange(n + 1)

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    def union(a, b):
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[max(ra, rb)] = min(ra, rb)

    # join labels that touch across each periodic face (26-connectivity: the face
    # neighbour and its 8 in-plane shifts)
    nz, ny, nx = mask.shape
    for axis in range(3):
        lo = np.take(lab, 0, axis=axis)
        hi = np.take(lab, lab.shape[axis] - 1, axis=axis)
        for d0 in (-1, 0, 1):
            for d1 in (-1, 0, 1):
                sh = np.roll(np.roll(hi, d0, axis=0), d1, axis=1)
                both = (lo > 0) & (sh > 0)
                for a, b in zip(lo[both].ravel(), sh[both].ravel()):
                    union(int(a), int(b))
    roots = np.array([find(i) for i in range(n + 1)])
    sizes = np.bincount(roots[lab.ravel()], minlength=n + 1)
    sizes[0] = 0
    return sizes[sizes > 0]


def defect_count(q5: np.ndarray, psi: np.ndarray, s_max: float = 0.25, psi_min: float = 0.0,
                 min_sites: int = 3) -> int:
    """Number of disordered regions inside the droplet: periodic 26-connected components of
    at least `min_sites` sites where psi > psi_min and S < s_max.  psi > 0 keeps the
    inner half of the interface, where the equilibrium order is still S >= 0.38 (chi >=
    2.75), so the interface itself is not counted."""
    mask = (psi > psi_min) & (scalar_order(q5) < s_max)
    sizes = _periodic_components(mask)
    return int(np.sum(sizes >= min_sites))


def centroid(obs: np.ndarray, grid) -> np.ndarray:
    """Per-axis circular mean of phi_c from lbcad_observables' cos/sin moments."""
    L = np.asarray(grid, dtype=float)
    ang = np.arctan2(obs[8:11], obs[5:8])
    return np.mod(ang, 2 * np.pi) * L / (2 * np.pi)


def unwrap_trajectory(xs: np.ndarray, grid) -> np.ndarray:
    """Minimum-image unwrapping of a periodic centroid trajectory (T, 3)."""
    L = np.asarray(grid, dtype=float)
    d = np.diff(xs, axis=0)
    d -= L * np.round(d / L)
    return np.vstack([xs[:1], xs[:1] + np.cumsum(d, axis=0)])


def mean_speed(traj: np.ndarray, dt: float) -> float:
    """Mean speed |dX|/dt along an unwrapped trajectory sampled every dt steps."""
    v = np.linalg.norm(np.diff(traj, axis=0), axis=1) / dt
    return float(v.mean())
