"""Shared helpers for the oracle pin tests: smooth periodic fields with analytic
derivatives, the paper's free energy (Eq. 5) in sympy, and cubic-group transforms of a
state.  Nothing here calls the CUDA library."""
from __future__ import annotations

import functools

import numpy as np


def mode_sum(shape, modes, h=1.0):
    """Sum of A sin(k.x + phase) over ``modes`` = [(A, (m0, m1, m2), phase)], with
    k = 2 pi m / (n h) on a grid of n = shape sites per axis and spacing h.
    Returns value (nz,ny,nx), gradient (3,...), Hessian (3,3,...)."""
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz) * h, np.arange(ny) * h, np.arange(nx) * h, indexing="ij")
    L = (nx * h, ny * h, nz * h)
    val = np.zeros((nz, ny, nx))
    grad = np.zeros((3, nz, ny, nx))
    hess = np.zeros((3, 3, nz, ny, nx))
    for A, m, ph in modes:
        k = [2 * np.pi * m[a] / L[a] for a in range(3)]
        arg = k[0] * x + k[1] * y + k[2] * z + ph
        s, c = np.sin(arg), np.cos(arg)
        val += A * s
        for a in range(3):
            grad[a] += A * k[a] * c
            for b in range(3):
                hess[a, b] -= A * k[a] * k[b] * s
    return val, grad, hess


def smooth_state(shape, h=1.0, seed=0, amp=0.12, psi0=0.2):
    """A generic smooth state: 5 Q components, psi, each a few low Fourier modes with
    seeded amplitudes and phases.  Returns dict with q5, dq5 (5,3,...), hq5 (5,3,3,...),
    psi, dpsi, hpsi."""
    rng = np.random.default_rng(seed)

    def rand_modes(a):
        out = []
        for _ in range(2):
            m = tuple(int(v) for v in rng.integers(-2, 3, size=3))
            if m == (0, 0, 0):
                m = (1, 0, 0)
            out.append((a * rng.uniform(0.5, 1.0), m, rng.uniform(0, 2 * np.pi)))
        return out

    q5, dq5, hq5 = [], [], []
    offs = [0.15, 0.05, -0.03, -0.08, 0.02]
    for c in range(5):
        v, g, hh = mode_sum(shape, rand_modes(amp), h)
        q5.append(v + offs[c]); dq5.append(g); hq5.append(hh)
    pv, pg, ph = mode_sum(shape, rand_modes(0.5), h)
    return dict(q5=np.array(q5), dq5=np.array(dq5), hq5=np.array(hq5),
                psi=pv + psi0, dpsi=pg, hpsi=ph)


def full_from5(a5):
    """(5, ...) stored-component layout -> (3, 3, ...) symmetric traceless tensor."""
    xx, xy, xz, yy, yz = a5
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, -xx - yy]])


def st(A):
    """Symmetric traceless part of (3,3,...) arrays."""
    S = 0.5 * (A + np.swapaxes(A, 0, 1))
    tr = (S[0, 0] + S[1, 1] + S[2, 2]) / 3.0
    for i in range(3):
        S[i, i] = S[i, i] - tr
    return S


@functools.lru_cache(maxsize=4)
def sympy_variational():
    """Euler-Lagrange expressions of the free energy of Eq. 5, written in the paper's
    form with phi = 1 + psi, phi0 = 2, phi_cr = 1 and the binary coefficient a_p = a/2:

        f = (a_p/2) phi^2 ((phi - phi0)/phi_cr)^2 + (k_phi/2)(grad phi)^2
            + A0 [ (1 - chi/3)/2 tr Q^2 - chi/3 tr Q^3 + chi/4 (tr Q^2)^2 ],  chi = chi0 + chis phi
            + (K/2) [ (div Q)^2 + (curl Q + 2 q0 Q)^2 ] + W grad phi . Q . grad phi,

    with Q treated as nine independent components.  Returns (args, E, mu) where E[i][j] =
    dF/dQ_ij and mu = dF/dpsi as lambdified numpy functions of args."""
    import sympy as sp

    q = [[sp.Symbol(f"q{i}{j}") for j in range(3)] for i in range(3)]
    dq = [[[sp.Symbol(f"dq{i}{j}_{k}") for k in range(3)] for j in range(3)] for i in range(3)]
    ddq = [[[[sp.Symbol(f"ddq{i}{j}_{k}{m}") for m in range(3)] for k in range(3)] for j in range(3)]
           for i in range(3)]
    p = sp.Symbol("p")
    dp = [sp.Symbol(f"dp_{k}") for k in range(3)]
    ddp = [[sp.Symbol(f"ddp_{k}{m}") for m in range(3)] for k in range(3)]
    a, b, kphi, A0, chi0, chis, K, q0, W = sp.symbols("a b kphi A0 chi0 chis K q0 W")

    phi = 1 + p
    a_p = a / 2
    f = a_p / 2 * phi ** 2 * ((phi - 2) / 1) ** 2
    f += kphi / 2 * sum(dp[k] ** 2 for k in range(3))
    Q = sp.Matrix(3, 3, lambda i, j: q[i][j])
    chi = chi0 + chis * phi
    trQ2 = (Q * Q).trace()
    trQ3 = (Q * Q * Q).trace()
    f += A0 * (sp.Rational(1, 2) * (1 - chi / 3) * trQ2 - chi / 3 * trQ3 + chi / 4 * trQ2 ** 2)
    eps = sp.LeviCivita
    divQ = [sum(dq[a_][b_][b_] for b_ in range(3)) for a_ in range(3)]  # d_b Q_ab
    curl = [[sum(eps(a_, m, n) * dq[n][b_][m] for m in range(3) for n in range(3))
             for b_ in range(3)] for a_ in range(3)]                     # eps_amn d_m Q_nb
    f += K / 2 * (sum(v ** 2 for v in divQ) +
                  sum((curl[a_][b_] + 2 * q0 * q[a_][b_]) ** 2 for a_ in range(3) for b_ in range(3)))
    f += W * sum(dp[a_] * q[a_][b_] * dp[b_] for a_ in range(3) for b_ in range(3))

    def Dk(g, k):
        """Total derivative d/dx_k of an expression in the field symbols."""
        out = sp.diff(g, p) * dp[k]
        out += sum(sp.diff(g, dp[m]) * ddp[m][k] for m in range(3))
        for i in range(3):
            for j in range(3):
                out += sp.diff(g, q[i][j]) * dq[i][j][k]
                out += sum(sp.diff(g, dq[i][j][m]) * ddq[i][j][m][k] for m in range(3))
        return out

    E = [[sp.diff(f, q[i][j]) - sum(Dk(sp.diff(f, dq[i][j][k]), k) for k in range(3))
          for j in range(3)] for i in range(3)]
    mu = sp.diff(f, p) - sum(Dk(sp.diff(f, dp[k]), k) for k in range(3))

    flat = ([q[i][j] for i in range(3) for j in range(3)] +
            [dq[i][j][k] for i in range(3) for j in range(3) for k in range(3)] +
            [ddq[i][j][k][m] for i in range(3) for j in range(3) for k in range(3) for m in range(3)] +
            [p] + dp + [ddp[k][m] for k in range(3) for m in range(3)] +
            [a, b, kphi, A0, chi0, chis, K, q0, W])
    fE = sp.lambdify(flat, [E[i][j] for i in range(3) for j in range(3)], "numpy")
    fmu = sp.lambdify(flat, mu, "numpy")
    return fE, fmu


def analytic_H_mu(st_, prm):
    """H = -ST(dF/dQ) and mu = dF/dpsi for the analytic smooth state ``st_``."""
    fE, fmu = sympy_variational()
    Q = full_from5(st_["q5"])
    dQ = full_from5(st_["dq5"])            # dQ[i, j, k] = d_k Q_ij
    hQ = full_from5(st_["hq5"])            # hQ[i, j, k, m] = d_k d_m Q_ij
    args = ([Q[i, j] for i in range(3) for j in range(3)] +
            [dQ[i, j, k] for i in range(3) for j in range(3) for k in range(3)] +
            [hQ[i, j, k, m] for i in range(3) for j in range(3) for k in range(3) for m in range(3)] +
            [st_["psi"]] + [st_["dpsi"][k] for k in range(3)] +
            [st_["hpsi"][k, m] for k in range(3) for m in range(3)] +
            [prm[k] for k in ("a", "b", "kphi", "A0", "chi0", "chis", "K", "q0", "W")])
    shp = st_["psi"].shape
    E = np.array([np.broadcast_to(e, shp) for e in fE(*args)]).reshape((3, 3) + shp)
    mu = np.broadcast_to(fmu(*args), shp)
    return -st(E), np.array(mu)


def spectral_grad(g, h=1.0):
    """Exact derivative of a periodic grid function in its Fourier representation."""
    nz, ny, nx = g.shape
    G = np.fft.fftn(g)
    out = []
    for ax, n in ((2, nx), (1, ny), (0, nz)):
        k = 2 * np.pi * np.fft.fftfreq(n, d=h)
        shp = [1, 1, 1]
        shp[ax] = n
        out.append(np.real(np.fft.ifftn(1j * k.reshape(shp) * G)))
    return np.array(out)  # (3, ...) in x, y, z order


# ---- cubic-group transforms of an oracle state -------------------------------------------

def transform_state(f, q5, psi, u, P, c19):
    """Apply the signed permutation matrix P (r' = P r mod n) to a state on a cubic box."""
    nz, ny, nx = psi.shape
    assert nx == ny == nz
    n = nx
    Z, Y, X = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    R = np.stack([X, Y, Z])
    Rp = np.einsum("ab,b...->a...", P, R) % n
    idx = (Rp[2], Rp[1], Rp[0])

    def scal(a):
        out = np.empty_like(a)
        out[idx] = a
        return out

    psi2 = scal(psi)
    u2 = np.einsum("ab,b...->a...", P, u)
    u2 = np.array([scal(c) for c in u2])
    Q = full_from5(q5)
    Q2 = np.einsum("ai,ij...,bj->ab...", P, Q, P)
    Q2 = np.array([scal(Q2[0, 0]), scal(Q2[0, 1]), scal(Q2[0, 2]), scal(Q2[1, 1]), scal(Q2[1, 2])])
    f2 = np.empty_like(f)
    for j in range(19):
        cj = P @ c19[j]
        i = int(np.where((c19 == cj).all(axis=1))[0][0])
        f2[i] = scal(f[j])
    return f2, Q2, psi2, u2
