"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: closed forms of the
stencils, conservation laws of Eqs. 6-8, the Guo forcing moments, the viscosity of the
BGK scheme, the Landau-de Gennes transition at chi = 2.7 printed in Sec. 2, variational
derivatives of the free energy of Eq. 5 computed by sympy, the Ericksen (Noether)
identity for the passive stress, the Onsager reciprocity between the co-rotation term
of Eq. 2 and the reactive stress, and the symmetries of the model.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from tests import oracle_helpers as OH

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split()
        out[k] = float(v)
    return out


# ---------------------------------------------------------------- stencils (Sec. 3)

@pytest.mark.parametrize("shape", [(4, 4, 4), (5, 6, 7)])
def test_stencil_fourier_symbols(shape):
    """On exp(i k.x) the isotropic D3Q19 stencils act as their Fourier symbols:
    grad_a -> i (sin k_a / 3)(1 + sum_{b != a} cos k_b),
    lap    -> (2/3) sum_a (cos k_a - 1) + (2/3) sum_{a<b} (cos k_a cos k_b - 1),
    hess_aa -> 2 cos k_a - 2, hess_ab -> -sin k_a sin k_b."""
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for m in [(1, 0, 0), (0, 1, 1), (1, 2, 3), (2, -1, 1)]:
        k = [2 * np.pi * m[0] / nx, 2 * np.pi * m[1] / ny, 2 * np.pi * m[2] / nz]
        arg = k[0] * x + k[1] * y + k[2] * z
        for part, fn in (("re", np.cos), ("im", np.sin)):
            s = fn(arg)
            g, lap, h = O.stencils(s)
            c = [np.cos(v) for v in k]
            sn = [np.sin(v) for v in k]
            # derivative of e^{i arg} is i*symbol*e^{i arg}; real/imag parts accordingly
            ds = -np.sin(arg) if part == "re" else np.cos(arg)
            for a in range(3):
                sym = sn[a] / 3.0 * (1 + sum(c[b] for b in range(3) if b != a))
                np.testing.assert_allclose(g[a], sym * ds, atol=1e-13)
            lsym = (2 / 3) * sum(ci - 1 for ci in c) + (2 / 3) * sum(
                c[a] * c[b] - 1 for a in range(3) for b in range(a + 1, 3))
            np.testing.assert_allclose(lap, lsym * s, atol=1e-13)
            for a in range(3):
                for b in range(3):
                    hs = (2 * c[a] - 2) if a == b else -sn[a] * sn[b]
                    np.testing.assert_allclose(h[3 * a + b], hs * s, atol=1e-13)


def test_stencils_exact_on_quadratics():
    """Away from the periodic seam, gradient/Laplacian/Hessian are exact on quadratics."""
    n = 9
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    s = 0.3 * x * x - 0.7 * x * y + 0.2 * z * z + 1.1 * y * z + 0.5 * x - 2 * y + 0.25 * z + 3.0
    g, lap, h = O.stencils(s.astype(np.float64))
    sl = (slice(1, n - 1),) * 3
    np.testing.assert_allclose(g[0][sl], (0.6 * x - 0.7 * y + 0.5)[sl], atol=1e-12)
    np.testing.assert_allclose(g[1][sl], (-0.7 * x + 1.1 * z - 2)[sl], atol=1e-12)
    np.testing.assert_allclose(g[2][sl], (0.4 * z + 1.1 * y + 0.25)[sl], atol=1e-12)
    np.testing.assert_allclose(lap[sl], 0.6 + 0.4, atol=1e-12)
    H = np.array([[0.6, -0.7, 0.0], [-0.7, 0.0, 1.1], [0.0, 1.1, 0.4]])
    for a in range(3):
        for b in range(3):
            np.testing.assert_allclose(h[3 * a + b][sl], H[a, b], atol=1e-12)


@pytest.mark.parametrize("shape", [(5, 5, 5), (6, 7, 9)])
def test_radius2_stencil_fourier_symbols(shape):
    """The fourth-order radius-2 set (the other reading of Sec. 3) on exp(i k.x):
    d_a -> i (8 sin k_a - sin 2k_a)/6, d_aa -> (16 cos k_a - cos 2k_a - 15)/6, Laplacian = sum of
    the d_aa, d_a d_b -> -(8 sin k_a - sin 2k_a)(8 sin k_b - sin 2k_b)/36 for a != b."""
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for m in [(1, 0, 0), (0, 1, 1), (1, 2, 3), (2, -1, 1)]:
        k = [2 * np.pi * m[0] / nx, 2 * np.pi * m[1] / ny, 2 * np.pi * m[2] / nz]
        arg = k[0] * x + k[1] * y + k[2] * z
        d1 = [(8 * np.sin(v) - np.sin(2 * v)) / 6 for v in k]
        d2 = [(16 * np.cos(v) - np.cos(2 * v) - 15) / 6 for v in k]
        for part, fn in (("re", np.cos), ("im", np.sin)):
            s = fn(arg)
            g, lap, h = O.stencils(s, stencil=1)
            ds = -np.sin(arg) if part == "re" else np.cos(arg)
            for a in range(3):
                np.testing.assert_allclose(g[a], d1[a] * ds, atol=1e-13)
            np.testing.assert_allclose(lap, sum(d2) * s, atol=1e-13)
            for a in range(3):
                for b in range(3):
                    hs = d2[a] if a == b else -d1[a] * d1[b]
                    np.testing.assert_allclose(h[3 * a + b], hs * s, atol=1e-13)


def test_radius2_stencils_exact_on_quartics():
    """Away from the periodic seam, the radius-2 gradient, Laplacian and Hessian are exact on
    polynomials of degree four (the isotropic set is exact only up to degree two)."""
    n = 13
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    x, y, z = (v.astype(float) / n for v in (x, y, z))
    s = 0.3 * x ** 4 - 0.7 * x ** 2 * y ** 2 + 0.2 * z ** 3 * y + 1.1 * x * y * z + 0.5 * y ** 4 - 2 * z + 3.0
    gx = 1.2 * x ** 3 - 1.4 * x * y ** 2 + 1.1 * y * z
    gy = -1.4 * x ** 2 * y + 0.2 * z ** 3 + 1.1 * x * z + 2.0 * y ** 3
    gz = 0.6 * z ** 2 * y + 1.1 * x * y - 2
    H = [[3.6 * x ** 2 - 1.4 * y ** 2, -2.8 * x * y + 1.1 * z, 1.1 * y],
         [-2.8 * x * y + 1.1 * z, -1.4 * x ** 2 + 6.0 * y ** 2, 0.6 * z ** 2 + 1.1 * x],
         [1.1 * y, 0.6 * z ** 2 + 1.1 * x, 1.2 * z * y]]
    g, lap, h = O.stencils(s, stencil=1)
    sl = (slice(2, n - 2),) * 3
    sc = [1.0 / n, 1.0 / n ** 2]  # grid spacing 1 in the index, x = index / n
    for a, ga in enumerate((gx, gy, gz)):
        np.testing.assert_allclose(g[a][sl], (ga * sc[0])[sl], atol=1e-12)
    np.testing.assert_allclose(lap[sl], ((H[0][0] + H[1][1] + H[2][2]) * sc[1])[sl], atol=1e-12)
    for a in range(3):
        for b in range(3):
            np.testing.assert_allclose(h[3 * a + b][sl], (H[a][b] * sc[1])[sl], atol=1e-12)
    gi, lapi, hi = O.stencils(s, stencil=0)
    assert np.abs(lapi[sl] - ((H[0][0] + H[1][1] + H[2][2]) * sc[1])[sl]).max() > 1e-6


# ---------------------------------------------------------------- LB (Eqs. 6-8, Guo forcing)

def _feq(rho, v, c, w):
    cu = np.einsum("ia,a...->i...", c, v)
    v2 = (v * v).sum(0)
    return w.reshape((len(w),) + (1,) * rho.ndim) * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * v2)


def test_lb_conservation_unforced():
    c, w = O.lattice()
    rng = np.random.default_rng(3)
    shp = (6, 5, 7)
    nx, ny, nz = shp
    f = w.reshape(19, 1, 1, 1) * (1 + 0.05 * rng.standard_normal((19, nz, ny, nx)))
    p = O.default_params(shp, tau=0.8)
    F = np.zeros((3, nz, ny, nx))
    fn, un = O.lb(f, F, p)
    assert abs(fn.sum() - f.sum()) < 1e-12 * f.sum()
    for a in range(3):
        m0 = np.tensordot(c[:, a].astype(float), f, axes=(0, 0)).sum()
        m1 = np.tensordot(c[:, a].astype(float), fn, axes=(0, 0)).sum()
        assert abs(m1 - m0) < 1e-12


def test_lb_rest_state_exact():
    c, w = O.lattice()
    shp = (4, 5, 6)
    f = np.broadcast_to(w.reshape(19, 1, 1, 1), (19, 6, 5, 4)).copy() * 1.3
    p = O.default_params(shp)
    fn, un = O.lb(f, np.zeros((3, 6, 5, 4)), p)
    assert np.abs(fn - f).max() < 4e-16  # one rounding of rho
    assert np.abs(un).max() == 0.0


@pytest.mark.parametrize("tau", [1.0, 0.8, 1.7])
def test_guo_forcing_moments(tau):
    """Uniform fluid, uniform force F: the collision adds exactly F to the momentum,
    u = (j + F/2)/rho, and the second moment of the forcing is (1 - 1/2tau)(uF + Fu)."""
    c, w = O.lattice()
    shp = (4, 4, 4)
    rho = 1.2 * np.ones((4, 4, 4))
    v = np.array([0.01, -0.02, 0.005]).reshape(3, 1, 1, 1) * np.ones((3, 4, 4, 4))
    F = np.array([1e-3, 2e-4, -5e-4]).reshape(3, 1, 1, 1) * np.ones((3, 4, 4, 4))
    f = _feq(rho, v, c, w)
    p = O.default_params(shp, tau=tau)
    fn, un = O.lb(f, F, p)
    u = v + F / (2 * rho)
    np.testing.assert_allclose(un, u, atol=1e-15)
    cf = c.astype(float)
    j1 = np.einsum("ia,i...->a...", cf, fn)
    np.testing.assert_allclose(j1, rho * v + F, atol=1e-15)
    np.testing.assert_allclose(fn.sum(0), rho, atol=1e-14)
    Pi1 = np.einsum("ia,ib,i...->ab...", cf, cf, fn)[:, :, 0, 0, 0]
    r, vv, uu, FF = rho[0, 0, 0], v[:, 0, 0, 0], u[:, 0, 0, 0], F[:, 0, 0, 0]
    expect = (r * (np.outer(vv, vv) + np.eye(3) / 3) - r * (np.outer(vv, vv) - np.outer(uu, uu)) / tau
              + (1 - 0.5 / tau) * (np.outer(uu, FF) + np.outer(FF, uu)))
    np.testing.assert_allclose(Pi1, expect, atol=1e-15)


def test_shear_wave_decay_matches_viscosity():
    """u_x = U sin(2 pi z / L) decays at nu k^2 with nu = (tau - 1/2)/3 (BGK)."""
    c, w = O.lattice()
    L = 32
    for tau in (1.0, 0.7):
        p = O.default_params((4, 4, L), tau=tau)
        z = np.arange(L).reshape(L, 1, 1) * np.ones((L, 4, 4))
        U = 1e-4
        v = np.zeros((3, L, 4, 4))
        v[0] = U * np.sin(2 * np.pi * z / L)
        f = _feq(np.ones((L, 4, 4)), v, c, w)
        F = np.zeros((3, L, 4, 4))
        amps = []
        nsteps = 200
        for t in range(nsteps + 1):
            fn, un = O.lb(f, F, p)
            amps.append(2 * np.mean(un[0] * np.sin(2 * np.pi * z / L)))
            f = fn
        amps = np.array(amps)
        ts = np.arange(nsteps + 1)
        rate = -np.polyfit(ts[20:], np.log(amps[20:]), 1)[0]
        nu = (tau - 0.5) / 3
        assert abs(rate / (nu * (2 * np.pi / L) ** 2) - 1) < 0.01


def test_full_step_reduces_to_lb_without_order():
    """With Q = 0, uniform psi and xi = 0 the hybrid step is the plain BGK LB step."""
    c, w = O.lattice()
    L = 16
    shp = (4, 4, L)
    p = O.default_params(shp, xi=0.0)
    s = O.State(shp, p)
    z = np.arange(L).reshape(L, 1, 1) * np.ones((L, 4, 4))
    v = np.zeros((3, L, 4, 4))
    v[0] = 1e-3 * np.sin(2 * np.pi * z / L)
    s.f = _feq(np.ones((L, 4, 4)), v, c, w)
    s.q[:] = 0.0
    s.psi[:] = 0.3
    s.u[:] = 0.0
    f_ref = s.f.copy()
    for _ in range(5):
        f_ref, _ = O.lb(f_ref, np.zeros((3, L, 4, 4)), p)
    s.step(5)
    np.testing.assert_allclose(s.f, f_ref, atol=1e-15)
    assert np.abs(s.q).max() == 0.0
    np.testing.assert_allclose(s.psi, 0.3, atol=1e-15)


# ---------------------------------------------------------------- Landau-de Gennes bulk (Eq. 5)

def _uniform_uniaxial(S, shp):
    n = np.array([0.6, 0.0, 0.8])
    Q = S * (np.outer(n, n) - np.eye(3) / 3)
    nx, ny, nz = shp
    q5 = np.array([Q[0, 0], Q[0, 1], Q[0, 2], Q[1, 1], Q[1, 2]]).reshape(5, 1, 1, 1) * np.ones((5, nz, ny, nx))
    return q5


@pytest.mark.parametrize("chi", [2.7, 2.8, 3.0, 3.5])
def test_ldg_equilibrium_order(chi):
    """With no gradients and no chirality, H = 0 at S = 0 and at
    S_eq = 1/4 + 3/4 sqrt(1 - 8/(3 chi)), the stationary points of the LdG bulk term."""
    shp = (4, 4, 4)
    p = O.default_params(shp, q0=0.0, chi0=chi - 0.5, chis=0.25)
    psi = np.ones((4, 4, 4))
    Seq = 0.25 + 0.75 * np.sqrt(1 - 8 / (3 * chi))
    for S, zero in ((0.0, True), (Seq, True), (Seq + 0.02, False), (0.7 * Seq, False)):
        out = O.fields(_uniform_uniaxial(S, shp), psi, p)
        hmax = np.abs(out["H"]).max()
        if zero:
            assert hmax < 1e-14, (chi, S, hmax)
        else:
            assert hmax > 1e-4


def test_ldg_transition_at_paper_threshold():
    """Sec. 2 states the LC phase is confined where chi > 2.7.  For the LdG bulk term this
    is the first-order transition: at chi = 2.7 the ordered stationary state (S = 1/3)
    has the same free energy as the isotropic one; above it, it is lower; below, higher."""
    thr = _golden("paper_constants.txt")["chi_threshold"]
    shp = (4, 4, 4)
    psi = np.ones((4, 4, 4))
    for chi, sign in ((thr, 0), (thr + 0.05, -1), (thr - 0.02, +1)):
        p = O.default_params(shp, q0=0.0, chi0=chi - 0.5, chis=0.25)
        Seq = 0.25 + 0.75 * np.sqrt(1 - 8 / (3 * chi))
        out = O.fields(_uniform_uniaxial(Seq, shp), psi, p)
        fd = out["fden"][0, 0, 0]
        f0 = O.fields(_uniform_uniaxial(0.0, shp), psi, p)["fden"][0, 0, 0]
        if sign == 0:
            assert abs(Seq - 1 / 3) < 1e-12
            assert abs(fd - f0) < 1e-14
            assert np.abs(out["H"]).max() < 1e-14
        else:
            assert np.sign(fd - f0) == sign


# ---------------------------------------------------------------- H and mu = variational derivatives of Eq. 5

def _scaled_params(base, h):
    """Lattice parameters that represent grid spacing h in lattice units (dx = 1)."""
    p = O.default_params((4, 4, 4))
    for k, v in base.items():
        setattr(p, k, v)
    p.K = base["K"] / h ** 2
    p.q0 = base["q0"] * h
    p.W = base["W"] / h ** 2
    p.kphi = base["kphi"] / h ** 2
    return p


BASE = dict(a=0.07, b=0.07, kphi=0.14, A0=1.0, chi0=2.5, chis=0.25, K=0.04, q0=2 * np.pi / 16,
            W=0.1, xi=0.7, zeta=0.0)


@pytest.mark.parametrize("stencil,order", [(0, 2), (1, 4)])
def test_H_mu_are_variational_derivatives_of_eq5(stencil, order):
    """The oracle's H and mu converge to -dF/dQ (traceless-symmetric) and dF/dpsi of the free
    energy of Eq. 5 as written in the paper (curl form of the chiral term, binary term in phi
    with phi0 = 2), differentiated by sympy: at second order with the isotropic radius-1
    stencils, at fourth order with the radius-2 set."""
    Lp = 16.0
    errs_H, errs_mu = [], []
    for n in (16, 32, 64):
        h = Lp / n
        st_ = OH.smooth_state((n, n, n), h=h, seed=5)
        H_a, mu_a = OH.analytic_H_mu(st_, BASE)
        prm = _scaled_params(BASE, h)
        prm.stencil = stencil
        out = O.fields(np.ascontiguousarray(st_["q5"]), np.ascontiguousarray(st_["psi"]), prm)
        H_o = OH.full_from5(out["H"])
        errs_H.append(np.abs(H_o - H_a).max() / np.abs(H_a).max())
        errs_mu.append(np.abs(out["mu"] - mu_a).max() / np.abs(mu_a).max())
    # each halving of h cuts the error by ~2^order
    lo = 0.8 * 2 ** order
    for e in (errs_H, errs_mu):
        assert e[2] < 0.02, e
        assert e[1] / e[2] > lo and e[0] / e[1] > 0.75 * 2 ** order, e


def test_helix_minimises_chiral_energy():
    """The sign of q0: n = (cos q0 z, sin q0 z, 0) has no oscillating curl-energy
    (curl Q + 2 q0 Q has no 2q0 Fourier component), the opposite twist does."""
    n = 64
    h = 16.0 / n
    q0 = BASE["q0"]
    z = np.arange(n) * h
    for sgn, small in ((1, True), (-1, False)):
        th = sgn * q0 * z
        S = 0.5
        nn = np.array([np.cos(th), np.sin(th), 0 * th])
        Q = S * (np.einsum("a...,b...->ab...", nn, nn) - np.eye(3).reshape(3, 3, 1) / 3)
        q5 = np.array([Q[0, 0], Q[0, 1], Q[0, 2], Q[1, 1], Q[1, 2]]).reshape(5, n, 1, 1) * np.ones((5, n, 4, 4))
        q5 = np.ascontiguousarray(q5)
        p = _scaled_params(dict(BASE, W=0.0), h)
        p.chi0, p.chis = 2.5, 0.25
        out = O.fields(q5, np.ones((n, 4, 4)), p)
        # oscillating (xx-yy, xy) part of H at the helix wavevector
        osc = np.abs(out["H"][1]).max()
        if small:
            assert osc < 2e-3 * 4 * BASE["K"] * q0 ** 2 * S * 1e2
        else:
            assert osc > 0.5 * 4 * BASE["K"] * (2 * q0) ** 2 * S * 0.5


# ---------------------------------------------------------------- stresses (Eq. 3, Eq. 4)

def test_ericksen_identity_for_passive_stress():
    """Translation invariance of Eq. 5 (Noether): div of the pressure + elastic + interface
    stress equals -psi grad mu - H : grad Q, at second order in the grid spacing."""
    Lp = 16.0
    errs = []
    for n in (16, 32, 64):
        h = Lp / n
        st_ = OH.smooth_state((n, n, n), h=h, seed=11)
        out = O.fields(np.ascontiguousarray(st_["q5"]), np.ascontiguousarray(st_["psi"]), _scaled_params(BASE, h))
        sE = out["sE"].reshape(3, 3, n, n, n)
        div = np.zeros((3, n, n, n))
        for a in range(3):
            for b in range(3):
                div[a] += OH.spectral_grad(sE[a, b], h)[b]
        gmu = OH.spectral_grad(out["mu"], h)
        H = OH.full_from5(out["H"])
        Q = OH.full_from5(st_["q5"])
        dQ = np.array([[OH.spectral_grad(Q[i, j], h) for j in range(3)] for i in range(3)])  # [i,j,a]
        rhs = -st_["psi"] * gmu - np.einsum("ij...,ija...->a...", H, dQ)
        errs.append(np.abs(div - rhs).max() / np.abs(rhs).max())
    assert errs[2] < 0.02, errs
    assert errs[1] / errs[2] > 3.0, errs


def test_onsager_reciprocity_reactive_stress():
    """The flow-coupling of Eq. 2 and the reactive stress are Onsager partners:
    H : S(W, Q) + sigma_R : W = 0 for every traceless velocity gradient W (W_ab = d_b u_a)."""
    n = 8
    st_ = OH.smooth_state((n, n, n), seed=2)
    p = O.default_params((n, n, n), xi=0.7)
    out = O.fields(np.ascontiguousarray(st_["q5"]), np.ascontiguousarray(st_["psi"]), p)
    H = OH.full_from5(out["H"])
    Q = OH.full_from5(st_["q5"])
    sR = out["sR"].reshape(3, 3, n, n, n)
    rng = np.random.default_rng(0)
    for _ in range(40):
        z, y, x = rng.integers(0, n, size=3)
        W = rng.standard_normal((3, 3))
        W -= np.eye(3) * np.trace(W) / 3
        S = O.corotation(W, Q[:, :, z, y, x], 0.7)
        lhs = np.sum(H[:, :, z, y, x] * S) + np.sum(sR[:, :, z, y, x] * W)
        scale = np.abs(H[:, :, z, y, x]).max() * np.abs(W).max()
        assert abs(lhs) < 1e-13 * max(scale, 1.0)
        # symmetric part is traceless; antisymmetric part is Q H - H Q
        assert abs(np.trace(sR[:, :, z, y, x])) < 1e-14
        Hs, Qs = H[:, :, z, y, x], Q[:, :, z, y, x]
        np.testing.assert_allclose(sR[:, :, z, y, x] - sR[:, :, z, y, x].T, 2 * (Qs @ Hs - Hs @ Qs), atol=1e-14)


def test_corotation_closed_forms():
    """The co-rotation term of Eq. 2 in two limits that fix it apart from the stress: a pure
    rotation of the flow (W antisymmetric, so D = 0 and tr(QW) = 0) rotates Q, S = Omega Q -
    Q Omega; a pure strain acting on the isotropic phase (Q = 0) gives S = 2 xi D / 3."""
    rng = np.random.default_rng(11)
    for xi in (0.7, -0.4):
        for _ in range(10):
            A = rng.standard_normal((3, 3))
            Q = 0.5 * (A + A.T)
            Q -= np.eye(3) * np.trace(Q) / 3
            B = rng.standard_normal((3, 3))
            Om = 0.5 * (B - B.T)
            np.testing.assert_allclose(O.corotation(Om, Q, xi), Om @ Q - Q @ Om, atol=1e-14)
            D = 0.5 * (B + B.T)
            D -= np.eye(3) * np.trace(D) / 3
            np.testing.assert_allclose(O.corotation(D, np.zeros((3, 3)), xi), 2 * xi * D / 3, atol=1e-14)


def test_active_stress_eq4():
    """Eq. 4: sigma_act = -zeta Q inside the droplet (phi_c = 1), zero outside."""
    n = 4
    st_ = OH.smooth_state((n, n, n), seed=4)
    for psi_v, phic in ((1.0, 1.0), (-1.0, 0.0), (0.0, 0.5)):
        p = O.default_params((n, n, n), zeta=0.01)
        out = O.fields(np.ascontiguousarray(st_["q5"]), np.full((n, n, n), psi_v), p)
        Q = OH.full_from5(st_["q5"]).reshape(9, n, n, n)
        np.testing.assert_allclose(out["sA"], -0.01 * phic * Q, atol=1e-16)


def test_force_is_divergence_of_total_stress():
    n = 6
    st_ = OH.smooth_state((n, n, n), seed=8)
    p = O.default_params((n, n, n))
    out = O.fields(np.ascontiguousarray(st_["q5"]), np.ascontiguousarray(st_["psi"]), p)
    np.testing.assert_allclose(out["sigma"], out["sE"] + out["sR"] + out["sA"], atol=1e-15)
    F = O.force(out["sigma"])
    s9 = out["sigma"].reshape(3, 3, n, n, n)
    ref = np.zeros((3, n, n, n))
    for a in range(3):
        for b in range(3):
            ref[a] += O.stencils(np.ascontiguousarray(s9[a, b]))[0][b]
    np.testing.assert_allclose(F, ref, atol=1e-15)
    # a telescoping divergence: total force vanishes
    assert np.abs(F.sum(axis=(1, 2, 3))).max() < 1e-13


def _grad_symbol(k, stencil):
    """Symbol of the gradient stencils on cos(k.x + ph): d_b -> -s_b(k) sin(k.x + ph), written
    out from the stencil definitions of Sec. 3 (not from the oracle's tables).
    Isotropic D3Q19 (stencil 0): 3 sum_i w_i c_ib sin(k.c_i) = sin(k_b)(1 + cos k_c + cos k_d)/3 with
    c, d the other two axes (two faces of weight 1/18, eight edges of weight 1/36).  Fourth-order
    radius-2 differences (stencil 1): (8 sin k_b - sin 2k_b)/6."""
    if stencil == 1:
        return [(8 * np.sin(k[b]) - np.sin(2 * k[b])) / 6 for b in range(3)]
    return [np.sin(k[b]) * (1 + np.cos(k[(b + 1) % 3]) + np.cos(k[(b + 2) % 3])) / 3 for b in range(3)]


def _distinct_modes(rng, count, shape):
    """count wave vectors with every component nonzero and no two alike."""
    seen, out = set(), []
    while len(out) < count:
        m = tuple(int(v) for v in rng.integers(1, 3, size=3) * rng.choice([-1, 1], size=3))
        if m not in seen:
            seen.add(m)
            out.append([2 * np.pi * m[a] / shape[a] for a in range(3)])
    return out


@pytest.mark.parametrize("stencil", [0, 1])
def test_force_symbols_fix_the_divergence_index(stencil):
    """F_a = d_b sigma_ab (Sec. 3 stress divergence) on sigma_ab = A_ab cos(k_ab . x + ph_ab), each
    component with its own wave vector, against the closed-form symbols of both stencil sets.
    The index swaps F_a = d_b sigma_ba and F_a = d_a sigma_ab, and a sign error in either
    difference, give O(1) differences here (asserted), so each would fail."""
    shape = (8, 10, 12)
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    rng = np.random.default_rng(31 + stencil)
    ks = _distinct_modes(rng, 9, shape)
    A = rng.uniform(0.5, 1.5, size=9)
    ph = rng.uniform(0, 2 * np.pi, size=9)
    theta = [ks[c][0] * x + ks[c][1] * y + ks[c][2] * z + ph[c] for c in range(9)]
    sig = np.array([A[c] * np.cos(theta[c]) for c in range(9)])
    F = O.force(np.ascontiguousarray(sig), stencil=stencil)

    def div(index):
        out = np.zeros((3, nz, ny, nx))
        for a in range(3):
            for b in range(3):
                c, d = index(a, b)
                out[a] += -A[c] * _grad_symbol(ks[c], stencil)[d] * np.sin(theta[c])
        return out

    exp = div(lambda a, b: (3 * a + b, b))
    np.testing.assert_allclose(F, exp, atol=1e-13)
    for wrong in (lambda a, b: (3 * b + a, b), lambda a, b: (3 * a + b, a)):
        assert np.abs(div(wrong) - exp).max() > 1e-2


@pytest.mark.parametrize("stencil", [0, 1])
def test_velocity_gradient_symbols_fix_its_orientation(stencil):
    """The co-rotation term of Eq. 2 takes W_ab = d_b u_a.  On u_a = B_a sin(k_a . x + ph_a), each
    component with its own wave vector, W_ab = B_a s_b(k_a) cos(k_a . x + ph_a) with the closed-form
    symbols of both stencil sets.  A transposed W (d_a u_b) differs at O(1) (asserted)."""
    shape = (8, 10, 12)
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    rng = np.random.default_rng(41 + stencil)
    ks = _distinct_modes(rng, 3, shape)
    Bm = rng.uniform(1e-3, 2e-3, size=3)
    ph = rng.uniform(0, 2 * np.pi, size=3)
    theta = [ks[a][0] * x + ks[a][1] * y + ks[a][2] * z + ph[a] for a in range(3)]
    u = np.ascontiguousarray(np.array([Bm[a] * np.sin(theta[a]) for a in range(3)]))
    p = O.default_params(shape, stencil=stencil)
    zero = np.zeros((nz, ny, nx))
    _, _, W = O.op_rhs(np.zeros((5, nz, ny, nx)), zero, u, np.zeros((5, nz, ny, nx)), zero, p)
    W = W.reshape(3, 3, nz, ny, nx)
    exp = np.array([[Bm[a] * _grad_symbol(ks[a], stencil)[b] * np.cos(theta[a]) for b in range(3)]
                    for a in range(3)])
    np.testing.assert_allclose(W, exp, atol=1e-16)
    assert np.abs(np.swapaxes(exp, 0, 1) - exp).max() > 1e-4


# ---------------------------------------------------------------- the order-parameter update

def test_upwind_exact_for_linear_profiles():
    """First-order upwind advection is exact on linear profiles with uniform u; the
    upwind flux form conserves psi."""
    n = 8
    p = O.default_params((n, n, n), gammaQ=0.0, M=0.0, xi=0.0)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    q5 = np.zeros((5, n, n, n))
    q5[1] = 0.01 * x + 0.02 * y - 0.01 * z
    psi = 0.05 * y
    for uu in ([0.01, -0.02, 0.005], [-0.01, 0.02, -0.005]):
        u = np.array(uu).reshape(3, 1, 1, 1) * np.ones((3, n, n, n))
        H = np.zeros((5, n, n, n))
        mu = np.zeros((n, n, n))
        rq, rp, W = O.op_rhs(q5, psi, u, H, mu, p)
        sl = (slice(1, n - 1),) * 3
        np.testing.assert_allclose(rq[1][sl], -(0.01 * uu[0] + 0.02 * uu[1] - 0.01 * uu[2]), atol=1e-15)
        np.testing.assert_allclose(rp[sl], -0.05 * uu[1], atol=1e-15)
        assert np.abs(W).max() < 1e-17
        assert abs(rp.sum()) < 1e-14


def test_relaxation_and_diffusion_terms():
    """At rest (u = 0) the right-hand side of Eq. 2 is Gamma_Q H and that of Eq. 1 is M lap mu.
    For mu = cos(k x) the isotropic D3Q19 Laplacian 6 sum_i w_i (mu(x + c_i) - mu(x)) has the
    exact symbol 6 (2/18 + 8/36)(cos k - 1) = 2 (cos k - 1): the two faces along x and the eight
    edges with c_x != 0; every other neighbour sees the same mu."""
    n = 8
    p = O.default_params((n, n, n), gammaQ=0.3, M=0.1)
    rng = np.random.default_rng(5)
    q5 = 0.1 * rng.standard_normal((5, n, n, n))
    psi = 0.2 * rng.standard_normal((n, n, n))
    H = rng.standard_normal((5, n, n, n))
    kx = 2 * np.pi * 3 / n
    for axis in range(3):
        r = np.arange(n, dtype=float)
        shape_a = [1, 1, 1]
        shape_a[2 - axis] = n
        mu = np.ascontiguousarray(np.broadcast_to(np.cos(kx * r).reshape(shape_a), (n, n, n)))
        rq, rp, W = O.op_rhs(q5, psi, np.zeros((3, n, n, n)), H, mu, p)
        np.testing.assert_allclose(rq, 0.3 * H, atol=1e-15)
        np.testing.assert_allclose(rp, 0.1 * 2 * (np.cos(kx) - 1) * mu, atol=1e-14)
        assert np.abs(W).max() == 0.0


# ---------------------------------------------------------------- full step: conservation and symmetry

def _droplet_state(n=16, R=5.0, **kw):
    p = O.default_params((n, n, n), R=R, p0=8.0, **kw)
    return O.State((n, n, n), p, seed=1)


def _sums(s):
    import math
    c, _ = O.lattice(s.f.shape[0])
    mom = [math.fsum(np.tensordot(c[:, a].astype(float), s.f, axes=(0, 0)).ravel()) for a in range(3)]
    return math.fsum(s.f.ravel()), math.fsum(s.psi.ravel()), np.array(mom)


def test_full_step_conserves_mass_psi_momentum():
    """Eqs. 6-8 with Guo forcing conserve mass; the total force is a telescoping sum, so
    momentum is conserved too; the Cahn-Hilliard flux form conserves psi (Eq. 1)."""
    s = _droplet_state(zeta=0.01)
    m0, p0_, j0 = _sums(s)
    s.step(20)
    m1, p1, j1 = _sums(s)
    N = 16 ** 3
    assert abs(m1 - m0) < 1e-14 * N
    assert abs(p1 - p0_) < 1e-14 * N
    assert np.abs(j1 - j0).max() < 1e-15 * N
    assert np.abs(s.u).max() > 1e-6  # the droplet does drive a flow


def test_heun_sync_and_lb_variants_conserve():
    for kw in (dict(integrator=1), dict(coupling=1), dict(lb_form=1), dict(lattice=15),
               dict(lattice=15, lb_form=1, integrator=1, coupling=1), dict(stencil=1)):
        s = _droplet_state(n=12, R=4.0, **kw)
        m0, p0_, j0 = _sums(s)
        s.step(5)
        m1, p1, j1 = _sums(s)
        assert abs(p1 - p0_) < 1e-14 * 12 ** 3, kw
        assert abs(m1 - m0) < 1e-14 * 12 ** 3, kw
        # every force here is a telescoping difference (radius 1 or 2), so momentum is conserved
        # too; a one-sided or non-antisymmetric radius-2 difference would break this
        assert np.abs(j1 - j0).max() < 1e-14 * 12 ** 3, kw
        assert np.abs(s.u).max() > 1e-7, kw


# ---------------------------------------------------------------- D3Q15 and the stress-in-equilibrium form (Eqs. 9-11)

@pytest.mark.parametrize("q", [15, 19])
def test_velocity_sets_are_isotropic(q):
    """D3Q15 (Sec. 3, Fig. 1: rest, 6 faces, 8 corners; weights 2/9, 1/9, 1/72) and D3Q19
    carry the moment conditions that make BGK recover Navier-Stokes: sum w = 1, odd moments
    zero, sum w c c = I/3, sum w c c c c = (1/9)(dd + dd + dd).  Opposite velocities sit in
    adjacent slots."""
    c, w = O.lattice(q)
    cf = c.astype(float)
    assert len({tuple(v) for v in c}) == q and (c[0] == 0).all()
    assert abs(w.sum() - 1) < 1e-15
    np.testing.assert_allclose(np.einsum("i,ia->a", w, cf), 0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, cf, cf), np.eye(3) / 3, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic->abc", w, cf, cf, cf), 0, atol=1e-16)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic,id->abcd", w, cf, cf, cf, cf), iso, atol=1e-16)
    for i in range(1, q, 2):
        assert (c[i] == -c[i + 1]).all()


def test_d3q15_shear_wave_decay_matches_viscosity():
    """The D3Q15 BGK scheme has the same viscosity nu = (tau - 1/2)/3 as D3Q19."""
    c, w = O.lattice(15)
    L = 32
    for tau in (1.0, 0.7):
        p = O.default_params((4, 4, L), tau=tau, lattice=15)
        z = np.arange(L).reshape(L, 1, 1) * np.ones((L, 4, 4))
        v = np.zeros((3, L, 4, 4))
        v[0] = 1e-4 * np.sin(2 * np.pi * z / L)
        f = _feq(np.ones((L, 4, 4)), v, c, w)
        F = np.zeros((3, L, 4, 4))
        amps = []
        for t in range(201):
            f, un = O.lb(f, F, p)
            amps.append(2 * np.mean(un[0] * np.sin(2 * np.pi * z / L)))
        rate = -np.polyfit(np.arange(20, 201), np.log(np.array(amps[20:])), 1)[0]
        assert abs(rate / ((tau - 0.5) / 3 * (2 * np.pi / L) ** 2) - 1) < 0.01


@pytest.mark.parametrize("q", [15, 19])
@pytest.mark.parametrize("tau", [1.0, 0.7])
def test_stress_form_moments(q, tau):
    """Eqs. 8-10 for the form with the symmetric stress in the equilibrium.  For a uniform
    state with arbitrary populations f, stress sigma and antisymmetric force FA, one collision
    (streaming a uniform state changes nothing) gives sum f* = rho, sum f* c = rho u + FA with
    rho u = sum f c, and sum f* c c = P_f - (P_f - (rho/3 I + rho u u - sigma^S))/tau with
    P_f = sum f c c: the equilibrium moment of Eq. 9 with the lattice pressure rho c_s^2 and
    forcing moments 0, FA, 0 (Eq. 10)."""
    c, w = O.lattice(q)
    cf = c.astype(float)
    rng = np.random.default_rng(q + int(10 * tau))
    shp = (4, 4, 4)
    f0 = w * (1 + 0.1 * rng.standard_normal(q))
    sig = 1e-2 * rng.standard_normal(9)
    FA = 1e-3 * rng.standard_normal(3)
    one = np.ones((4, 4, 4))
    p = O.default_params(shp, tau=tau, lattice=q, lb_form=1)
    fn, un = O.lb_stress(f0.reshape(q, 1, 1, 1) * one, FA.reshape(3, 1, 1, 1) * one,
                         sig.reshape(9, 1, 1, 1) * one, p)
    assert np.abs(fn - fn[:, :1, :1, :1]).max() < 1e-17
    g = fn[:, 0, 0, 0]
    rho, j = f0.sum(), cf.T @ f0
    u = j / rho
    S = sig.reshape(3, 3)
    Peq = rho / 3 * np.eye(3) + rho * np.outer(u, u) - 0.5 * (S + S.T)
    Pf = np.einsum("i,ia,ib->ab", f0, cf, cf)
    assert abs(g.sum() - rho) < 1e-15
    np.testing.assert_allclose(cf.T @ g, j + FA, atol=1e-16)
    np.testing.assert_allclose(un[:, 0, 0, 0], u, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", g, cf, cf), Pf - (Pf - Peq) / tau, atol=2e-16)


@pytest.mark.parametrize("q", [15, 19])
def test_lb_forms_agree_without_stress(q):
    """With Q = 0, psi = 0 and xi = 0 the stress vanishes (mu = 0, f = 0, H = 0) and no order
    is generated by the shear: both LB forms reduce to the same unforced BGK step, which the
    LB stage alone reproduces."""
    c, w = O.lattice(q)
    L = 16
    shp = (4, 4, L)
    z = np.arange(L).reshape(L, 1, 1) * np.ones((L, 4, 4))
    v = np.zeros((3, L, 4, 4))
    v[0] = 1e-3 * np.sin(2 * np.pi * z / L)
    f0 = _feq(np.ones((L, 4, 4)), v, c, w)
    out = []
    for form in (0, 1):
        p = O.default_params(shp, lattice=q, lb_form=form, xi=0.0)
        s = O.State(shp, p)
        s.f, s.q, s.psi, s.u = f0.copy(), np.zeros((5, L, 4, 4)), np.zeros((L, 4, 4)), np.zeros((3, L, 4, 4))
        s.step(5)
        out.append(s.f.copy())
    ref = f0.copy()
    for _ in range(5):
        ref, _ = O.lb(ref, np.zeros((3, L, 4, 4)), O.default_params(shp, lattice=q))
    np.testing.assert_allclose(out[0], ref, atol=1e-16)
    np.testing.assert_allclose(out[1], ref, atol=1e-16)


# ---------------------------------------------------------------- integrator and coupling (Sec. 3)

def _uniform_H(q5, prm):
    """H of a uniform Q (no gradients) with psi = 1, from the sympy derivative of Eq. 5."""
    st_ = dict(q5=np.asarray(q5, float), dq5=np.zeros((5, 3)), hq5=np.zeros((5, 3, 3)), psi=np.array(1.0),
               dpsi=np.zeros(3), hpsi=np.zeros((3, 3)))
    H, _ = OH.analytic_H_mu(st_, prm)
    return np.array([H[0, 0], H[0, 1], H[0, 2], H[1, 1], H[1, 2]], float)


def _bulk_relaxation_state(prm, S, integrator, gammaQ):
    shp = (4, 4, 4)
    p = O.default_params(shp, integrator=integrator, gammaQ=gammaQ, zeta=0.0,
                         **{k: prm[k] for k in ("a", "b", "kphi", "A0", "chi0", "chis", "K", "q0", "W")})
    s = O.State(shp, p)
    _, w = O.lattice()
    s.f = np.ascontiguousarray(w.reshape(19, 1, 1, 1) * np.ones((19, 4, 4, 4)))
    s.q = np.ascontiguousarray(_uniform_uniaxial(S, shp))
    s.psi = np.ones((4, 4, 4))
    s.u = np.zeros((3, 4, 4, 4))
    return s


def test_heun_step_on_uniform_relaxation():
    """A uniform Q with psi = 1 and fluid at rest: sigma is uniform, F = 0, u stays 0 and
    Q follows dQ/dt = Gamma_Q H(Q).  One step of the oracle must equal the Euler map
    Q + Gamma H(Q) (integrator 0) and the Heun map Q + (Gamma H(Q) + Gamma H(Q*))/2 with
    Q* = Q + Gamma H(Q) (integrator 1), with H from the sympy derivative of Eq. 5."""
    prm = dict(BASE, q0=2 * np.pi / 16, W=0.02)
    S = 0.3  # away from S_eq = 0.5 at chi = 3: H != 0
    for gam in (0.3, 1.0):
        q = _uniform_uniaxial(S, (4, 4, 4))[:, 0, 0, 0]
        h1 = gam * _uniform_H(q, prm)
        euler = q + h1
        heun = q + 0.5 * (h1 + gam * _uniform_H(q + h1, prm))
        for integ, ref in ((0, euler), (1, heun)):
            s = _bulk_relaxation_state(prm, S, integ, gam).step(1)
            got = s.q[:, 0, 0, 0]
            assert np.abs(s.q - got.reshape(5, 1, 1, 1)).max() == 0.0  # stays uniform
            assert np.abs(got - ref).max() < 1e-15, (integ, got - ref)
            assert np.abs(s.u).max() < 1e-16
        assert np.abs(heun - euler).max() > 1e-5  # the two maps are distinguishable here


def test_heun_is_second_order_in_time():
    """Local error of one step against the exact flow of dQ/dt = Gamma H(Q) (scipy RK45 at
    1e-13 tolerance on the sympy H): third order in Gamma for Heun, second for Euler."""
    from scipy.integrate import solve_ivp
    prm = dict(BASE, q0=0.0, W=0.02)
    S = 0.3
    q = _uniform_uniaxial(S, (4, 4, 4))[:, 0, 0, 0]
    errs = {0: [], 1: []}
    gams = (0.4, 0.2, 0.1)
    for gam in gams:
        sol = solve_ivp(lambda t, y: gam * _uniform_H(y, prm), (0.0, 1.0), q, rtol=1e-13, atol=1e-15)
        exact = sol.y[:, -1]
        for integ in (0, 1):
            got = _bulk_relaxation_state(prm, S, integ, gam).step(1).q[:, 0, 0, 0]
            errs[integ].append(np.abs(got - exact).max())
    for integ, order in ((0, 2), (1, 3)):
        e = errs[integ]
        for k in range(len(gams) - 1):
            assert abs(np.log2(e[k] / e[k + 1]) - order) < 0.25, (integ, e)


def test_sync_coupling_advects_with_this_steps_velocity():
    """Ordered uniform Q (n = x, S = S_eq, q0 = 0 so H = 0), psi = 1, populations at
    equilibrium with the shear u_x = A sin(2 pi z / L), u_prev = 0.  sigma is uniform, F = 0
    and the LB velocity of the step is the shear itself.  Lagged coupling advects with
    u_prev = 0: Q is unchanged.  Sync coupling uses the shear: W_xz = A sin(2 pi/L)
    cos(2 pi z/L) (central difference of the sine) and the co-rotation of Eq. 2 for this
    Q and W reduces by hand to S_xz = S_zx = (W_xz/2)[S0 (xi - 1) + 2 xi (1 - S0)/3], the
    other components zero."""
    c, w = O.lattice()
    L, n = 16, 4
    shp = (n, n, L)
    xi, A = 0.7, 1e-3
    S0 = 0.5  # S_eq at chi = 3
    z = np.arange(L).reshape(L, 1, 1) * np.ones((L, n, n))
    v = np.zeros((3, L, n, n))
    v[0] = A * np.sin(2 * np.pi * z / L)
    Q = S0 * (np.diag([1.0, 0.0, 0.0]) - np.eye(3) / 3)
    q5 = np.array([Q[0, 0], Q[0, 1], Q[0, 2], Q[1, 1], Q[1, 2]]).reshape(5, 1, 1, 1) * np.ones((5, L, n, n))
    out = {}
    for coupling in (0, 1):
        p = O.default_params(shp, coupling=coupling, q0=0.0, xi=xi, zeta=0.003)
        s = O.State(shp, p)
        s.f = np.ascontiguousarray(_feq(np.ones((L, n, n)), v, c, w))
        s.q = q5.copy()
        s.psi = np.ones((L, n, n))
        s.u = np.zeros((3, L, n, n))
        s.step(1)
        np.testing.assert_allclose(s.u, v, atol=1e-17)
        out[coupling] = s.q - q5
    assert np.abs(out[0]).max() < 1e-16
    Wxz = A * np.sin(2 * np.pi / L) * np.cos(2 * np.pi * z / L)
    Sxz = 0.5 * Wxz * (S0 * (xi - 1) + 2 * xi * (1 - S0) / 3)
    exp = np.zeros_like(q5)
    exp[2] = Sxz
    assert np.abs(out[1] - exp).max() < 1e-17, np.abs(out[1] - exp).max()
    assert np.abs(Sxz).max() > 1e-6


def _random_state(n, seed):
    c, w = O.lattice()
    st_ = OH.smooth_state((n, n, n), seed=seed)
    rng = np.random.default_rng(seed)
    f = w.reshape(19, 1, 1, 1) * (1 + 0.01 * rng.standard_normal((19, n, n, n)))
    u = 1e-3 * rng.standard_normal((3, n, n, n))
    return f, np.ascontiguousarray(st_["q5"]), np.ascontiguousarray(np.clip(st_["psi"], -0.95, 0.95)), u


def _run(f, q, psi, u, p, nsteps):
    s = O.State.__new__(O.State)
    nz = psi.shape[0]
    s.shape, s.p, s.t = (nz, nz, nz), p, 0
    s.f, s.q, s.psi, s.u = f.copy(), q.copy(), psi.copy(), u.copy()
    s.step(nsteps)
    return s


@pytest.mark.parametrize("P,name", [
    (np.array([[0, 1, 0], [0, 0, 1], [1, 0, 0]]), "cyclic"),
    (np.array([[0, 1, 0], [1, 0, 0], [0, 0, 1]]), "swap-xy"),
    (np.diag([1, 1, -1]), "mirror-z"),
])
def test_cubic_symmetry_equivariance(P, name):
    """Rotations and reflections of the lattice commute with the step; improper ones flip
    the handedness q0 -> -q0 (the chiral term is a pseudo-scalar)."""
    c, w = O.lattice()
    n = 6
    f, q, psi, u = _random_state(n, seed=21)
    p = O.default_params((n, n, n), zeta=0.01, W=0.05)
    s1 = _run(f, q, psi, u, p, 3)
    a = OH.transform_state(s1.f, s1.q, s1.psi, s1.u, P, c)
    p2 = O.default_params((n, n, n), zeta=0.01, W=0.05)
    p2.q0 = p.q0 * round(np.linalg.det(P))
    t = OH.transform_state(f, q, psi, u, P, c)
    s2 = _run(*t, p2, 3)
    for x1, x2 in zip(a, (s2.f, s2.q, s2.psi, s2.u)):
        np.testing.assert_allclose(x2, x1, atol=2e-13)


@pytest.mark.parametrize("lat,form,stencil", [(19, 0, 0), (19, 1, 0), (15, 0, 0), (15, 1, 0), (19, 0, 1)])
def test_cholesteric_helix_is_stationary(lat, form, stencil):
    """A uniform helix (psi = 1, Q period pi/q0 commensurate with the box) drives no flow
    with or without activity: rotation by pi about z maps it to itself, so sigma_xz =
    sigma_yz = 0, and screw symmetry makes sigma_zz and sigma_xx + sigma_yy uniform.  Its
    phase does not drift.  This holds for both LB velocity sets and both LB forms."""
    nz = 16
    shp = (4, 4, nz)
    for zeta in (0.0, 0.005):
        p = O.default_params(shp, p0=16.0, zeta=zeta, R=1e9, lattice=lat, lb_form=form, stencil=stencil)
        s = O.State(shp, p)
        s.psi[:] = 1.0
        z = np.arange(nz).reshape(nz, 1, 1)
        th = p.q0 * (z - p.cz) * np.ones((nz, 4, 4))
        nn = np.array([np.cos(th), np.sin(th), 0 * th])
        Q = 0.5 * (np.einsum("a...,b...->ab...", nn, nn) - np.eye(3).reshape(3, 3, 1, 1, 1) / 3)
        s.q = np.ascontiguousarray(np.array([Q[0, 0], Q[0, 1], Q[0, 2], Q[1, 1], Q[1, 2]]))
        s.step(30)
        assert np.abs(s.u).max() < 1e-13
        assert np.abs(s.q[2]).max() < 1e-15 and np.abs(s.q[4]).max() < 1e-15
        # screw symmetry: Q(z+1) = R(q0) Q(z) R(q0)^T
        Qf = OH.full_from5(s.q)
        c, sn = np.cos(p.q0), np.sin(p.q0)
        Rm = np.array([[c, -sn, 0], [sn, c, 0], [0, 0, 1]])
        for k in range(nz - 1):
            np.testing.assert_allclose(Qf[:, :, k + 1, 0, 0], Rm @ Qf[:, :, k, 0, 0] @ Rm.T, atol=1e-13)
        # phase: at z = cz the director stays along x (Q_xy = 0)
        assert abs(s.q[1][int(p.cz), 0, 0]) < 1e-13
        np.testing.assert_allclose(s.psi, 1.0, atol=1e-14)


def test_flat_interface_is_equilibrium():
    """psi = tanh(x/2) with Q = 0 is the flat-interface equilibrium for k_phi = 2a: mu
    vanishes as the grid is refined (second order)."""
    Lp = 64.0
    errs = []
    for n in (64, 128, 256):
        h = Lp / n
        x = np.arange(n) * h
        psi1 = np.tanh((x - Lp / 4) / 2) - np.tanh((x - 3 * Lp / 4) / 2) - 1.0
        psi = np.ascontiguousarray(np.broadcast_to(psi1, (4, 4, n)))
        p = _scaled_params(BASE, h)
        out = O.fields(np.zeros((5, 4, 4, n)), psi, p)
        errs.append(np.abs(out["mu"]).max())
    assert errs[2] < 1e-3 and errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs


# ---------------------------------------------------------------- initial state

def test_noise_is_splitmix64():
    vals = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt")) if l.strip()
            and not l.startswith("#")]
    for k, r in enumerate(vals):
        # counter k+1 = 1 + 5*site + comp for instance 0
        site, comp = divmod(k, 5)
        expect = 2.0 * ((r >> 11) * 2.0 ** -53) - 1.0
        assert O.noise(1234567, 0, site, comp) == expect


def test_initial_droplet():
    n = 32
    p = O.default_params((n, n, n), R=8.0, p0=16.0)
    s = O.State((n, n, n), p, seed=3)
    assert np.all(np.abs(s.q) <= 0.5)
    assert abs(s.psi[16, 16, 16] - np.tanh(4.0)) < 1e-15
    inside = s.psi > np.tanh(0.0)
    Q = OH.full_from5(s.q)
    # away from the noise, the order inside is S0 = 0.5 along the helix
    lam = np.linalg.eigvalsh(np.moveaxis(Q[:, :, 16, 16, 16], (0, 1), (0, 1)))
    assert abs(1.5 * lam.max() - 0.5) < 5e-3
    assert np.all(s.q[:, ~inside] == 0.0)
    assert s.f.sum() == pytest.approx(n ** 3)


def test_forward_mode_tangent_matches_central_differences():
    """The oracle's dual-number tangent (used to pin the adjoint) against central
    differences of its own FP64 step, at a horizon where the step is smooth."""
    shape = (8, 8, 8)
    kw = dict(R=2.5, p0=6.0, zeta=0.02, W=0.0)

    def run(**over):
        s = O.State(shape, O.default_params(shape, **dict(kw, **over)), seed=3)
        s.step(2)
        return np.concatenate([s.f.ravel(), s.q.ravel(), s.psi.ravel(), s.u.ravel()])

    s = O.State(shape, O.default_params(shape, **kw), seed=3)
    t = s.step_tangent(2, {}, dzeta=1.0)
    tv = np.concatenate([t[k].ravel() for k in ("f", "q", "psi", "u")])
    h = 1e-6
    fd = (run(zeta=0.02 + h) - run(zeta=0.02 - h)) / (2 * h)
    assert np.abs(tv - fd).max() <= 1e-6 * np.abs(fd).max()
    # tangent of the values: unchanged arithmetic for the state itself
    s2 = O.State(shape, O.default_params(shape, **kw), seed=3).step(2)
    np.testing.assert_array_equal(s.psi, s2.psi)


# ---------------------------------------------------------------- a6: the conserved and centroid sums

@pytest.mark.parametrize("q", [19, 15])
def test_observables_closed_forms(q):
    """The oracle's a6 sums against closed forms.  Populations at equilibrium with uniform
    density rho and velocity v: mass N rho and momentum N rho v, from the lattice moments
    (sum w = 1, sum w c = 0, sum w c c = I/3, sum w c c c = 0), not from the sum itself.
    psi = A cos(2 pi (r_a - r0)/L_a) + B along one axis a at a time: sum psi = B N, sum phi_c =
    (1 + B) N / 2, the phi_c moments along a are (A/2)(L_a/2)(N/L_a) (cos, sin)(2 pi r0/L_a),
    and along the other two axes they vanish (a constant summed against a full period)."""
    c, w = O.lattice(q)
    shp = (8, 6, 5)
    nx, ny, nz = shp
    N = nx * ny * nz
    rho, v = 1.2, np.array([0.01, -0.02, 0.005])
    f = _feq(np.full((nz, ny, nx), rho), v.reshape(3, 1, 1, 1) * np.ones((3, nz, ny, nx)), c, w)
    A, B, r0 = 0.6, -0.3, 1.7
    for a, La in enumerate(shp):
        r = np.arange(La, dtype=float)
        prof = A * np.cos(2 * np.pi * (r - r0) / La) + B
        shape_a = [1, 1, 1]
        shape_a[2 - a] = La  # arrays are [z][y][x]
        psi = np.ascontiguousarray(np.broadcast_to(prof.reshape(shape_a), (nz, ny, nx)))
        o = O.observables(np.ascontiguousarray(f), psi)
        assert abs(o[0] - N * rho) <= 1e-12 * N
        np.testing.assert_allclose(o[2:5], N * rho * v, rtol=0, atol=1e-12 * N)
        assert abs(o[1] - B * N) <= 1e-12 * N
        assert abs(o[11] - 0.5 * (1 + B) * N) <= 1e-12 * N
        amp = 0.5 * A * 0.5 * La * (N / La)
        for b in range(3):
            want_c = amp * np.cos(2 * np.pi * r0 / La) if b == a else 0.0
            want_s = amp * np.sin(2 * np.pi * r0 / La) if b == a else 0.0
            assert abs(o[5 + b] - want_c) <= 1e-11 * N, (a, b)
            assert abs(o[8 + b] - want_s) <= 1e-11 * N, (a, b)


def test_openmp_build_is_bitwise_identical():
    """The all-cores build of the oracle (its per-stage parallel-for over z) computes every
    site's values in the same order as the single-thread build, so the states are identical."""
    shape = (12, 10, 14)
    p = O.default_params(shape, R=4.0, p0=8.0, zeta=0.01)
    a = O.State(shape, p, seed=2)
    b = O.State(shape, p, seed=2, omp=True)
    a.step(4)
    b.step(4)
    for k in ("f", "q", "psi", "u"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k
    assert O.num_threads(False) == 1 and O.num_threads(True) >= 1
