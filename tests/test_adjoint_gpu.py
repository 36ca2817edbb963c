"""Adjoint of the hybrid step: J = |centroid displacement|^2 / 2 over n steps.

References, both independent of the CUDA path:
- The oracle's forward-mode derivative. The FP64 CPU step runs on dual numbers of its own,
  seeded in zeta, in q0, along a direction of the initial Q, or along a direction of the
  whole initial state. This differentiates exactly the same arithmetic, so the GPU adjoint
  must agree to rounding (1e-5 relative).
- Central finite differences of the GPU FP64 forward (h = 1e-4 relative, 1e-4 relative
  agreement).

J is only piecewise smooth. The first-order upwind terms of the scheme (Sec. 3) put kinks
where a face velocity changes sign, and over tens of steps those kinks lie closer together
than any usable finite-difference step. So the finite-difference comparison runs at a short
horizon and first checks that J is smooth there: differences with h and 10 h must agree.
"""
import numpy as np
import pytest

import paper_2011_00287_gb300 as L
from paper_2011_00287_gb300 import observables as OB
from oracle import oracle as O

pytestmark = pytest.mark.gpu

SHAPE = (16, 16, 16)
KW = dict(R=5.0, p0=8.0, zeta=0.02, W=0.05)
NSTEPS = 24
CKPT = 7  # several segments and a partial one
SEED = 3


def _perm():
    cl, _ = L.lattice()
    co, _ = O.lattice()
    return np.array([int(np.where((co == v).all(1))[0][0]) for v in cl])


def _dX(x0, x1):
    d = x1 - x0
    return d - np.array(SHAPE) * np.round(d / np.array(SHAPE))


def _centroid_tangent(psi, dpsi):
    """Tangent of the periodic centroid for a tangent dpsi of psi."""
    nz, ny, nx = psi.shape
    out = np.zeros(3)
    for a, n, axis in ((0, nx, 2), (1, ny, 1), (2, nz, 0)):
        th = 2 * np.pi * np.arange(n) / n
        shp = [1, 1, 1]
        shp[axis] = n
        sn, cs = np.sin(th).reshape(shp), np.cos(th).reshape(shp)
        pc = 0.5 * (1 + psi)
        S, C = np.sum(pc * sn), np.sum(pc * cs)
        dS, dC = np.sum(0.5 * dpsi * sn), np.sum(0.5 * dpsi * cs)
        out[a] = n / (2 * np.pi) * (C * dS - S * dC) / (C * C + S * S)
    return out


def _oracle_dJ(nsteps=NSTEPS, kw=KW, dzeta=0.0, dq0=0.0, tangent=None, state=None):
    """(J, dJ) from the oracle's forward-mode tangent."""
    s = O.State(SHAPE, O.default_params(SHAPE, **kw), seed=SEED)
    if state is not None:
        s.f, s.q, s.psi, s.u = (np.ascontiguousarray(state[k]).copy() for k in ("f", "q", "psi", "u"))
    x0 = OB.centroid(s.observables(), SHAPE)
    t = s.step_tangent(nsteps, tangent or {}, dzeta=dzeta, dq0=dq0)
    x1 = OB.centroid(s.observables(), SHAPE)
    d = _dX(x0, x1)
    return 0.5 * float(d @ d), float(d @ _centroid_tangent(s.psi, t["psi"]))


def _J_gpu(nsteps=NSTEPS, prec=L.FP64, q5=None, **over):
    kw = dict(KW, **over)
    sim = L.Simulation([SHAPE], [L.default_params(SHAPE, precision=prec, **kw)], seed=SEED)
    if q5 is not None:
        sim.set_fields(0, {"q": q5})
    x0 = OB.centroid(sim.observables(0), SHAPE)
    sim.step(nsteps)
    d = _dX(x0, OB.centroid(sim.observables(0), SHAPE))
    sim.close()
    return 0.5 * float(d @ d)


def _adjoint(prec=L.FP64, nsteps=NSTEPS, ckpt=CKPT, kw=KW):
    sim = L.Simulation([SHAPE], [L.default_params(SHAPE, precision=prec, **kw)], seed=SEED)
    q0 = sim.get_fields(0, L.FIELD_Q)["q"].copy()
    J, dz, dq, dQ0 = sim.adjoint(nsteps, ckpt)
    assert sim.step_count == nsteps
    sim.close()
    return J, dz, dq, dQ0, q0


@pytest.fixture(scope="module")
def adj64():
    return _adjoint(L.FP64)


def test_objective_matches_forward_and_oracle(adj64):
    J = adj64[0]
    assert J > 0 and abs(J - _J_gpu()) <= 1e-12 * J
    Jo, _ = _oracle_dJ()
    assert abs(J - Jo) <= 1e-9 * J


def test_dJ_dzeta_matches_oracle_forward_mode(adj64):
    _, dz, _, _, _ = adj64
    _, ref = _oracle_dJ(dzeta=1.0)
    assert abs(dz - ref) <= 1e-5 * abs(ref), (dz, ref)


def test_dJ_dq0_matches_oracle_forward_mode(adj64):
    """q0 enters through H and sigma; the initial helix is held fixed."""
    _, _, dq, _, _ = adj64
    _, ref = _oracle_dJ(dq0=1.0)
    assert abs(dq - ref) <= 1e-5 * abs(ref), (dq, ref)


def test_dJ_dQ0_matches_oracle_forward_mode(adj64):
    _, _, _, dQ0, q0 = adj64
    rng = np.random.default_rng(11)
    for _ in range(3):
        v = rng.standard_normal(q0.shape)
        _, ref = _oracle_dJ(tangent={"q": v})
        ad = float(np.sum(dQ0 * v))
        assert abs(ad - ref) <= 1e-5 * abs(ref), (ad, ref)


def test_gradient_of_the_whole_initial_state_matches_oracle():
    """lbcad_adjoint_fields from a developed state: dJ/d(f, u, Q, psi) along random
    directions against the oracle's tangent (the reference centroid X(t0) held fixed)."""
    sim = L.Simulation([SHAPE], [L.default_params(SHAPE, precision=L.FP64, **KW)], seed=SEED)
    sim.step(3)
    st = sim.get_fields(0)
    sim.adjoint(NSTEPS, CKPT)
    lam = sim.adjoint_fields()
    sim.close()
    perm = _perm()
    inv = np.argsort(perm)
    ostate = dict(f=st["g"][inv], q=st["q"], psi=st["psi"], u=st["u"])
    rng = np.random.default_rng(5)
    for name, okey in (("g", "f"), ("u", "u"), ("q", "q"), ("psi", "psi")):
        v = rng.standard_normal(st[name].shape)
        tv = v[inv] if name == "g" else v
        s = O.State(SHAPE, O.default_params(SHAPE, **KW), seed=SEED)
        s.f, s.q, s.psi, s.u = (np.ascontiguousarray(ostate[k]).copy() for k in ("f", "q", "psi", "u"))
        x0 = OB.centroid(s.observables(), SHAPE)
        t = s.step_tangent(NSTEPS, {okey: tv})
        d = _dX(x0, OB.centroid(s.observables(), SHAPE))
        ref = float(d @ _centroid_tangent(s.psi, t["psi"]))
        ad = float(np.sum(lam[name] * v))
        assert abs(ad - ref) <= 1e-5 * abs(ref), (name, ad, ref)


def _fd_smooth(fun, x, rel=1e-4):
    """Central difference at h; asserts the one at 10 h agrees (J smooth here)."""
    def fd(r):
        h = r * abs(x)
        return (fun(x + h) - fun(x - h)) / (2 * h)
    a, b = fd(rel), fd(10 * rel)
    assert abs(a - b) <= 1e-4 * abs(a), ("J is not smooth at this point", a, b)
    return a


def test_short_horizon_finite_differences():
    """At two steps J is smooth in zeta and along a direction of the initial Q: central
    differences of the GPU forward agree with the adjoint within 1e-4."""
    n = 2
    _, dz, _, dQ0, q5 = _adjoint(L.FP64, nsteps=n, ckpt=1)
    fd = _fd_smooth(lambda v: _J_gpu(nsteps=n, zeta=v), KW["zeta"])
    assert abs(dz - fd) <= 1e-4 * abs(fd), (dz, fd)
    v = np.random.default_rng(2).standard_normal(q5.shape) * (np.abs(q5).sum(0) > 0)
    v *= 1e-2 / np.abs(v).max()  # small direction: curvature of J stays below the check
    fdv = _fd_smooth(lambda e: _J_gpu(nsteps=n, q5=q5 + (e - 1.0) * v), 1.0, rel=1e-4)
    ad = float(np.sum(dQ0 * v))
    assert abs(ad - fdv) <= 1e-4 * abs(fdv), (ad, fdv)


def test_repeated_adjoint_calls_reuse_buffers_exactly():
    """lbcad_adjoint keeps its buffers for later calls: a call after calls of other sizes
    (fewer and more checkpoints, a longer segment) gives the result of a fresh context at the
    same state, and the context's device memory stops growing.  (FP64, 1e-10 relative: the
    two contexts take the starting centroid from different passes of the a6 sums, the fused
    one and the separate one, which add in different orders.)"""
    import torch
    prm = [L.default_params(SHAPE, precision=L.FP64, **KW)]
    a = L.Simulation([SHAPE], prm, seed=SEED)
    a.adjoint(9, 3)
    a.adjoint(5, 5)
    free0, _ = torch.cuda.mem_get_info()
    ra = a.adjoint(8, 3)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    fa = a.adjoint_fields(L.FIELD_Q | L.FIELD_PSI)
    b = L.Simulation([SHAPE], prm, seed=SEED)
    b.step(14)
    rb = b.adjoint(8, 3)
    fb = b.adjoint_fields(L.FIELD_Q | L.FIELD_PSI)
    assert a.step_count == b.step_count == 22
    for x, y in zip(ra[:3], rb[:3]):
        assert abs(x - y) <= 1e-10 * abs(y), (x, y)
    assert np.abs(ra[3] - rb[3]).max() <= 1e-10 * np.abs(rb[3]).max()
    for k in fa:
        assert np.abs(fa[k] - fb[k]).max() <= 1e-10 * np.abs(fb[k]).max(), k
    assert free1 == free0, (free0, free1)
    a.close()
    b.close()


def test_fp32_adjoint_close_to_fp64(adj64):
    _, dz64, dq64, dQ64, _ = adj64
    _, dz32, dq32, dQ32, _ = _adjoint(L.FP32)
    assert abs(dz32 - dz64) <= 2e-2 * abs(dz64)
    assert abs(dq32 - dq64) <= 2e-2 * abs(dq64)
    assert np.linalg.norm(dQ32 - dQ64) <= 5e-2 * np.linalg.norm(dQ64)


def test_torch_autograd_function(adj64):
    import torch
    from paper_2011_00287_gb300.autograd import centroid_drift
    J0, dz, dq, dQ0, q0 = adj64
    zeta = torch.tensor(KW["zeta"], dtype=torch.float64, requires_grad=True)
    q0v = torch.tensor(2 * np.pi / KW["p0"], dtype=torch.float64, requires_grad=True)
    Q0 = torch.tensor(q0, dtype=torch.float64, requires_grad=True)
    prm = L.default_params(SHAPE, precision=L.FP64, **KW)
    J = centroid_drift(zeta, q0v, Q0, SHAPE, prm, NSTEPS, CKPT, seed=SEED)
    (2.0 * J).backward()
    assert abs(J.item() - J0) <= 1e-12 * J0
    assert abs(zeta.grad.item() - 2 * dz) <= 1e-12 * abs(dz)
    assert abs(q0v.grad.item() - 2 * dq) <= 1e-12 * abs(dq)
    assert np.allclose(Q0.grad.numpy(), 2 * dQ0, rtol=1e-12, atol=0)


# ---------------------------------------------------------------- the differentiation workload (500 steps)
# The workload asks for the adjoint over 500 steps with checkpoints every 50, checked against
# the FP64 reference gradient on a 16^3 copy.  Two copies: the workload's own parameters
# scaled to 16^3 (R = 16/4, pitch 16/4, zeta = 0.005) and the resolved droplet used above
# (R = 5, pitch 8).  Over 500 steps the forward-mode tangent of the oracle and the GPU adjoint
# still differentiate the same arithmetic, but each follows its own trajectory's upwind
# branches (Sec. 3's first-order upwind terms switch where a face velocity changes sign), and
# FP64 rounding can put a velocity near zero on different sides in the two programs.  Such a
# site changes the derivative by the jump of the upwind term (Q(+a) - 2 Q + Q(-a)) times the
# velocity's derivative.  On the resolved copy every derivative agrees within 1e-5 (measured
# at most 1.3e-6); on the scaled copy, whose pitch of 4 sites makes Q vary by 90 degrees per
# site, one direction of Q0 differs by 3.8e-5, so the Q0 directions there are held to 1e-4.
CFG4_CASES = [("scaled-config", dict(R=4.0, p0=4.0, zeta=0.005), 1e-4), ("resolved", dict(R=5.0, p0=8.0, zeta=0.02), 1e-5)]
CFG4_STEPS, CFG4_CKPT = 500, 50


def _oracle_dJ_kw(kw, nsteps, dzeta=0.0, dq0=0.0, tangent=None):
    s = O.State(SHAPE, O.default_params(SHAPE, **kw), seed=SEED, omp=True)
    x0 = OB.centroid(s.observables(), SHAPE)
    t = s.step_tangent(nsteps, tangent or {}, dzeta=dzeta, dq0=dq0)
    x1 = OB.centroid(s.observables(), SHAPE)
    d = _dX(x0, x1)
    return 0.5 * float(d @ d), float(d @ _centroid_tangent(s.psi, t["psi"]))


@pytest.mark.parametrize("name,kw,tol_dir", CFG4_CASES, ids=[c[0] for c in CFG4_CASES])
def test_500_step_adjoint_on_16cube_matches_oracle(name, kw, tol_dir):
    """FP64 GPU adjoint (500 steps, checkpoints every 50) against the oracle's forward-mode
    derivative: dJ/dzeta and dJ/dq0 within 1e-5, three seeded directions of Q0 within the
    case's tolerance.  The FP32 adjoint against the same references within 1e-1: its forward
    trajectory is the FP32 one, whose J differs from FP64 by about 1% here (the displacement is
    about 1e-5 lattice units), and over 500 steps the gradient follows the FP32 rounding
    pattern: two FP32 variants of the step that differ only in how the collision and the
    co-rotation term group their operations measured 0.5-2.1% and up to 5.5%."""
    J64, dz64, dq64, dQ64, _ = _adjoint(L.FP64, nsteps=CFG4_STEPS, ckpt=CFG4_CKPT, kw=kw)
    J32, dz32, dq32, dQ32, _ = _adjoint(L.FP32, nsteps=CFG4_STEPS, ckpt=CFG4_CKPT, kw=kw)
    Jo, rz = _oracle_dJ_kw(kw, CFG4_STEPS, dzeta=1.0)
    _, rq = _oracle_dJ_kw(kw, CFG4_STEPS, dq0=1.0)
    assert abs(J64 - Jo) <= 1e-8 * Jo, (J64, Jo)
    assert abs(dz64 - rz) <= 1e-5 * abs(rz), (dz64, rz)
    assert abs(dq64 - rq) <= 1e-5 * abs(rq), (dq64, rq)
    assert abs(dz32 - rz) <= 1e-1 * abs(rz), (dz32, rz)
    assert abs(dq32 - rq) <= 1e-1 * abs(rq), (dq32, rq)
    rng = np.random.default_rng(11)
    for _ in range(3):
        v = rng.standard_normal(dQ64.shape)
        _, ref = _oracle_dJ_kw(kw, CFG4_STEPS, tangent={"q": v})
        a64, a32 = float(np.sum(dQ64 * v)), float(np.sum(dQ32 * v))
        assert abs(a64 - ref) <= tol_dir * abs(ref), (a64, ref)
        assert abs(a32 - ref) <= 1e-1 * abs(ref), (a32, ref)


def test_500_step_adjoint_on_64cube_fp32_against_fp64():
    """The differentiation workload itself: 64^3, R = 16, pitch 16, zeta = 0.005, 500 steps,
    checkpoints every 50.  FP32 against FP64 on the GPU, each within 1e-1 (measured: dJ/dzeta 3.0%,
    dJ/dq0 4.4%, dJ/dQ0 0.9% in norm with cosine 0.99996; before the order-parameter update added
    its increments in one rounding, dJ/dq0 differed by 27%: q0 enters only through H and sigma with
    the initial helix fixed, and its dimensionless size q0 dJ/dq0 is a third of zeta dJ/dzeta, so
    the FP32 trajectory's difference weighs most in it).  (Finite differences are no reference at this horizon:
    central differences of the FP64 forward in zeta give 9.8e-8, 1.5e-8 and -4.6e-10 for steps
    of 1e-4, 1e-3 and 1e-2 relative, against an adjoint of 1.09e-8, because J has upwind kinks
    closer together than any of these steps.)"""
    shape = (64, 64, 64)
    kw = dict(R=16.0, p0=16.0, zeta=0.005)
    out = {}
    for prec in (L.FP64, L.FP32):
        sim = L.Simulation([shape], [L.default_params(shape, precision=prec, **kw)], seed=1)
        out[prec] = sim.adjoint(CFG4_STEPS, CFG4_CKPT)
        sim.close()
    (J64, dz64, dq64, dQ64), (J32, dz32, dq32, dQ32) = out[L.FP64], out[L.FP32]
    assert np.isfinite([J32, dz32, dq32]).all() and np.isfinite(dQ32).all()
    assert abs(dz32 - dz64) <= 1e-1 * abs(dz64), (dz32, dz64)
    assert np.linalg.norm(dQ32 - dQ64) <= 1e-1 * np.linalg.norm(dQ64)
    assert abs(dq32 - dq64) <= 1e-1 * abs(dq64), (dq32, dq64)
