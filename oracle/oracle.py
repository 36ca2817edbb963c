"""Python access to the plain FP64 CPU oracle (``lbcad_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The product path never
imports it.  It shares no code with the CUDA library.

Fields are numpy float64 arrays in ``[component][z][y][x]`` order (x fastest).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbcad_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblbcad_oracle.so")
# the same source with its per-stage OpenMP parallel-for over z switched on (all host cores)
_LIB_OMP = os.path.join(_BUILD, "liblbcad_oracle_omp.so")
_lock = threading.Lock()
_libs = {}


class orc_params(ctypes.Structure):
    """Parameters of Eqs. 1-11; field order mirrors the C struct."""

    _fields_ = [(n, ctypes.c_double) for n in (
        "tau", "rho0", "A0", "chi0", "chis", "K", "q0", "gammaQ", "xi",
        "a", "b", "kphi", "M", "W", "zeta", "R", "cx", "cy", "cz", "S0", "noise")] + [
        ("integrator", ctypes.c_int), ("coupling", ctypes.c_int), ("lattice", ctypes.c_int),
        ("lb_form", ctypes.c_int), ("stencil", ctypes.c_int)]


def default_params(n=(32, 32, 32), R=8.0, p0=16.0, **kw) -> orc_params:
    """Droplet workload parameters (A0=1, chi_in=3, K=0.04, Gamma_Q=0.3, xi=0.7,
    a=b=0.07, M=0.1, zeta=0.005, tau=1) with the readings chi0=2.5, chis=0.25,
    W=0.02, kphi=2a; centre at the box centre, S0=0.5, noise 1e-3; D3Q19 LB with the
    whole stress as a body force (lattice=15 selects D3Q15, lb_form=1 the form of Eqs. 9-11);
    isotropic radius-1 stencils (stencil=1 selects the fourth-order radius-2 set)."""
    nx, ny, nz = n
    d = dict(tau=1.0, rho0=1.0, A0=1.0, chi0=2.5, chis=0.25, K=0.04,
             q0=2.0 * np.pi / p0, gammaQ=0.3, xi=0.7, a=0.07, b=0.07, kphi=0.14,
             M=0.1, W=0.02, zeta=0.005, R=R, cx=nx / 2.0, cy=ny / 2.0, cz=nz / 2.0,
             S0=0.5, noise=1e-3, integrator=0, coupling=0, lattice=19, lb_form=0, stencil=0)
    d.update(kw)
    p = orc_params()
    for k, v in d.items():
        setattr(p, k, v)
    return p


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle with g++ (no fast-math, no FP contraction); omp=True builds the
    variant whose stage loops run on all host cores (same arithmetic per site)."""
    out = _LIB_OMP if omp else _LIB
    with _lock:
        if (not force and os.path.exists(out)
                and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
            return out
        os.makedirs(_BUILD, exist_ok=True)
        tmp = out + ".%d.tmp" % os.getpid()
        extra = ["-fopenmp"] if omp else []
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", *extra,
                               "-shared", _SRC, "-o", tmp])
        os.replace(tmp, out)
        return out


def lib(omp: bool = False):
    if omp not in _libs:
        L = ctypes.CDLL(build(omp=omp))
        dp = ctypes.POINTER(ctypes.c_double)
        P = ctypes.POINTER(orc_params)
        i = ctypes.c_int
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_lattice.argtypes = [ctypes.POINTER(ctypes.c_int), dp]
        L.orc_lattice_q.argtypes = [i, ctypes.POINTER(ctypes.c_int), dp]
        L.orc_lb_stress.argtypes = [i, i, i, P, dp, dp, dp, dp, dp]
        L.orc_observables_q.argtypes = [i, i, i, i, dp, dp, dp]
        L.orc_noise.argtypes = [ctypes.c_uint64, i, ctypes.c_long, i]
        L.orc_noise.restype = ctypes.c_double
        L.orc_init.argtypes = [i, i, i, P, ctypes.c_uint64, i, dp, dp, dp, dp]
        L.orc_fields.argtypes = [i, i, i, P, dp, dp] + [dp] * 7
        L.orc_force.argtypes = [i, i, i, dp, dp]
        L.orc_force_st.argtypes = [i, i, i, i, dp, dp]
        L.orc_stencils_st.argtypes = [i, i, i, i, dp, dp, dp, dp]
        L.orc_stencils.argtypes = [i, i, i, dp, dp, dp, dp]
        L.orc_corotation.argtypes = [dp, dp, ctypes.c_double, dp]
        L.orc_op_rhs.argtypes = [i, i, i, P, dp, dp, dp, dp, dp, dp, dp, dp]
        L.orc_step.argtypes = [i, i, i, P, dp, dp, dp, dp, ctypes.c_long]
        L.orc_lb.argtypes = [i, i, i, P, dp, dp, dp, dp]
        L.orc_observables.argtypes = [i, i, i, dp, dp, dp]
        L.orc_step_tangent.argtypes = [i, i, i, P, ctypes.c_double, ctypes.c_double] + [dp] * 8 + [ctypes.c_long]
        _libs[omp] = L
    return _libs[omp]


def num_threads(omp: bool = False) -> int:
    """Threads the oracle's stage loops run on (1 for the single-thread build)."""
    return int(lib(omp).orc_num_threads())


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def lattice(q=19):
    """LB velocities (q, 3) and weights (q,) of D3Q19 (q = 19) or D3Q15 (q = 15)."""
    c = np.zeros(3 * q, dtype=np.int32)
    w = np.zeros(q)
    lib().orc_lattice_q(q, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(w))
    return c.reshape(q, 3), w


class State:
    """Oracle state: f (q, nz, ny, nx) pre-collision populations (q = params.lattice),
    q (5, ...), psi (nz, ny, nx), u (3, ...) = velocity of the previous step.  omp=True
    steps it with the all-cores build (same arithmetic per site)."""

    omp = False

    def __init__(self, shape, params: orc_params, seed: int = 1, inst: int = 0, omp: bool = False):
        nx, ny, nz = shape
        self.omp = omp
        self.shape = (nx, ny, nz)
        self.p = params
        g = (nz, ny, nx)
        self.f = np.zeros((params.lattice,) + g)
        self.q = np.zeros((5,) + g)
        self.psi = np.zeros(g)
        self.u = np.zeros((3,) + g)
        lib().orc_init(nx, ny, nz, ctypes.byref(params), seed, inst,
                       _p(self.f), _p(self.q), _p(self.psi), _p(self.u))
        self.t = 0

    def step(self, n: int = 1):
        nx, ny, nz = self.shape
        lib(self.omp).orc_step(nx, ny, nz, ctypes.byref(self.p), _p(self.f), _p(self.q),
                       _p(self.psi), _p(self.u), n)
        self.t += n
        return self

    def observables(self):
        return observables(self.f, self.psi)

    def step_tangent(self, n, tangent, dzeta=0.0, dq0=0.0):
        """Advance n steps carrying the forward-mode tangent `tangent` = dict(f, q, psi, u)
        (arrays like the state; missing entries are zero) and parameter tangents; returns
        the tangent of the final state."""
        nx, ny, nz = self.shape
        t = {k: np.ascontiguousarray(tangent.get(k, np.zeros_like(getattr(self, k))), dtype=np.float64).copy()
             for k in ("f", "q", "psi", "u")}
        lib(self.omp).orc_step_tangent(nx, ny, nz, ctypes.byref(self.p), float(dzeta), float(dq0), _p(self.f), _p(t["f"]),
                               _p(self.q), _p(t["q"]), _p(self.psi), _p(t["psi"]), _p(self.u), _p(t["u"]), n)
        self.t += n
        return t

    def copy(self):
        s = State.__new__(State)
        s.shape, s.p, s.t, s.omp = self.shape, self.p, self.t, self.omp
        s.f, s.q, s.psi, s.u = self.f.copy(), self.q.copy(), self.psi.copy(), self.u.copy()
        return s


def fields(q, psi, params: orc_params):
    """Stages 1-4: dict with H (5), mu, sigma (9 = 3a+b), sE, sR, sA, fden."""
    nz, ny, nx = psi.shape
    g = psi.shape
    out = dict(H=np.zeros((5,) + g), mu=np.zeros(g), sigma=np.zeros((9,) + g),
               sE=np.zeros((9,) + g), sR=np.zeros((9,) + g), sA=np.zeros((9,) + g),
               fden=np.zeros(g))
    lib().orc_fields(nx, ny, nz, ctypes.byref(params), _p(np.ascontiguousarray(q)),
                     _p(np.ascontiguousarray(psi)), _p(out["H"]), _p(out["mu"]),
                     _p(out["sigma"]), _p(out["sE"]), _p(out["sR"]), _p(out["sA"]),
                     _p(out["fden"]))
    return out


def force(sigma9, stencil=0):
    nz, ny, nx = sigma9.shape[1:]
    F = np.zeros((3, nz, ny, nx))
    lib().orc_force_st(stencil, nx, ny, nz, _p(np.ascontiguousarray(sigma9)), _p(F))
    return F


def stencils(s, stencil=0):
    """Gradient (3), Laplacian, Hessian (9 = 3a+b) of a scalar field with the isotropic
    radius-1 set (stencil 0) or the fourth-order radius-2 set (stencil 1)."""
    nz, ny, nx = s.shape
    g = np.zeros((3,) + s.shape)
    lap = np.zeros(s.shape)
    h = np.zeros((9,) + s.shape)
    lib().orc_stencils_st(stencil, nx, ny, nz, _p(np.ascontiguousarray(s, dtype=np.float64)), _p(g), _p(lap),
                          _p(h))
    return g, lap, h


def corotation(W, Q, xi):
    S = np.zeros(9)
    lib().orc_corotation(_p(np.ascontiguousarray(W, dtype=np.float64).reshape(9)),
                         _p(np.ascontiguousarray(Q, dtype=np.float64).reshape(9)), xi, _p(S))
    return S.reshape(3, 3)


def op_rhs(q, psi, uadv, H, mu, params: orc_params):
    nz, ny, nx = psi.shape
    rq = np.zeros((5,) + psi.shape)
    rp = np.zeros(psi.shape)
    W = np.zeros((9,) + psi.shape)
    c = np.ascontiguousarray
    lib().orc_op_rhs(nx, ny, nz, ctypes.byref(params), _p(c(q)), _p(c(psi)), _p(c(uadv)),
                     _p(c(H)), _p(c(mu)), _p(rq), _p(rp), _p(W))
    return rq, rp, W


def lb(f, F, params: orc_params):
    nz, ny, nx = f.shape[1:]
    fn = np.zeros_like(f)
    un = np.zeros((3, nz, ny, nx))
    lib().orc_lb(nx, ny, nz, ctypes.byref(params), _p(np.ascontiguousarray(f)),
                 _p(np.ascontiguousarray(F)), _p(fn), _p(un))
    return fn, un


def observables(f, psi):
    nz, ny, nx = psi.shape
    out = np.zeros(12)
    lib().orc_observables_q(f.shape[0], nx, ny, nz, _p(np.ascontiguousarray(f)), _p(np.ascontiguousarray(psi)),
                            _p(out))
    return out


def lb_stress(f, FA, sig9, params: orc_params):
    """Collision and streaming in the form of Eqs. 9-11 with the force FA of the
    antisymmetric stress and the stress sig9 whose symmetric part enters the equilibrium."""
    nz, ny, nx = f.shape[1:]
    fn = np.zeros_like(f)
    un = np.zeros((3, nz, ny, nx))
    c = np.ascontiguousarray
    lib().orc_lb_stress(nx, ny, nz, ctypes.byref(params), _p(c(f)), _p(c(FA)), _p(c(sig9)), _p(fn), _p(un))
    return fn, un


def noise(seed, inst, site, comp):
    return lib().orc_noise(seed, inst, site, comp)


def q_full(q5):
    """(5, ...) stored components -> (3, 3, ...) full tensor."""
    xx, xy, xz, yy, yz = q5
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, -xx - yy]])
