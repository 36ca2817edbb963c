"""The D3Q15 velocity set and the stress-in-equilibrium LB form (Eqs. 9-11) on the GPU
fused path (their default) and the staged path against the FP64 oracle, through the C ABI.

Tolerances: FP64 within 1e-12 max abs per field after 10 steps; FP32 within 1e-5 relative L2
per field after 100 steps for D3Q15 with the body force, 1e-4 for the stress-in-equilibrium form
(FP32_TOL and FP32_STEPS below give the reasons).
"""
import numpy as np
import pytest

import paper_2011_00287_gb300 as L
from oracle import oracle as O
from tests.test_parity_gpu import KW0, _lib_params, _oracle, _rel_l2

pytestmark = pytest.mark.gpu

VARIANTS = {
    "d3q15": dict(lattice=15, lb_form=0),
    "stress-eq": dict(lattice=19, lb_form=1),
    "d3q15-stress-eq": dict(lattice=15, lb_form=1),
}
# The stress-in-equilibrium form is unstable on the droplet at tau <= 1 (D3Q19) and tau <= 1.5
# (D3Q15): over 100 steps the FP64 trajectory amplifies any perturbation, so FP32 parity runs
# where each variant is stable.
TAU_STABLE = {"d3q15": 1.0, "stress-eq": 1.5, "d3q15-stress-eq": 2.5}
# FP32 tolerance (relative L2 after 100 steps).  In the stress-in-equilibrium form the stored
# populations carry the stress, (9/2) w_i (c c - I/3) : sigma^S, a part about ten times larger
# than their velocity part; FP32 rounding of that part enters the momentum sum each step, so the
# bound is ten times the body-force one.
FP32_TOL = {"d3q15": 1e-5, "stress-eq": 1e-4, "d3q15-stress-eq": 1e-4}
# D3Q15 with the stress in the equilibrium is only marginally stable even at tau = 2.5 (max |u|
# starts to grow after about 100 steps), so its FP32 check stops at 50 steps.
FP32_STEPS = {"d3q15": 100, "stress-eq": 100, "d3q15-stress-eq": 50}


def _lib_kw(var):
    return dict(lattice=L.D3Q15 if var["lattice"] == 15 else L.D3Q19,
                lb_form=L.LB_STRESS_EQ if var["lb_form"] else L.LB_BODY_FORCE)


def _perm(q):
    cl, _ = L.lattice(L.D3Q15 if q == 15 else L.D3Q19)
    co, _ = O.lattice(q)
    return np.array([int(np.where((co == v).all(1))[0][0]) for v in cl])


def _compare(got, ref, q, fp64, tol):
    perm = _perm(q)
    _, w = O.lattice(q)
    wq = w.reshape(q, 1, 1, 1)
    if fp64:
        errs = {"g": np.abs(got["g"] - ref.f[perm]).max(), "q": np.abs(got["q"] - ref.q).max(),
                "psi": np.abs(got["psi"] - ref.psi).max(), "u": np.abs(got["u"] - ref.u).max()}
    else:
        errs = {"g": _rel_l2(got["g"] - wq[perm], (ref.f - wq)[perm]), "q": _rel_l2(got["q"], ref.q),
                "psi": _rel_l2(got["psi"], ref.psi), "u": _rel_l2(got["u"], ref.u)}
    for k, e in errs.items():
        assert e <= tol, errs
    return errs


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2011_00287_gb300 import build as B
    B.build()
    O.build()


def test_velocity_set_tables_match_the_oracle():
    for q, code in ((15, L.D3Q15), (19, L.D3Q19)):
        cl, wl = L.lattice(code)
        co, wo = O.lattice(q)
        assert cl.shape == (q, 3)
        perm = _perm(q)
        assert np.array_equal(cl, co[perm]) and np.array_equal(wl, wo[perm])


@pytest.mark.parametrize("path", ["fused", "staged"])
@pytest.mark.parametrize("name", list(VARIANTS))
@pytest.mark.parametrize("shape,kw", [
    ((32, 32, 32), KW0),
    ((21, 13, 10), dict(R=4.0, p0=8.0, zeta=0.01, W=0.05)),
    ((4, 5, 6), dict(R=2.0, p0=6.0)),
])
def test_fp64_parity_10_steps(shape, kw, name, path):
    var = VARIANTS[name]
    sim = L.Simulation([shape], [_lib_params(shape, L.FP64, **kw, **_lib_kw(var))], seed=2)
    if path == "staged":
        sim.set_path(L.lbcad.PATH_STAGED)
    got0 = sim.get_fields(0)
    ref = _oracle(shape, seed=2, **kw, **var)
    assert np.array_equal(got0["g"], ref.f[_perm(var["lattice"])])
    sim.step(10)
    ref.step(10)
    _compare(sim.get_fields(0), ref, var["lattice"], True, 1e-12)


@pytest.mark.parametrize("name", list(VARIANTS))
def test_fp32_parity_100_steps(name):
    var = VARIANTS[name]
    shape = (32, 32, 32)
    tau = TAU_STABLE[name]
    sim = L.Simulation([shape], [_lib_params(shape, L.FP32, **KW0, tau=tau, **_lib_kw(var))], seed=1)
    n = FP32_STEPS[name]
    sim.step(n)
    ref = _oracle(shape, seed=1, **KW0, tau=tau, **var).step(n)
    print(name, "fp32 rel L2 after %d steps:" % n, _compare(sim.get_fields(0), ref, var["lattice"], False,
                                                           FP32_TOL[name]))


@pytest.mark.parametrize("name", list(VARIANTS))
@pytest.mark.parametrize("prec", [L.FP32, L.FP64])
def test_fused_shapes_and_staged_path_agree(name, prec):
    """Both fused tile shapes of a variant give identical results (the per-site arithmetic
    does not depend on the shape), and the staged path, a different kernel split of the same
    per-site functions, agrees to rounding (after 20 steps, within a tenth of the variant's
    100-step FP32 parity bound)."""
    var = VARIANTS[name]
    shape = (40, 18, 12)
    kw = dict(R=5.0, p0=8.0, zeta=0.01, tau=TAU_STABLE[name])
    sims = [L.Simulation([shape], [_lib_params(shape, prec, **kw, **_lib_kw(var))], seed=3) for _ in range(3)]
    if prec == L.FP32:
        sims[1].set_tiles(3)
    sims[2].set_path(L.lbcad.PATH_STAGED)
    for s_ in sims:
        s_.step(20)
    f = [s_.get_fields(0) for s_ in sims]
    _, w = O.lattice(var["lattice"])
    wq = w[_perm(var["lattice"])].reshape(-1, 1, 1, 1)
    for k in f[0]:
        assert np.array_equal(f[0][k], f[1][k]), k
        if prec == L.FP64:
            assert np.abs(f[0][k] - f[2][k]).max() <= 1e-13, k
        else:
            x, y = (f[0][k] - wq, f[2][k] - wq) if k == "g" else (f[0][k], f[2][k])
            # the staged split rounds differently; a tenth of the 100-step parity bound
            assert _rel_l2(x, y) <= FP32_TOL[name] / 10, k


def test_variant_contexts_refuse_what_covers_the_default_lb_only():
    shape = (8, 8, 8)
    for var in VARIANTS.values():
        sim = L.Simulation([shape], [_lib_params(shape, L.FP32, **_lib_kw(var))], seed=1)
        for call in (lambda: sim.set_path(L.lbcad.PATH_TWO_KERNEL), lambda: sim.set_tiles(1),
                     lambda: sim.set_tiles(6), lambda: sim.adjoint(2, 1)):
            with pytest.raises(L.LbcadError):
                call()
        cfg, ms = sim.autotune(1)
        assert cfg in (0, 3) and all(m < 0 for i, m in enumerate(ms) if i not in (0, 3))
        sim.step(2)


def test_all_options_together_match_the_oracle():
    shape = (20, 16, 12)
    kw = dict(R=4.0, p0=8.0, zeta=0.01)
    var = dict(lattice=15, lb_form=1)
    sim = L.Simulation([shape], [_lib_params(shape, L.FP64, **kw, **_lib_kw(var), integrator=L.HEUN,
                                             coupling=L.SYNC)], seed=4)
    sim.step(8)
    ref = _oracle(shape, seed=4, **kw, **var, integrator=1, coupling=1).step(8)
    _compare(sim.get_fields(0), ref, 15, True, 1e-12)


def test_d3q15_observables_and_checkpoint_roundtrip():
    shape = (16, 12, 10)
    kw = dict(R=4.0, p0=8.0)
    var = dict(lattice=15, lb_form=1)
    ref = _oracle(shape, seed=5, **kw, **var).step(3)
    sim = L.Simulation([shape], [_lib_params(shape, L.FP64, **kw, **_lib_kw(var))], seed=99)
    perm = _perm(15)
    sim.set_fields(0, {"g": ref.f[perm], "u": ref.u, "q": ref.q, "psi": ref.psi})
    assert np.array_equal(sim.get_fields(0)["g"], ref.f[perm])
    sim.step(4)
    ref.step(4)
    _compare(sim.get_fields(0), ref, 15, True, 1e-12)
    np.testing.assert_allclose(sim.observables(0), ref.observables(), rtol=1e-12, atol=1e-10)


def test_stress_form_stability_and_difference_from_body_force():
    """The two forms of Sec. 3 discretise the same momentum equation.  Measured on the
    droplet workload (32^3, FP64, the library's staged path): max |u| every 25 steps for
    each form and velocity set at tau = 1 and 1.5, and where both are stable the relative
    difference of the flows after 150 steps.  The numbers printed here are the ones quoted
    in the design notes."""
    shape = (32, 32, 32)
    out = {}
    for lat in (19, 15):
        for form in (0, 1):
            for tau in (1.0, 1.5):
                var = dict(lattice=lat, lb_form=form)
                sim = L.Simulation([shape], [_lib_params(shape, L.FP64, **KW0, tau=tau, **_lib_kw(var))], seed=1)
                um = []
                for _ in range(6):
                    sim.step(25)
                    um.append(float(np.abs(sim.get_fields(0, L.FIELD_U)["u"]).max()))
                out[(lat, form, tau)] = (um, sim.get_fields(0, L.FIELD_U | L.FIELD_Q))
                print("D3Q%d %s tau %.1f max|u| per 25 steps:" % (lat, "stress-eq" if form else "body-force", tau),
                      " ".join("%.2e" % v for v in um))
    # bounded where the measurements of this workload found each scheme stable
    for key in ((19, 0, 1.0), (19, 0, 1.5), (15, 0, 1.0), (19, 1, 1.5)):
        um = out[key][0]
        assert all(np.isfinite(um)) and max(um) < 0.02, key
    a, b = out[(19, 0, 1.5)][1], out[(19, 1, 1.5)][1]
    du, dq = _rel_l2(b["u"], a["u"]), _rel_l2(b["q"], a["q"])
    print("D3Q19 tau 1.5 after 150 steps, stress-eq vs body-force: rel L2 u %.3e, Q %.3e" % (du, dq))
    # the order parameter, driven by the same free energy, stays close; the small flows (max |u|
    # a few 1e-3, mostly interface currents) differ at order one between the two discretisations
    assert dq < 0.1 and du < 2.0
