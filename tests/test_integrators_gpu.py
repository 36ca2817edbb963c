"""Heun predictor-corrector and sync coupling (Sec. 3) on the GPU against the FP64 oracle,
through the C ABI, on the fused split and the staged path.

Tolerances as for the default step: FP64 within 1e-12 max abs per field after 10 steps,
FP32 within 1e-5 relative L2 per field after 100 steps.
"""
import numpy as np
import pytest

import paper_2011_00287_gb300 as L
from oracle import oracle as O
from tests.test_parity_gpu import KW0, _compare_fp32, _compare_fp64, _lib_params, _oracle, _rel_l2, _shifted

pytestmark = pytest.mark.gpu

VARIANTS = [
    dict(integrator=L.HEUN, coupling=L.LAGGED),
    dict(integrator=L.EULER, coupling=L.SYNC),
    dict(integrator=L.HEUN, coupling=L.SYNC),
]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2011_00287_gb300 import build as B
    B.build()
    O.build()


@pytest.mark.parametrize("path", ["default", "staged"])
@pytest.mark.parametrize("var", VARIANTS, ids=["heun-lagged", "euler-sync", "heun-sync"])
@pytest.mark.parametrize("shape,kw", [
    ((32, 32, 32), KW0),
    ((21, 13, 10), dict(R=4.0, p0=8.0, zeta=0.01, W=0.05)),
    ((4, 5, 6), dict(R=2.0, p0=6.0)),
])
def test_fp64_parity_10_steps(shape, kw, var, path):
    """By default on the fused path (the LB half in the fused kernel, then the
    order-parameter kernels), or staged."""
    sim = L.Simulation([shape], [_lib_params(shape, L.FP64, **kw, **var)], seed=2)
    if path == "staged":
        sim.set_path(L.lbcad.PATH_STAGED)
    sim.step(10)
    ref = _oracle(shape, seed=2, **kw, **var).step(10)
    _compare_fp64(sim.get_fields(0), ref)


@pytest.mark.parametrize("var", VARIANTS, ids=["heun-lagged", "euler-sync", "heun-sync"])
def test_fp32_parity_100_steps(var):
    shape = (32, 32, 32)
    sim = L.Simulation([shape], [_lib_params(shape, L.FP32, **KW0, **var)], seed=1)
    sim.step(100)
    ref = _oracle(shape, seed=1, **KW0, **var).step(100)
    errs = _compare_fp32(sim.get_fields(0), ref)
    print(var, "fp32 rel L2 after 100 steps:", errs)


def test_variants_differ_from_the_default_step():
    """The three variants give different trajectories from Euler/lagged (so the flags
    reach the kernels), by more than the FP64 parity tolerance."""
    shape = (16, 16, 16)
    kw = dict(R=5.0, p0=8.0, zeta=0.01)
    base = L.Simulation([shape], [_lib_params(shape, L.FP64, **kw)], seed=3).step(6).get_fields(0)
    for var in VARIANTS:
        got = L.Simulation([shape], [_lib_params(shape, L.FP64, **kw, **var)], seed=3).step(6).get_fields(0)
        assert np.abs(got["q"] - base["q"]).max() > 1e-9, var


@pytest.mark.parametrize("prec", [L.FP32, L.FP64])
def test_staged_euler_lagged_agrees_with_fused(prec):
    """Euler/lagged on the staged path evaluates the same per-site functions in a
    different kernel split: agreement to rounding with the fused path."""
    shape = (40, 18, 12)
    kw = dict(R=5.0, p0=8.0, zeta=0.01)
    a = L.Simulation([shape], [_lib_params(shape, prec, **kw)], seed=3)
    b = L.Simulation([shape], [_lib_params(shape, prec, **kw)], seed=3)
    b.set_path(L.lbcad.PATH_STAGED)
    a.step(20)
    b.step(20)
    fa, fb = a.get_fields(0), b.get_fields(0)
    for k in fa:
        if prec == L.FP64:
            assert np.abs(fa[k] - fb[k]).max() <= 1e-13, k
        else:
            x, y = (_shifted(fa[k]), _shifted(fb[k])) if k == "g" else (fa[k], fb[k])
            assert _rel_l2(x, y) <= 1e-6, k


@pytest.mark.parametrize("var", VARIANTS, ids=["heun-lagged", "euler-sync", "heun-sync"])
@pytest.mark.parametrize("prec", [L.FP32, L.FP64])
def test_split_agrees_with_the_staged_path(prec, var):
    """Heun or sync coupling: the fused split (the LB half in the fused kernel, then the
    order-parameter kernels; the default) and the staged path evaluate the same per-site
    functions in a different kernel split; agreement to rounding, also for a batch of uneven
    instances replayed from a graph."""
    shapes = [(40, 18, 12), (16, 12, 10)]
    kws = [dict(R=5.0, p0=8.0, zeta=0.01), dict(R=3.0, p0=8.0, zeta=0.004)]
    prm = [_lib_params(s_, prec, **k, **var) for s_, k in zip(shapes, kws)]
    a = L.Simulation(shapes, prm, seed=3)
    b = L.Simulation(shapes, prm, seed=3)
    b.set_path(L.lbcad.PATH_STAGED)
    a.set_graph(4)
    a.step(20)
    b.step(20)
    for i in range(len(shapes)):
        fa, fb = a.get_fields(i), b.get_fields(i)
        for k in fa:
            if prec == L.FP64:
                assert np.abs(fa[k] - fb[k]).max() <= 1e-13, (i, k)
            else:
                x, y = (_shifted(fa[k]), _shifted(fb[k])) if k == "g" else (fa[k], fb[k])
                assert _rel_l2(x, y) <= 1e-6, (i, k)


def test_batch_heun_sync_instances_match_oracle():
    shapes = [(16, 12, 10), (12, 12, 12)]
    kws = [dict(R=3.0, p0=8.0, zeta=0.002), dict(R=3.0, p0=12.0, zeta=0.008)]
    var = dict(integrator=L.HEUN, coupling=L.SYNC)
    sim = L.Simulation(shapes, [_lib_params(s, L.FP64, **k, **var) for s, k in zip(shapes, kws)], seed=9)
    sim.step(6)
    for i, (s, k) in enumerate(zip(shapes, kws)):
        ref = _oracle(s, seed=9, inst=i, **k, **var).step(6)
        _compare_fp64(sim.get_fields(i), ref)


def test_graph_replay_of_the_staged_step_is_bitwise_identical():
    shape = (20, 16, 12)
    kw = dict(R=4.0, p0=8.0, integrator=L.HEUN, coupling=L.SYNC)
    a = L.Simulation([shape], [_lib_params(shape, L.FP32, **kw)], seed=6)
    b = L.Simulation([shape], [_lib_params(shape, L.FP32, **kw)], seed=6)
    b.set_graph(4)
    a.step(11)
    b.step(11)
    fa, fb = a.get_fields(0), b.get_fields(0)
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k


def test_options_of_the_euler_lagged_step_are_refused():
    """Heun and sync contexts run the LB half on one fixed fused tile shape: tile choices, the
    two-kernel path and the adjoint are refused; the fused and staged paths both run."""
    shape = (8, 8, 8)
    for var in VARIANTS:
        sim = L.Simulation([shape], [_lib_params(shape, L.FP32, **var)], seed=1)
        for call in (lambda: sim.set_path(L.lbcad.PATH_TWO_KERNEL), lambda: sim.set_tiles(0),
                     lambda: sim.autotune(1), lambda: sim.adjoint(2, 1)):
            with pytest.raises(L.LbcadError):
                call()
        sim.step(1)
        sim.set_path(L.lbcad.PATH_STAGED)
        sim.step(1)
        sim.set_path(L.lbcad.PATH_FUSED)
        sim.step(1)
        assert np.isfinite(sim.observables(0)).all()
    with pytest.raises(L.LbcadError):
        L.Simulation([shape, shape], [_lib_params(shape, L.FP32), _lib_params(shape, L.FP32, coupling=L.SYNC)])
