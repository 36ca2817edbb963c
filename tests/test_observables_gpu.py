"""The a6 sums (FP64 mass, sum psi, momentum, centroid moments of phi_c) as the fused step
computes them, in every block's warps and column segments, against the separate reduction
pass over the stored state, and against the oracle.

After a step on the fused path lbcad_observables returns the sums the step kernel produced;
setting the state (here: the raw state onto itself) makes it run the separate pass instead.
The two add the same quantities in different orders and, for the momentum, from different
but equal expressions (the post-collision momentum j + F of each site against the sum of the
stored populations times c_i), so FP64 agrees to rounding and FP32 to its resolution.
"""
import numpy as np
import pytest

import paper_2011_00287_gb300 as L
from oracle import oracle as O
from tests.test_parity_gpu import KW0, _lib_params, _oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2011_00287_gb300 import build as B
    B.build()
    O.build()


def _fused_and_separate(sim, inst):
    a = sim.observables(inst)
    sim.set_state(inst, sim.get_state(inst))
    b = sim.observables(inst)
    return a, b


def _check(a, b, N, fp64):
    if fp64:
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-10)
        return
    # FP32 states: mass and psi sums to 1e-7 per site, momentum to 1e-9 per site, the
    # centroid moments to 1e-7 per site
    assert abs(a[0] - b[0]) <= 1e-7 * N and abs(a[1] - b[1]) <= 1e-7 * N, (a, b)
    assert np.abs(a[2:5] - b[2:5]).max() <= 1e-9 * N, (a, b)
    assert np.abs(a[5:] - b[5:]).max() <= 1e-7 * N, (a, b)


CASES = [("fp64", L.FP64, 0), ("fp32-32x8", L.FP32, 0), ("fp32-pipelined", L.FP32, 3), ("fp32-32x16", L.FP32, 1)]


@pytest.mark.parametrize("name,prec,tiles", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("shape", [(32, 32, 32), (21, 13, 10), (40, 18, 12), (4, 5, 6), (8, 4, 4)])
def test_fused_sums_match_the_separate_pass(shape, name, prec, tiles):
    """Includes the smallest boxes (edges of 4): many short column segments per block, so
    many a6 slots per instance, and tiles far larger than the box."""
    sim = L.Simulation([shape], [_lib_params(shape, prec, R=5.0, p0=8.0, zeta=0.01)], seed=3)
    sim.set_tiles(tiles)
    sim.step(7)
    a, b = _fused_and_separate(sim, 0)
    _check(a, b, sim.sites(0), prec == L.FP64)


@pytest.mark.parametrize("variant", [dict(lattice=L.D3Q15), dict(lb_form=L.LB_STRESS_EQ, tau=1.5),
                                     dict(lattice=L.D3Q15, lb_form=L.LB_STRESS_EQ, tau=2.5)],
                         ids=["d3q15", "stress-eq", "d3q15-stress-eq"])
@pytest.mark.parametrize("prec", [L.FP64, L.FP32])
def test_fused_sums_of_the_lb_variants(variant, prec):
    shape = (24, 20, 16)
    sim = L.Simulation([shape], [_lib_params(shape, prec, R=5.0, p0=8.0, zeta=0.01, **variant)], seed=4)
    sim.step(6)
    a, b = _fused_and_separate(sim, 0)
    _check(a, b, sim.sites(0), prec == L.FP64)


def test_fused_sums_match_the_oracle_fp64():
    shape = (32, 32, 32)
    sim = L.Simulation([shape], [_lib_params(shape, L.FP64, **KW0)], seed=1)
    ref = _oracle(shape, seed=1, **KW0)
    for n in (1, 9):
        sim.step(n)
        ref.step(n)
        np.testing.assert_allclose(sim.observables(0), ref.observables(), rtol=1e-12, atol=1e-10)


@pytest.mark.parametrize("prec", [L.FP64, L.FP32])
def test_batch_graph_sums_per_instance(prec):
    """Uneven instances in one launch, steps replayed from a CUDA graph: every instance's
    fused sums against its separate pass (instances share column segments of blocks)."""
    shapes = [(16, 12, 10), (12, 12, 12), (20, 8, 14), (8, 24, 8), (16, 16, 4)]
    prm = [_lib_params(s, prec, R=3.0, p0=8.0, zeta=0.002 * (i + 1)) for i, s in enumerate(shapes)]
    sim = L.Simulation(shapes, prm, seed=9)
    sim.set_graph(2)
    sim.step(8)
    fused = [sim.observables(i) for i in range(len(shapes))]
    for i in range(len(shapes)):
        sim.set_state(i, sim.get_state(i))
    for i in range(len(shapes)):
        _check(fused[i], sim.observables(i), sim.sites(i), prec == L.FP64)


def test_sums_follow_the_state():
    """The fused sums describe the state after the last step: setting fields makes the
    next call see the new state, and stepping again brings the fused sums back."""
    shape = (16, 16, 16)
    sim = L.Simulation([shape], [_lib_params(shape, L.FP64, R=4.0, p0=8.0)], seed=2)
    sim.step(3)
    f = sim.get_fields(0, L.FIELD_PSI)
    f["psi"] = f["psi"] + 0.25
    sim.set_fields(0, f)
    o = sim.observables(0)
    assert abs(o[1] - f["psi"].sum()) <= 1e-9 * f["psi"].size
    sim.step(1)
    a, b = _fused_and_separate(sim, 0)
    _check(a, b, sim.sites(0), True)


@pytest.mark.parametrize("prec,tiles", [(L.FP32, 3), (L.FP32, 0), (L.FP64, 0)])
def test_sums_off_leave_the_state_unchanged(prec, tiles):
    """The step kernels without the sums write the same state bit for bit; observables then
    come from the separate pass and agree with the fused sums to rounding."""
    shape = (40, 18, 12)
    a = L.Simulation([shape], [_lib_params(shape, prec, R=5.0, p0=8.0, zeta=0.01)], seed=3)
    b = L.Simulation([shape], [_lib_params(shape, prec, R=5.0, p0=8.0, zeta=0.01)], seed=3)
    for s_ in (a, b):
        s_.set_tiles(tiles)
    b.set_observe(False)
    a.step(9)
    b.step(9)
    fa, fb = a.get_fields(0), b.get_fields(0)
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    _check(a.observables(0), b.observables(0), a.sites(0), prec == L.FP64)
