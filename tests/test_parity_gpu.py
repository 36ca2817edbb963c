"""Parity of the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances: the FP64 GPU path within 1e-12 max abs per field after 10 steps; the FP32
path (populations shifted by w_i rho0) within 1e-5 relative L2 per field after 100
steps.  Populations are compared shifted (f_i - w_i rho0), which is the stricter test.
"""
import math

import numpy as np
import pytest

import paper_2011_00287_gb300 as L
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2011_00287_gb300 import build as B
    B.build()
    O.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _perm():
    """Index map from the library's D3Q19 order to the oracle's."""
    cl, _ = L.lattice()
    co, _ = O.lattice()
    return np.array([int(np.where((co == v).all(1))[0][0]) for v in cl])


def _oracle(shape, seed=1, inst=0, **kw):
    return O.State(shape, O.default_params(shape, **kw), seed=seed, inst=inst)


def _lib_params(shape, prec, **kw):
    return L.default_params(shape, precision=prec, **kw)


def _shifted(f):
    _, w = O.lattice()
    return f - w.reshape(19, 1, 1, 1)


def _compare_fp64(got, ref, tol=1e-12):
    perm = _perm()
    errs = {
        "g": np.abs(got["g"] - ref.f[perm]).max(),
        "q": np.abs(got["q"] - ref.q).max(),
        "psi": np.abs(got["psi"] - ref.psi).max(),
        "u": np.abs(got["u"] - ref.u).max(),
    }
    for k, e in errs.items():
        assert e <= tol, errs
    return errs


def _rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _compare_fp32(got, ref, tol=1e-5):
    perm = _perm()
    errs = {
        "g": _rel_l2(_shifted(got["g"]), _shifted(ref.f)[perm]),
        "q": _rel_l2(got["q"], ref.q),
        "psi": _rel_l2(got["psi"], ref.psi),
        "u": _rel_l2(got["u"], ref.u),
    }
    for k, e in errs.items():
        assert e <= tol, errs
    return errs


KW0 = dict(R=8.0, p0=16.0)  # droplet R = 8, pitch 16 in a 32^3 box


@pytest.mark.parametrize("prec", [L.FP64, L.FP32])
def test_initial_state_matches_oracle(prec):
    shape = (32, 32, 32)
    sim = L.Simulation([shape], [_lib_params(shape, prec, **KW0)], seed=3)
    got = sim.get_fields(0, L.FIELD_G | L.FIELD_RHO | L.FIELD_U | L.FIELD_Q | L.FIELD_PSI)
    ref = _oracle(shape, seed=3, **KW0)
    if prec == L.FP64:
        assert np.array_equal(got["q"], ref.q) and np.array_equal(got["psi"], ref.psi)
        assert np.array_equal(got["g"], ref.f[_perm()])
    else:
        assert np.array_equal(got["q"], ref.q.astype(np.float32).astype(np.float64))
        assert np.array_equal(got["psi"], ref.psi.astype(np.float32).astype(np.float64))
        assert np.abs(got["g"] - ref.f[_perm()]).max() < 1e-16 + 1e-7
    assert np.all(got["u"] == 0.0)
    np.testing.assert_allclose(got["rho"], 1.0, atol=1e-15)


@pytest.mark.parametrize("path", [L.lbcad.PATH_FUSED, L.lbcad.PATH_TWO_KERNEL])
@pytest.mark.parametrize("shape,kw", [
    ((32, 32, 32), KW0),
    ((21, 13, 10), dict(R=4.0, p0=8.0, zeta=0.01, W=0.05)),   # ragged, non-cubic, odd edges
    ((4, 5, 6), dict(R=2.0, p0=6.0)),                           # minimum edges: everything wraps
    ((70, 9, 40), dict(R=4.0, p0=10.0)),                        # several tiles in x, ragged y
])
def test_fp64_parity_10_steps(shape, kw, path):
    sim = L.Simulation([shape], [_lib_params(shape, L.FP64, **kw)], seed=2)
    sim.set_path(path)
    sim.step(10)
    ref = _oracle(shape, seed=2, **kw).step(10)
    _compare_fp64(sim.get_fields(0), ref)


def test_fp32_parity_100_steps():
    shape = (32, 32, 32)
    sim = L.Simulation([shape], [_lib_params(shape, L.FP32, **KW0)], seed=1)
    sim.step(100)
    ref = _oracle(shape, seed=1, **KW0).step(100)
    errs = _compare_fp32(sim.get_fields(0), ref)
    print("fp32 rel L2 after 100 steps:", errs)


def test_observables_match_oracle():
    shape = (24, 20, 16)
    kw = dict(R=5.0, p0=8.0)
    sim = L.Simulation([shape], [_lib_params(shape, L.FP64, **kw)], seed=4)
    sim.step(7)
    ref = _oracle(shape, seed=4, **kw).step(7)
    got = sim.observables(0)
    exp = ref.observables()
    np.testing.assert_allclose(got, exp, rtol=1e-12, atol=1e-10)


def test_batch_uneven_instances_match_separate_oracle_runs():
    shapes = [(16, 12, 10), (12, 12, 12), (20, 8, 9)]
    kws = [dict(R=3.0, p0=8.0, zeta=0.002), dict(R=3.0, p0=12.0, zeta=0.008), dict(R=2.5, p0=6.0, zeta=0.005)]
    sim = L.Simulation(shapes, [_lib_params(s, L.FP64, **k) for s, k in zip(shapes, kws)], seed=9)
    sim.step(6)
    for i, (s, k) in enumerate(zip(shapes, kws)):
        ref = _oracle(s, seed=9, inst=i, **k).step(6)
        _compare_fp64(sim.get_fields(i), ref)


def test_set_get_roundtrip_and_resume():
    """set_fields of the oracle state, then stepping, reproduces the oracle (checkpoint
    resume through the ABI)."""
    shape = (16, 12, 10)
    kw = dict(R=4.0, p0=8.0)
    ref = _oracle(shape, seed=5, **kw).step(3)
    sim = L.Simulation([shape], [_lib_params(shape, L.FP64, **kw)], seed=99)
    perm = _perm()
    inv = np.argsort(perm)
    sim.set_fields(0, {"g": ref.f[perm], "u": ref.u, "q": ref.q, "psi": ref.psi})
    got = sim.get_fields(0)
    assert np.array_equal(got["g"], ref.f[perm]) and np.array_equal(got["q"], ref.q)
    sim.step(4)
    ref.step(4)
    _compare_fp64(sim.get_fields(0), ref)
    assert inv.shape == (19,)


def test_graph_replay_is_bitwise_identical():
    shape = (20, 16, 12)
    kw = dict(R=4.0, p0=8.0)
    a = L.Simulation([shape], [_lib_params(shape, L.FP32, **kw)], seed=6)
    b = L.Simulation([shape], [_lib_params(shape, L.FP32, **kw)], seed=6)
    b.set_graph(4)
    a.step(11)
    b.step(11)
    fa, fb = a.get_fields(0), b.get_fields(0)
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    assert b.step_count == 11
    # a graph holds an even number of steps (a replay keeps the buffer parity): odd sizes are
    # rejected and the previous setting stays
    for bad in (3, -2):
        with pytest.raises(L.LbcadError):
            b.set_graph(bad)
    b.step(4)
    a.step(4)
    assert np.array_equal(a.get_fields(0, L.FIELD_Q)["q"], b.get_fields(0, L.FIELD_Q)["q"])


def test_fp32_conservation_at_bench_size():
    """128^3, R = 32, p0 = 32 (the benchmarked workload): the FP64 sums of mass, psi and momentum
    that the FP32 step forms stay conserved over 20 steps.  The sums add the FP32 per-site shares
    without rounding error (tested against host FP64 sums of the state in
    test_observables_gpu.py), so what drifts here is the FP32 state itself: its arithmetic
    conserves mass, psi and momentum only in exact arithmetic.
    - psi: each step rounds every site's new psi to FP32.  Most sites sit near psi = -1 or +1
      and change by less than half an ulp there, so the rounding is not a random walk: it drops
      the same small updates step after step (measured drift 0.024 over 20 steps, against the
      1.3e-3 that six standard deviations of a random walk would allow).  The bound is the
      worst case, half an ulp of a value below 2 in magnitude (2^-23) per site and step.
    - mass: the rounded values are the shifted populations, of order 1e-4 to 1e-3, and the
      collision's rounding errors do behave like a random walk: 5e-12 of N.
    - momentum: the same walk, plus the FP32 rounding of each site's force (whose exact sum is
      zero): 1e-10 of N."""
    shape = (128, 128, 128)
    steps = 20
    sim = L.Simulation([shape], [_lib_params(shape, L.FP32, R=32.0, p0=32.0)], seed=1)
    o0 = sim.observables(0)
    sim.step(steps)
    o1 = sim.observables(0)
    N = 128 ** 3
    print("128^3 FP32, 20 steps: drift of mass %.3e, psi %.3e, momentum %s" % (
        o1[0] - o0[0], o1[1] - o0[1], o1[2:5]))
    assert abs(o1[0] - o0[0]) < 5e-12 * N, (o0[0], o1[0])
    assert abs(o1[1] - o0[1]) <= N * steps * 2.0 ** -23, (o0[1], o1[1])
    assert np.abs(o1[2:5]).max() < 1e-10 * N, o1[2:5]


def test_fp32_parity_at_bench_size_2_steps():
    """Full-size parity: the 128^3 workload in the benchmarked launch configuration,
    two steps, every field against the oracle."""
    shape = (128, 128, 128)
    kw = dict(R=32.0, p0=32.0)
    sim = L.Simulation([shape], [_lib_params(shape, L.FP32, **kw)], seed=1)
    sim.autotune(2)  # as the benchmark does; the state is left where it was
    sim.step(2)
    ref = _oracle(shape, seed=1, **kw).step(2)
    _compare_fp32(sim.get_fields(0), ref, tol=1e-5)


def test_deterministic():
    shape = (16, 16, 16)
    kw = dict(R=4.0, p0=8.0)
    outs = []
    for _ in range(2):
        s = L.Simulation([shape], [_lib_params(shape, L.FP32, **kw)], seed=8)
        s.step(5)
        outs.append((s.get_fields(0), s.observables(0)))
    for k in outs[0][0]:
        assert np.array_equal(outs[0][0][k], outs[1][0][k])
    assert np.array_equal(outs[0][1], outs[1][1])


def test_invalid_instance_and_sizes_raise():
    shape = (8, 8, 8)
    sim = L.Simulation([shape], [_lib_params(shape, L.FP32)], seed=1)
    with pytest.raises(L.LbcadError):
        sim.get_fields(1)
    with pytest.raises(L.LbcadError):
        sim.observables(3)
    lib = L.library()
    import ctypes
    buf = np.zeros(10)
    assert lib.lbcad_get_fields(sim.ctx, 0, L.FIELD_Q, ctypes.c_void_p(buf.ctypes.data), buf.nbytes, 0) == \
        L.lbcad.LBCAD_E_INVALID_ARG


@pytest.mark.parametrize("prec", [L.FP32, L.FP64])
def test_fused_and_two_kernel_paths_agree(prec):
    """The fused kernel and the two-kernel path share the per-site arithmetic; their
    results agree to rounding (the compiler may contract differently)."""
    shape = (40, 18, 12)
    kw = dict(R=5.0, p0=8.0, zeta=0.01)
    a = L.Simulation([shape], [_lib_params(shape, prec, **kw)], seed=3)
    b = L.Simulation([shape], [_lib_params(shape, prec, **kw)], seed=3)
    b.set_path(L.lbcad.PATH_TWO_KERNEL)
    a.step(20)
    b.step(20)
    fa, fb = a.get_fields(0), b.get_fields(0)
    for k in fa:
        if prec == L.FP64:
            assert np.abs(fa[k] - fb[k]).max() <= 1e-13, k
        else:
            x, y = (_shifted(fa[k]), _shifted(fb[k])) if k == "g" else (fa[k], fb[k])
            assert _rel_l2(x, y) <= 1e-6, k


def test_path_switch_mid_run():
    shape = (24, 16, 12)
    kw = dict(R=4.0, p0=8.0)
    sim = L.Simulation([shape], [_lib_params(shape, L.FP64, **kw)], seed=5)
    sim.step(3)
    sim.set_path(L.lbcad.PATH_TWO_KERNEL)
    sim.step(3)
    sim.set_path(L.lbcad.PATH_FUSED)
    sim.step(2)
    ref = _oracle(shape, seed=5, **kw).step(8)
    _compare_fp64(sim.get_fields(0), ref)


def test_tile_shapes_and_autotune_give_identical_results():
    """The per-site arithmetic does not depend on the tile shape; autotuning times the
    shapes without advancing the state."""
    shape = (70, 36, 20)
    kw = dict(R=6.0, p0=10.0, zeta=0.01)
    ref = L.Simulation([shape], [_lib_params(shape, L.FP32, **kw)], seed=4)
    ref.step(5)
    fr = ref.get_fields(0)
    for cfg in range(L.lbcad.N_TILE_CONFIGS):
        s = L.Simulation([shape], [_lib_params(shape, L.FP32, **kw)], seed=4)
        s.set_tiles(cfg)
        s.step(5)
        f = s.get_fields(0)
        for k in fr:
            assert np.array_equal(f[k], fr[k]), (cfg, k)
    s = L.Simulation([shape], [_lib_params(shape, L.FP32, **kw)], seed=4)
    s.step(2)
    chosen, ms = s.autotune(3)
    assert 0 <= chosen < L.lbcad.N_TILE_CONFIGS and s.step_count == 2
    s.step(3)
    f = s.get_fields(0)
    for k in fr:
        assert np.array_equal(f[k], fr[k]), k


@pytest.mark.parametrize("prec", [L.FP32, L.FP64])
def test_raw_state_checkpoint_restores_bit_for_bit(prec):
    """lbcad_get_state / lbcad_set_state: an exact checkpoint in the storage precision, through
    host memory and through a device buffer."""
    import torch
    shape = (20, 12, 10)
    kw = dict(R=4.0, p0=8.0, zeta=0.01)
    sim = L.Simulation([shape], [_lib_params(shape, prec, **kw)], seed=7)
    sim.step(3)
    n = sim.state_bytes(0)
    assert n == (19 + 9) * 20 * 12 * 10 * (8 if prec == L.FP64 else 4)
    host = sim.get_state(0)
    dev = sim.get_state(0, out=torch.empty(n, dtype=torch.uint8, device="cuda"))
    sim.step(5)
    ref = sim.get_fields(0)
    for src in (host, dev):
        sim.set_state(0, src)
        sim.step(5)
        got = sim.get_fields(0)
        for k in ref:
            assert np.array_equal(got[k], ref[k]), k
    with pytest.raises(ValueError):
        sim.set_state(0, host[:10])
