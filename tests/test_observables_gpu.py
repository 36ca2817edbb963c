"""The a6 sums (FP64 mass, sum psi, momentum, centroid moments of phi_c) as the fused step
computes them, in every block's warps and column segments, against the separate reduction
pass over the stored state, and against the oracle.

After a step on the fused path lbcad_observables returns the sums the step kernel produced;
setting the state (here: the raw state onto itself) makes it run the separate pass instead.
The two add the same quantities in different orders and, for the momentum, from different
but equal expressions (the post-collision momentum j + F of each site against the sum of the
stored populations times c_i), so FP64 agrees to rounding and FP32 to its resolution.
"""
import math

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
    st = sim.get_state(inst)
    sim.set_state(inst, st)
    b = sim.observables(inst)
    # sum of |g| over the stored populations: the scale of the per-site rounding.  The raw state
    # holds (q + 9) values per site of the storage type: 112, 96, 224 or 192 bytes for
    # D3Q19/D3Q15 in FP32/FP64.
    N = sim.sites(inst)
    q, dt = {112: (19, np.float32), 96: (15, np.float32), 224: (19, np.float64), 192: (15, np.float64)}[st.nbytes // N]
    g = st.view(dt)[:q * N]
    return a, b, float(np.abs(g.astype(np.float64)).sum())


def _check(a, b, N, fp64, abs_g=0.0):
    if fp64:
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-10)
        return
    # FP32 states.  Both passes add their FP32 per-site shares without rounding error (error-free
    # pairs, then FP64).  psi, phi_c and its moments have the same shares on both sides, so they
    # agree to 1e-12 per site.  The fused mass and momentum come from the collision (each site's
    # pulled populations added in FP32, and j + F), the separate pass's from the stored
    # populations of each site added in FP32: both are sums of 19 FP32 values per site (each off
    # by at most 18 u sum|g_i|, u = 2^-24), and the stored populations carry the collision's own
    # rounding (a few u |g_i|).  So the two agree within 40 u sum|g| over the state.
    assert abs(a[1] - b[1]) <= 1e-12 * N and np.abs(a[5:] - b[5:]).max() <= 1e-12 * N, (a, b)
    tol = 40 * 2.0 ** -24 * abs_g
    assert abs(a[0] - b[0]) <= tol and np.abs(a[2:5] - b[2:5]).max() <= tol, (a, b, tol)


CASES = [("fp64", L.FP64, 0), ("fp32-32x8", L.FP32, 0), ("fp32-pipelined", L.FP32, 3), ("fp32-32x16", L.FP32, 1)]


@pytest.mark.parametrize("name,prec,tiles", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("shape", [(32, 32, 32), (21, 13, 10), (40, 18, 12), (4, 5, 6), (8, 4, 4)])
def test_fused_sums_match_the_separate_pass(shape, name, prec, tiles):
    """Includes the smallest boxes (edges of 4): many short column segments per block, so
    many a6 slots per instance, and tiles far larger than the box."""
    sim = L.Simulation([shape], [_lib_params(shape, prec, R=5.0, p0=8.0, zeta=0.01)], seed=3)
    sim.set_tiles(tiles)
    sim.step(7)
    a, b, ag = _fused_and_separate(sim, 0)
    _check(a, b, sim.sites(0), prec == L.FP64, ag)


@pytest.mark.parametrize("variant", [dict(lattice=L.D3Q15), dict(lb_form=L.LB_STRESS_EQ, tau=1.5),
                                     dict(lattice=L.D3Q15, lb_form=L.LB_STRESS_EQ, tau=2.5)],
                         ids=["d3q15", "stress-eq", "d3q15-stress-eq"])
@pytest.mark.parametrize("prec", [L.FP64, L.FP32])
def test_fused_sums_of_the_lb_variants(variant, prec):
    shape = (24, 20, 16)
    sim = L.Simulation([shape], [_lib_params(shape, prec, R=5.0, p0=8.0, zeta=0.01, **variant)], seed=4)
    sim.step(6)
    a, b, ag = _fused_and_separate(sim, 0)
    _check(a, b, sim.sites(0), prec == L.FP64, ag)


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
    states = [sim.get_state(i) for i in range(len(shapes))]
    for i in range(len(shapes)):
        sim.set_state(i, states[i])
    for i in range(len(shapes)):
        ag = float(np.abs(states[i].view(np.float32 if prec == L.FP32 else np.float64)[:19 * sim.sites(i)]
                          .astype(np.float64)).sum())
        _check(fused[i], sim.observables(i), sim.sites(i), prec == L.FP64, ag)


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
    a, b, _ = _fused_and_separate(sim, 0)
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
    ag = float(np.abs(a.get_state(0).view(np.float32 if prec == L.FP32 else np.float64)[:19 * a.sites(0)]
                      .astype(np.float64)).sum())
    _check(a.observables(0), b.observables(0), a.sites(0), prec == L.FP64, ag)


def _plane_fsum(x, planes):
    """FP64 sum of float32 values: pairwise float64 sums per plane (relative error ~1e-15),
    then an exact sum of the plane sums."""
    return math.fsum(np.sum(x.astype(np.float64).reshape(planes, -1), axis=1).tolist())


def _host_sums(sim, inst, rho0=1.0):
    """The twelve a6 quantities of the stored FP32 state, summed in FP64 on the host from the
    raw state, with |.| sums as scales: mass (N rho0 + the shifted populations), psi, momentum
    (sum_i c_i g_i), and phi_c = (1 + psi)/2 with its centroid moments, each site's phi_c and
    moment share formed in FP32 as the step forms it (numpy float32 arithmetic rounds to nearest,
    as the GPU does) with the FP32 cos/sin table the library builds from cos(2 pi x / L)."""
    nx, ny, nz = sim.grids[inst]
    N = nx * ny * nz
    raw = sim.get_state(inst).view(np.float32)
    g = raw[:19 * N].reshape(19, N)
    psi = raw[24 * N:25 * N]
    c, _ = L.lattice()
    one, half = np.float32(1.0), np.float32(0.5)
    h = (half * (one + psi)).astype(np.float32).reshape(nz, ny, nx)

    def table(n):
        ph = [2.0 * math.pi * x / n for x in range(n)]
        return (np.array([math.cos(v) for v in ph]).astype(np.float32),
                np.array([math.sin(v) for v in ph]).astype(np.float32))

    (cx, sx), (cy, sy), (cz, sz) = table(nx), table(ny), table(nz)
    shares = [h * cx[None, None, :], h * cy[None, :, None], h * cz[:, None, None],
              h * sx[None, None, :], h * sy[None, :, None], h * sz[:, None, None]]
    out = np.zeros(12)
    scale = np.zeros(12)
    out[0] = N * rho0 + _plane_fsum(g, nz)
    scale[0] = N * rho0 + _plane_fsum(np.abs(g), nz)
    out[1], scale[1] = _plane_fsum(psi, nz), _plane_fsum(np.abs(psi), nz)
    for a in range(3):
        ja = (c[:, a].astype(np.float32)[:, None] * g).astype(np.float32)
        out[2 + a], scale[2 + a] = _plane_fsum(ja, nz), _plane_fsum(np.abs(ja), nz)
    for k, sh in enumerate(shares):
        sh = sh.astype(np.float32)
        out[5 + k], scale[5 + k] = _plane_fsum(sh, nz), _plane_fsum(np.abs(sh), nz)
    out[11], scale[11] = _plane_fsum(h, nz), _plane_fsum(np.abs(h), nz)
    return out, scale, _plane_fsum(np.abs(g), nz)


@pytest.mark.parametrize("tiles", [3, 0], ids=["pipelined-8+8", "32x8"])
def test_fp32_fused_sums_are_the_fp64_sums_of_the_state(tiles):
    """The benchmarked workload (128^3, R = 32, pitch 32): the FP64 sums the FP32 step forms
    against FP64 sums of its stored state formed on the host.
    - psi, phi_c and the centroid moments: the same FP32 shares on both sides, so the sums agree to
      1e-12 relative (of the sum of |share|); the reduction in the kernel loses nothing.
    - mass: the step adds, at each site, the 19 pulled populations of the state it read; in exact
      arithmetic that is the mass of the state it writes.  It matches the read state's FP64 mass
      within the FP32 rounding of those 19-term sums (at most 18 u sum|g|, u = 2^-24) and both
      states' masses to 1e-12 relative.
    - momentum: the step adds j + F per site, the post-collision momentum; against sum_i c_i g_i of
      the written state to 1e-12 N."""
    shape = (128, 128, 128)
    N = 128 ** 3
    sim = L.Simulation([shape], [_lib_params(shape, L.FP32, R=32.0, p0=32.0)], seed=1)
    sim.set_tiles(tiles)
    sim.step(10)
    prev, _, abs_g_prev = _host_sums(sim, 0)
    sim.step(1)
    o = sim.observables(0)
    cur, scale, _ = _host_sums(sim, 0)
    for k in [1] + list(range(5, 12)):
        assert abs(o[k] - cur[k]) <= 1e-12 * scale[k], (k, o[k], cur[k], scale[k])
    u = 2.0 ** -24
    assert abs(o[0] - prev[0]) <= 18 * u * abs_g_prev, (o[0], prev[0], abs_g_prev)
    assert abs(o[0] - prev[0]) <= 1e-12 * prev[0] and abs(o[0] - cur[0]) <= 1e-12 * cur[0], (o[0], prev[0], cur[0])
    assert np.abs(o[2:5] - cur[2:5]).max() <= 1e-12 * N, (o[2:5], cur[2:5])
    sim.close()
