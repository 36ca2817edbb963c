"""Second workload: bulk active liquid crystal with no droplet (psi = 1 everywhere), the
regimes of Fig. 4 (Sec. 4): quiescent at low activity, a stationary spontaneous flow above a
threshold, and a chaotic flow with defects at high activity.  Same kernels as the droplet.

Parity: the FP64 GPU step against the oracle from the same initial state.  The regimes are
physics without a number in the paper (parity unpinned beyond the qualitative statements of
Sec. 4); the thresholds below were measured on this workload (32^3, FP32, 6000 steps) and
bracket the onset of flow between zeta = 0.002 and 0.004.
"""
import numpy as np
import pytest

import paper_2011_00287_gb300 as L
from paper_2011_00287_gb300 import observables as OB
from paper_2011_00287_gb300 import workloads as W
from oracle import oracle as O
from tests.test_parity_gpu import _compare_fp64, _lib_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2011_00287_gb300 import build as B
    B.build()
    O.build()


@pytest.mark.parametrize("q0", [0.0, 2 * np.pi / 16])
def test_bulk_fp64_parity_10_steps(q0):
    shape = (24, 20, 16)
    kw = dict(R=1.0, p0=16.0, zeta=0.02)
    st = W.bulk_order(shape, q0=q0, noise=1e-2, seed=5)
    prm = _lib_params(shape, L.FP64, **kw)
    prm["q0"] = q0
    sim = L.Simulation([shape], [prm], seed=1)
    sim.set_fields(0, st)
    op = O.default_params(shape, **kw)
    op.q0 = q0
    ref = O.State(shape, op, seed=1)
    ref.q, ref.psi = st["q"].copy(), st["psi"].copy()
    sim.step(10)
    ref.step(10)
    _compare_fp64(sim.get_fields(0), ref)


def _run_bulk(zeta, n=32, steps=6000, every=100, q0=0.0):
    shape = (n, n, n)
    prm = L.default_params(shape, R=1.0, p0=16.0, precision=L.FP32, zeta=zeta)
    prm["q0"] = q0
    sim = L.Simulation([shape], [prm], seed=1)
    sim.set_fields(0, W.bulk_order(shape, q0=q0, noise=1e-3, seed=3))
    sim.set_graph(every)
    ek = []
    for _ in range(steps // every):
        sim.step(every)
        u = sim.get_fields(0, L.FIELD_U)["u"]
        ek.append(float(0.5 * (u * u).sum(0).mean()))
    f = sim.get_fields(0, L.FIELD_Q | L.FIELD_PSI)
    sim.close()
    late = np.array(ek[2 * len(ek) // 3:])
    S = OB.scalar_order(f["q"])
    return dict(ek=late.mean(), relstd=float(late.std() / max(late.mean(), 1e-300)), smin=float(S.min()),
                defects=OB.defect_count(f["q"], f["psi"], psi_min=-2.0))


def test_bulk_nematic_regimes_of_fig4():
    r = {z: _run_bulk(z) for z in (0.0, 0.002, 0.004, 0.008, 0.032)}
    for z, v in r.items():
        print("bulk nematic 32^3 zeta %.3f: late <E_k> %.3e (rel std %.3f), S_min %.3f, defects %d"
              % (z, v["ek"], v["relstd"], v["smin"], v["defects"]))
    # quiescent: flows almost suppressed, order uniform
    for z in (0.0, 0.002):
        assert r[z]["ek"] < 1e-7 and r[z]["defects"] == 0 and r[z]["smin"] > 0.49
    # spontaneous flow: a stationary flow, no defects
    for z in (0.004, 0.008):
        assert 1e-6 < r[z]["ek"] < 1e-3 and r[z]["relstd"] < 0.1 and r[z]["defects"] == 0
    # chaotic: fluctuating flow and defects (regions of S < 0.25)
    assert r[0.032]["defects"] >= 5 and r[0.032]["smin"] < 0.3 and r[0.032]["relstd"] > 0.03
    assert r[0.032]["ek"] > r[0.008]["ek"] > r[0.004]["ek"]


def test_bulk_cholesteric_flows_and_defects_at_high_activity():
    lo, hi = _run_bulk(0.001, q0=2 * np.pi / 16), _run_bulk(0.032, q0=2 * np.pi / 16)
    print("bulk cholesteric 32^3: zeta 0.001 <E_k> %.3e defects %d; zeta 0.032 <E_k> %.3e defects %d"
          % (lo["ek"], lo["defects"], hi["ek"], hi["defects"]))
    assert lo["ek"] < 1e-9 and lo["defects"] == 0
    assert hi["ek"] > 1e-4 and hi["defects"] >= 5


def test_passive_nematic_relaxes_with_sync_coupling():
    """A passive nematic (zeta = 0) at rest with seeded noise is a dissipative system: its
    flow must die out.  With sync coupling (u of the same step advects Q) the kinetic energy
    decays monotonically to rounding level.  The default lagged coupling (u of the previous
    step, which lets the step fuse into one kernel) leaves a weak residual flow instead; the
    printed numbers are quoted in the design notes."""
    shape = (16, 16, 16)
    out = {}
    for name, coupling in (("sync", L.SYNC), ("lagged", L.LAGGED)):
        prm = L.default_params(shape, R=1.0, p0=16.0, precision=L.FP64, zeta=0.0, coupling=coupling)
        prm["q0"] = 0.0
        sim = L.Simulation([shape], [prm], seed=1)
        sim.set_fields(0, W.bulk_order(shape, q0=0.0, noise=1e-3, seed=3))
        ek = []
        for _ in range(15):
            sim.step(200)
            u = sim.get_fields(0, L.FIELD_U)["u"]
            ek.append(float(0.5 * (u * u).sum(0).mean()))
        out[name] = ek
        print("passive nematic 16^3, %s coupling, <E_k> every 200 steps:" % name, " ".join("%.1e" % v for v in ek))
        sim.close()
    e = out["sync"]
    assert e[-1] < 1e-15 and all(b <= a * 1.0001 for a, b in zip(e[2:], e[3:]))
