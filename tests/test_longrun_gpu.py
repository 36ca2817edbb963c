"""Long-run checks of the FP32 path against the FP64 GPU path.

- The 128^3 droplet workload (R = 32, pitch 32), 10^4 steps: the mean droplet speed and the
  defect count, averaged over the last 20% of the run, agree within 2%.  At this horizon the
  droplet has barely moved (0.002 lattice units at zeta = 0.005), so the speed is mostly
  centroid jitter while the defect structure forms.
- Propulsion (Sec. 4: the chiral active droplet rotates and swims along its helix axis): a
  64^3 box, R = 16, pitch 32, zeta = 0.005, run for 60,000 steps.  After a transient of about
  10,000 steps the droplet swims steadily along z (about 2e-4 lattice units per step).  The drift
  velocity, fitted over steps 20,000-60,000, and the displacement agree within 2%, and the
  displacement is many lattice units.
"""
import numpy as np
import pytest

import paper_2011_00287_gb300 as L
from paper_2011_00287_gb300 import observables as OB

pytestmark = pytest.mark.gpu

N_STEPS = 10000
EVERY = 100
DEFECT_EVERY = 500


def _run(prec, zeta):
    n = 128
    prm = L.default_params((n, n, n), R=32.0, p0=32.0, precision=prec, zeta=zeta)
    sim = L.Simulation([(n, n, n)], [prm], seed=1)
    sim.set_graph(EVERY)
    xs, defects = [OB.centroid(sim.observables(0), (n, n, n))], []
    for t in range(EVERY, N_STEPS + 1, EVERY):
        sim.step(EVERY)
        xs.append(OB.centroid(sim.observables(0), (n, n, n)))
        if t >= 0.8 * N_STEPS and t % DEFECT_EVERY == 0:
            f = sim.get_fields(0, L.FIELD_Q | L.FIELD_PSI)
            defects.append(OB.defect_count(f["q"], f["psi"]))
    traj = OB.unwrap_trajectory(np.array(xs), (n, n, n))
    sim.close()
    return OB.mean_speed(traj, EVERY), float(np.mean(defects)), traj


ZETAS = (0.002, 0.005)


@pytest.fixture(scope="module")
def longrun():
    """Both precisions at both activities, run once for the tests below."""
    return {z: {prec: _run(prec, z) for prec in (L.FP64, L.FP32)} for z in ZETAS}


@pytest.mark.parametrize("zeta", ZETAS)
def test_fp32_long_run_observables_match_fp64(longrun, zeta):
    (v64, d64, t64), (v32, d32, t32) = longrun[zeta][L.FP64], longrun[zeta][L.FP32]
    print("zeta %.3f: speed fp64 %.6e fp32 %.6e; defects fp64 %.2f fp32 %.2f; drift fp64 %s" % (
        zeta, v64, v32, d64, d32, np.round(t64[-1] - t64[0], 3)))
    assert abs(v32 - v64) <= 0.02 * v64
    assert abs(d32 - d64) <= 0.02 * max(d64, 1.0)


def test_speed_grows_with_activity(longrun):
    """Sec. 4 states, without numbers, that the droplet moves faster at higher activity: the mean
    speed at zeta = 0.005 exceeds the one at zeta = 0.002, in both precisions (measured 3.2e-7
    against 4.4e-8 lattice units per step)."""
    for prec in (L.FP64, L.FP32):
        assert longrun[0.005][prec][0] > longrun[0.002][prec][0], prec


PROP_STEPS, PROP_EVERY, PROP_FIT0 = 60000, 1000, 20000


def _propulsion(prec):
    n = 64
    prm = L.default_params((n, n, n), R=16.0, p0=32.0, precision=prec, zeta=0.005)
    sim = L.Simulation([(n, n, n)], [prm], seed=1)
    sim.set_graph(PROP_EVERY)
    xs, defects = [OB.centroid(sim.observables(0), (n, n, n))], []
    for t in range(PROP_EVERY, PROP_STEPS + 1, PROP_EVERY):
        sim.step(PROP_EVERY)
        xs.append(OB.centroid(sim.observables(0), (n, n, n)))
        if t >= 0.8 * PROP_STEPS and t % 4000 == 0:
            f = sim.get_fields(0, L.FIELD_Q | L.FIELD_PSI)
            defects.append(OB.defect_count(f["q"], f["psi"]))
    traj = OB.unwrap_trajectory(np.array(xs), (n, n, n))
    sim.close()
    t = np.arange(len(traj)) * PROP_EVERY
    sel = t >= PROP_FIT0
    # drift velocity: least-squares slope of each coordinate over the steady part
    vel = np.array([np.polyfit(t[sel], traj[sel, a], 1)[0] for a in range(3)])
    return vel, traj[-1] - traj[0], float(np.mean(defects))


def test_fp32_propulsion_matches_fp64():
    v64, d64, k64 = _propulsion(L.FP64)
    v32, d32, k32 = _propulsion(L.FP32)
    print("propulsion 64^3 zeta 0.005: velocity fp64 %s fp32 %s; displacement fp64 %s fp32 %s; defects %.2f %.2f" % (
        v64, v32, np.round(d64, 4), np.round(d32, 4), k64, k32))
    assert np.linalg.norm(d64) >= 1.0  # the droplet swims, by many lattice units
    assert np.linalg.norm(v32 - v64) <= 0.02 * np.linalg.norm(v64), (v32, v64)
    assert np.linalg.norm(d32 - d64) <= 0.02 * np.linalg.norm(d64), (d32, d64)
    assert abs(k32 - k64) <= 0.02 * max(k64, 1.0)
