"""Long-run check of the FP32 path against the FP64 GPU path on the 128^3 droplet
workload (R = 32, pitch 32), 10^4 steps: the mean droplet speed and the defect count,
averaged over the last 20% of the run, agree within 2%."""
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


@pytest.mark.parametrize("zeta", [0.002, 0.005])
def test_fp32_long_run_observables_match_fp64(zeta):
    v64, d64, t64 = _run(L.FP64, zeta)
    v32, d32, t32 = _run(L.FP32, zeta)
    print("zeta %.3f: speed fp64 %.6e fp32 %.6e; defects fp64 %.2f fp32 %.2f; drift fp64 %s" % (
        zeta, v64, v32, d64, d32, np.round(t64[-1] - t64[0], 3)))
    assert abs(v32 - v64) <= 0.02 * v64
    assert abs(d32 - d64) <= 0.02 * max(d64, 1.0)
