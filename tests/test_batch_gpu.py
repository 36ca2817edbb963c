"""The batched workload: 64 independent droplets with box edges drawn from
{48, 64, 80, 96} per axis, advanced by one persistent launch per step (CUDA graph,
autotuned tiles).  Sampled instances are checked against the oracle run alone; every
instance conserves mass and psi."""
import numpy as np
import pytest

import paper_2011_00287_gb300 as L
from paper_2011_00287_gb300 import workloads as WL
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _perm():
    cl, _ = L.lattice()
    co, _ = O.lattice()
    return np.array([int(np.where((co == v).all(1))[0][0]) for v in cl])


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_batch_64_uneven_fp32_sampled_parity_and_conservation():
    work = WL.batch_uneven(seed=7, count=64)
    prms = [L.default_params(w["grid"], R=w["R"], p0=w["p0"], zeta=w["zeta"], precision=L.FP32) for w in work]
    sim = L.Simulation([w["grid"] for w in work], prms, seed=7)
    sim.autotune(2)
    sim.set_graph(2)
    o0 = [sim.observables(i) for i in range(64)]
    sim.step(4)
    # sample: the two smallest boxes against the oracle run of that instance alone
    sizes = [np.prod(w["grid"]) for w in work]
    _, w_ = O.lattice()
    for i in np.argsort(sizes)[:2]:
        w = work[i]
        ref = O.State(w["grid"], O.default_params(w["grid"], R=w["R"], p0=w["p0"], zeta=w["zeta"]),
                      seed=7, inst=int(i)).step(4)
        got = sim.get_fields(int(i))
        assert _rel(got["g"] - w_[_perm()].reshape(19, 1, 1, 1), ref.f[_perm()] - w_[_perm()].reshape(19, 1, 1, 1)) < 1e-5
        assert _rel(got["q"], ref.q) < 1e-5 and _rel(got["psi"], ref.psi) < 1e-5 and _rel(got["u"], ref.u) < 1e-5
    sim.step(16)
    for i in range(64):
        o1 = sim.observables(i)
        n = sizes[i]
        assert abs(o1[0] - o0[i][0]) < 1e-9 * n
        assert abs(o1[1] - o0[i][1]) < 1e-6 * n
