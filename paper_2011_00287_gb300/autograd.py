"""torch.autograd.Function around lbcad_adjoint: the droplet's centroid displacement as a
differentiable function of the activity zeta, the chirality q0 and the initial Q field.

    J = CentroidDrift.apply(zeta, q0, Q0, shape, params, nsteps, ckpt_every, seed)
    J.backward()   # zeta.grad, q0.grad, Q0.grad from the adjoint kernels

The forward and the gradients both come from one lbcad_adjoint call (forward steps with
checkpoints, then the reverse sweep); this module only moves tensors across the ABI.
"""
from __future__ import annotations

import numpy as np
import torch

from .lbcad import FP64, Simulation


class CentroidDrift(torch.autograd.Function):
    @staticmethod
    def forward(ctx, zeta, q0, Q0, shape, params, nsteps: int, ckpt_every: int = 50, seed: int = 1):
        prm = dict(params)
        prm["zeta"] = float(zeta)
        prm["q0"] = float(q0)
        prm.setdefault("precision", FP64)
        sim = Simulation([tuple(shape)], [prm], seed=seed)
        try:
            sim.set_fields(0, {"q": Q0.detach().to("cpu", torch.float64).numpy()})
            J, dz, dq, dQ0 = sim.adjoint(int(nsteps), int(ckpt_every))
        finally:
            sim.close()
        ctx.save_for_backward(torch.tensor(dz, dtype=torch.float64), torch.tensor(dq, dtype=torch.float64),
                              torch.from_numpy(np.ascontiguousarray(dQ0)).to(Q0.device, Q0.dtype))
        ctx.dtypes = (zeta.dtype, q0.dtype)
        return torch.tensor(J, dtype=torch.float64, device=Q0.device)

    @staticmethod
    def backward(ctx, gJ):
        dz, dq, dQ0 = ctx.saved_tensors
        g = gJ.detach().to("cpu", torch.float64)
        return ((g * dz).to(ctx.dtypes[0]), (g * dq).to(ctx.dtypes[1]), gJ.to(dQ0.dtype) * dQ0,
                None, None, None, None, None)


def centroid_drift(zeta, q0, Q0, shape, params, nsteps, ckpt_every=50, seed=1):
    return CentroidDrift.apply(zeta, q0, Q0, shape, params, nsteps, ckpt_every, seed)
