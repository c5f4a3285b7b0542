"""torch.autograd wrapper of a rollout: gradients by the library's discrete
adjoint (fe_adjoint), not by tracing.  Marshalling only: every step, solve and
adjoint sweep runs in the CUDA library."""
from __future__ import annotations

import numpy as np
import torch


class ImplicitRollout(torch.autograd.Function):
    """q_T, v_T = rollout(scale, loads).

    scale: [n_elems] per-element energy scale (Young's modulus / reference
    modulus at fixed nu); loads: [T, n] external nodal forces per step.
    fe: an FEContext created with keep_checkpoints=1; base_params: [3] or
    [n_elems, 3] parameters at scale 1; q0, v0: initial state ([n])."""

    @staticmethod
    def forward(ctx, scale, loads, fe, base_params, q0, v0):
        s = scale.detach().to("cpu", torch.float64).numpy()
        bp = np.asarray(base_params, dtype=np.float64)
        params = s[:, None] * (bp if bp.ndim == 2 else bp[None, :])
        fe.set_params(params)
        fe.set_state(np.asarray(q0, dtype=np.float64), np.asarray(v0, dtype=np.float64))
        fe.clear_checkpoints()
        P = loads.detach().to("cpu", torch.float64).numpy()
        q = np.empty(fe.n)
        v = np.empty(fe.n)
        for t in range(P.shape[0]):
            fe.step(np.ascontiguousarray(P[t]), q, v)
        ctx.fe = fe
        ctx.dev = scale.device
        return torch.from_numpy(q).to(scale.device), torch.from_numpy(v).to(scale.device)

    @staticmethod
    def backward(ctx, gq, gv):
        gq = np.ascontiguousarray(gq.detach().to("cpu", torch.float64).numpy())
        gv = None if gv is None else np.ascontiguousarray(gv.detach().to("cpu", torch.float64).numpy())
        ds, dp = ctx.fe.adjoint(gq, gv)
        return (torch.from_numpy(ds).to(ctx.dev), torch.from_numpy(dp).to(ctx.dev), None, None, None, None)


def rollout(scale, loads, fe, base_params, q0, v0):
    return ImplicitRollout.apply(scale, loads, fe, base_params, q0, v0)
