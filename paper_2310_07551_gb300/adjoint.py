"""Differentiation of a horizon of EXPRK3DS_REAL steps through the library's
hand-written adjoint step (ds_step_backward), with step-level checkpointing.

Forward: m graph-replayed steps from U0 (ds_integrate_ckpt), keeping the
state every `ckpt` steps.
Backward: for each segment, last first, recompute the segment's states from
its checkpoint (ds_step) and sweep ds_step_backward over them in reverse,
accumulating dL/dU and dL/dp for the reaction parameters.  Memory: m/ckpt
checkpoints plus ckpt states of the segment being reversed.

The diffusion coefficients enter through a relative scaling s_c of each
component's matrices (A_{c,mu} -> s_c A_{c,mu} at s_c = 1): the library's
adjoint returns dL/ds_c through K and through every phi-matrix, and
dL/d delta_c = dL/ds_c / delta_c when A_{c,mu} = delta_c D_mu.
"""
from __future__ import annotations

import torch

from . import ds


class Integrate(torch.autograd.Function):
    """U_T = Integrate.apply(U0, p, s, plan, nsteps, ckpt).

    U0: CUDA float64 state (2, n_d, ..., n_1); p: float64 tensor (3,) holding
    the model parameters the plan was created with (its gradient is dL/dp);
    s: float64 tensor (2,) of ones, the scalings of the two components'
    matrices (its gradient is dL/ds).
    """

    @staticmethod
    def forward(ctx, U0, p, s, plan: ds.Plan, nsteps: int, ckpt: int):
        if plan.precision != "f64":
            raise ValueError("the adjoint needs an FP64 plan")
        U = U0.detach().contiguous().clone()
        ckpts = [U.clone()]
        ck = plan.integrate_ckpt(U, nsteps, ckpt)
        ckpts += [ck[j] for j in range(ck.shape[0]) if (j + 1) * ckpt < nsteps]
        ctx.plan, ctx.nsteps, ctx.ckpt, ctx.ckpts = plan, nsteps, ckpt, ckpts
        ctx.p_device = p.device
        ctx.want_s = bool(ctx.needs_input_grad[2])
        return U

    @staticmethod
    def backward(ctx, gU):
        plan, nsteps, ckpt = ctx.plan, ctx.nsteps, ctx.ckpt
        lam = gU.detach().contiguous().clone()
        dp = torch.zeros(3, dtype=torch.float64, device=lam.device)
        dsc = torch.zeros(2, dtype=torch.float64, device=lam.device) if ctx.want_s else None
        for seg in reversed(range(len(ctx.ckpts))):
            start = seg * ckpt
            end = min(start + ckpt, nsteps)
            states = [ctx.ckpts[seg]]
            U = ctx.ckpts[seg].clone()
            for _ in range(start, end - 1):
                plan.step(U)
                states.append(U.clone())
            for n in reversed(range(start, end)):
                lam = plan.step_backward(states[n - start], lam, dp, dsc)
        return (lam, dp.to(ctx.p_device), dsc.to(ctx.p_device) if dsc is not None else None,
                None, None, None)


def integrate(U0, p, plan: ds.Plan, nsteps: int, ckpt: int = 20, s=None):
    if s is None:
        s = torch.ones(2, dtype=torch.float64)
    return Integrate.apply(U0, p, s, plan, nsteps, ckpt)
