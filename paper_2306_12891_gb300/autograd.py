"""torch.autograd bindings of the solver's discrete adjoint (argument marshalling only).

    Ut = rhs(dg, U)                              backward: dg_rhs_vjp
    UK = lserk_steps(dg, U0, dt, K, interval)    forward: dg_lserk_steps_record (every stage state in HBM
                                                 when it fits, else checkpoints every `interval` steps);
                                                 backward: dg_lserk_steps_vjp_recorded
    KE = kinetic_energy(dg, U)                   sum J w rho|u|^2/2; backward: dg_kinetic_energy_grad

`dg` is a paper_2306_12891_gb300.dg.DG context (FP64, no shock capturing, KG or Pirozzoli volume
flux). The library computes every derivative in its CUDA kernels; nothing here differentiates.
"""
from __future__ import annotations

import torch


class _Rhs(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, dg):
        U = U.detach().contiguous()
        ctx.dg = dg
        ctx.save_for_backward(U)
        return dg.rhs(U)

    @staticmethod
    def backward(ctx, grad_out):
        (U,) = ctx.saved_tensors
        return ctx.dg.rhs_vjp(U, grad_out.detach().contiguous()), None


class _Steps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, dg, dt, n_steps, interval):
        U0 = U0.detach().contiguous()
        ctx.dg, ctx.dt, ctx.n_steps, ctx.interval = dg, float(dt), int(n_steps), int(interval)
        ctx.save_for_backward(U0)
        UK = U0.clone()
        if ctx.n_steps > 0:  # record the run (every stage state if it fits, else checkpoints)
            ctx.tape = dg.lserk_steps_record(UK, dt, n_steps, interval)
        return UK

    @staticmethod
    def backward(ctx, grad_out):
        (U0,) = ctx.saved_tensors
        Ubar = grad_out.detach().contiguous().clone()
        if ctx.n_steps > 0:
            # a later forward may have recorded over this run's tape: then recompute from U0. Any
            # error of the reverse sweep itself propagates (Ubar is partly reversed by then).
            if ctx.dg.tape_current() == ctx.tape:
                ctx.dg.lserk_steps_vjp_recorded(ctx.tape, Ubar)
            else:
                ctx.dg.lserk_steps_vjp(U0, Ubar, ctx.dt, ctx.n_steps, ctx.interval)
        return Ubar, None, None, None, None


class _KineticEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, dg):
        U = U.detach().contiguous()
        ctx.dg = dg
        ctx.save_for_backward(U)
        ke = dg.invariants(U, U)[6]  # out[6] depends on U only
        return torch.tensor(ke, dtype=U.dtype, device=U.device)

    @staticmethod
    def backward(ctx, grad_out):
        (U,) = ctx.saved_tensors
        return grad_out * ctx.dg.kinetic_energy_grad(U), None


def rhs(dg, U):
    return _Rhs.apply(U, dg)


def lserk_steps(dg, U0, dt, n_steps, interval=10):
    return _Steps.apply(U0, dg, dt, n_steps, interval)


def kinetic_energy(dg, U):
    return _KineticEnergy.apply(U, dg)
