"""torch.autograd bindings: theta -> J with the adjoint as the backward pass.

``ALBMFunction`` maps the porosity field theta (N float32 values) to the
objective J of one unsteady solve: forward runs the N primal steps (Eq.
normal:iteration) through the library and returns J (FP64); backward runs
the N adjoint steps (Eqs. adjoint:iteration / adjoint:operator, unsteady
form) and returns gJ * dJ/dtheta (Eq. adjoint:derivative).  States the
adjoint needs are kept or recomputed by the library's checkpoint schedule
under the solver's memory budget, so trajectories that do not fit in HBM are
handled by recomputation.

``ALBMBatchFunction`` does the same for many solvers at once: the primal and
adjoint steps of all solvers of one kernel family advance in batched
launches (one kernel per step for the whole batch).

Only argument marshalling happens here; every step runs in the CUDA library.
"""
from __future__ import annotations

import itertools

import torch

from .albm import Solver, batch_adjoint_step, batch_primal_step

_gen = itertools.count(1)


def _family(s: Solver):
    P = s.P
    return (P.lattice, P.collision, P.nscalars, P.precision, id(s.stream))


class ALBMFunction(torch.autograd.Function):
    """J = ALBMFunction.apply(theta, solver)."""

    @staticmethod
    def forward(ctx, theta, solver):
        solver.set_theta(theta.detach().reshape(-1).to(torch.float32))
        solver.primal_step(solver.P.nsteps)
        J = solver.objective()
        gen = next(_gen)
        solver._autograd_gen = gen
        ctx.solver, ctx.gen = solver, gen
        ctx.shape, ctx.dtype = theta.shape, theta.dtype
        return torch.tensor(J, dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(ctx, gJ):
        s = ctx.solver
        if getattr(s, "_autograd_gen", None) != ctx.gen:
            raise RuntimeError("the solver ran another forward pass since this graph was built")
        remaining = s.time if s.adjoint_time < 0 else s.adjoint_time
        s.adjoint_step(remaining)
        g = s.gradient()
        return (gJ.to(g.dtype) * g).to(ctx.dtype).reshape(ctx.shape), None


def albm_objective(theta: torch.Tensor, solver: Solver) -> torch.Tensor:
    """Differentiable objective of one solve (FP64 scalar tensor)."""
    return ALBMFunction.apply(theta, solver)


class ALBMBatchFunction(torch.autograd.Function):
    """Js = ALBMBatchFunction.apply(solvers, *thetas) -> (B,) FP64 tensor."""

    @staticmethod
    def forward(ctx, solvers, *thetas):
        groups = {}
        for s, th in zip(solvers, thetas):
            s.set_theta(th.detach().reshape(-1).to(torch.float32))
            groups.setdefault(_family(s), []).append(s)
        for ss in groups.values():
            batch_primal_step(ss, max(s.P.nsteps for s in ss))
        Js = [s.objective() for s in solvers]
        gen = next(_gen)
        for s in solvers:
            s._autograd_gen = gen
        ctx.solvers, ctx.gen, ctx.groups = solvers, gen, list(groups.values())
        ctx.meta = [(t.shape, t.dtype) for t in thetas]
        return torch.tensor(Js, dtype=torch.float64, device=thetas[0].device)

    @staticmethod
    def backward(ctx, gJ):
        for s in ctx.solvers:
            if getattr(s, "_autograd_gen", None) != ctx.gen:
                raise RuntimeError("a solver ran another forward pass since this graph was built")
        for ss in ctx.groups:
            batch_adjoint_step(ss, max(s.P.nsteps for s in ss))
        grads = []
        for k, (s, (shape, dtype)) in enumerate(zip(ctx.solvers, ctx.meta)):
            g = s.gradient()
            grads.append((gJ[k].to(g.dtype) * g).to(dtype).reshape(shape))
        return (None, *grads)


def albm_objectives(thetas, solvers):
    """Differentiable objectives of a batch of solves (FP64 tensor of shape (B,))."""
    return ALBMBatchFunction.apply(list(solvers), *thetas)
