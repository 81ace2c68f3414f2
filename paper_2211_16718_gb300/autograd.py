"""torch.autograd bindings of the hand-written adjoint (argument marshalling only).

Each Function's forward and backward are single calls into libns3d.so: the right-hand
side and its vector-Jacobian product, one Runge-Kutta step and its reverse, a whole
trajectory (recorded with checkpoints, reversed by recomputing each segment), and the
kinetic-energy / enstrophy functionals with their gradients.  States are CUDA float64
tensors of shape (5, nz, ny, nx); the Solver fixes grid, parameters and integrator.
Gradients of a final-time statistic with respect to the initial fields, e.g.

    u0 = u0.requires_grad_()
    ke = functional(trajectory(u0, solver, dt, 256, every=16), solver, "ke")
    ke.backward()          # u0.grad = d KE(u_256) / d u0
"""
from __future__ import annotations

import torch

from .ns3d import Solver


class RHS(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, solver: Solver):
        u = u.detach().contiguous()
        ctx.solver = solver
        ctx.save_for_backward(u)
        return solver.rhs(u)

    @staticmethod
    def backward(ctx, g):
        (u,) = ctx.saved_tensors
        return ctx.solver.rhs_vjp(u, g.contiguous()), None


class RKStep(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, solver: Solver, dt: float, nsteps: int):
        u0 = u.detach().contiguous()
        ctx.solver, ctx.dt, ctx.nsteps = solver, float(dt), int(nsteps)
        ctx.save_for_backward(u0)
        out = u0.clone()
        solver.rk_step(out, dt, nsteps)  # the same launches as a recorded trajectory: the same bits
        return out

    @staticmethod
    def backward(ctx, g):
        (u0,) = ctx.saved_tensors
        gb = g.detach().contiguous().clone()
        if ctx.nsteps == 1:
            ctx.solver.rk_step_vjp(u0, gb, ctx.dt)
        elif ctx.nsteps > 1:
            out = u0.clone()
            ctx.solver.traj_forward(out, ctx.dt, ctx.nsteps, ctx.nsteps)
            ctx.solver.traj_vjp(gb)
        return gb, None, None, None


class Trajectory(torch.autograd.Function):
    """u_N = step^N(u_0) with checkpoints every `every` steps kept by the library; the
    backward reverses the recorded trajectory.  The library holds one recording per
    Solver: if another trajectory was recorded on the same Solver after this forward
    (a later trajectory() or rk_step(nsteps > 1) backward), this backward records its
    own again from the saved initial state before reversing it."""

    @staticmethod
    def forward(ctx, u, solver: Solver, dt: float, nsteps: int, every: int):
        u0 = u.detach().contiguous()
        out = u0.clone()
        solver.traj_forward(out, dt, nsteps, every)
        ctx.solver, ctx.args, ctx.generation = solver, (float(dt), int(nsteps), int(every)), solver.traj_generation
        ctx.save_for_backward(u0)
        return out

    @staticmethod
    def backward(ctx, g):
        (u0,) = ctx.saved_tensors
        gb = g.detach().contiguous().clone()
        if ctx.solver.traj_generation != ctx.generation:
            dt, nsteps, every = ctx.args
            ctx.solver.traj_forward(u0.clone(), dt, nsteps, every)
        ctx.solver.traj_vjp(gb)
        return gb, None, None, None, None


class Functional(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, solver: Solver, which: str):
        u = u.detach().contiguous()
        value, grad = solver.functional(u, which, grad=True)
        ctx.save_for_backward(grad)
        return torch.tensor(value, dtype=torch.float64, device=u.device)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return grad * g, None, None


def rhs(u, solver: Solver):
    return RHS.apply(u, solver)


def rk_step(u, solver: Solver, dt: float, nsteps: int = 1):
    return RKStep.apply(u, solver, dt, nsteps)


def trajectory(u, solver: Solver, dt: float, nsteps: int, every: int = 16):
    return Trajectory.apply(u, solver, dt, nsteps, every)


def functional(u, solver: Solver, which: str = "ke"):
    return Functional.apply(u, solver, which)
