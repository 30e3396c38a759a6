"""torch.autograd wrappers of the discrete adjoint (argument marshalling only;
the forward steps and the adjoint run in the CUDA library).

    U_T = rk_solve(U0, mu, solver, t0, dt, nsteps, max_snapshots=16)
    J = kinetic_energy(U_T, solver)
    J.backward()        # U0.grad = dJ/dU0, mu.grad = dJ/dmu

The backward pass runs the adjoint of the nsteps LSERK4-5 steps with binomial
checkpointing (at most max_snapshots stored states).
"""
from __future__ import annotations

import torch


class _RKSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, mu, solver, t0, dt, nsteps, max_snapshots):
        mu_val = float(mu)
        solver.set_viscosity(mu_val)
        U = U0.detach().clone()
        G = torch.empty_like(U)
        solver.rk_step(U, G, t0, dt, nsteps)
        ctx.save_for_backward(U0.detach().clone())
        ctx.solver, ctx.t0, ctx.dt, ctx.nsteps, ctx.snap = solver, t0, dt, nsteps, max_snapshots
        ctx.mu_shape = mu.shape
        ctx.mu = mu_val
        return U

    @staticmethod
    def backward(ctx, gU):
        (U0,) = ctx.saved_tensors
        dmu = torch.zeros(1, dtype=torch.float64, device=U0.device)
        # The adjoint recomputes the forward steps, so it must run with the
        # viscosity of this forward call, not whatever the solver holds now
        # (another rk_solve on the same solver may have changed it).
        solver = ctx.solver
        mu_now = solver.mu
        solver.set_viscosity(ctx.mu)
        try:
            lam0, _ = solver.adjoint_solve(U0, gU.contiguous(), ctx.t0, ctx.dt, ctx.nsteps, ctx.snap, dJdmu=dmu)
        finally:
            solver.set_viscosity(mu_now)
        return lam0, dmu.reshape(ctx.mu_shape), None, None, None, None, None


class _KineticEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, solver):
        g = torch.empty_like(U)
        J = solver.kinetic_energy(U.detach(), grad=g)
        ctx.save_for_backward(g)
        return torch.tensor(J, dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(ctx, gJ):
        (g,) = ctx.saved_tensors
        return gJ * g, None


def rk_solve(U0, mu, solver, t0, dt, nsteps, max_snapshots=16):
    """nsteps LSERK4-5 steps from U0 with viscosity mu (0-dim float64 tensor)."""
    return _RKSolve.apply(U0, mu, solver, float(t0), float(dt), int(nsteps), int(max_snapshots))


def kinetic_energy(U, solver):
    """Volume-integrated kinetic energy 1/2 rho |u|^2 (LGL quadrature)."""
    return _KineticEnergy.apply(U, solver)
