"""torch.autograd wrappers around the C ABI: the ground state as a differentiable function
of the potential values at the cell quadrature points, and the (constant, symmetric) mass
operator.  Argument marshalling only: the forward solves and the backward (Hellmann-Feynman
reduction, adjoint PCG solve) run in the library's kernels (dd_potential_gradient)."""
from __future__ import annotations

import torch

from . import (dd_apply_operator, dd_cell_eigenpair, dd_coarse_build, dd_inverse_iterate, dd_lopcg,
               dd_potential_gradient, dd_set_potential, DD_OP_MASS)


class _GroundState(torch.autograd.Function):
    @staticmethod
    def forward(fctx, V, solver, method, kw, rtol_adjoint):
        fctx.set_materialize_grads(False)
        Vd = V.detach().contiguous()
        dd_set_potential(solver.ctx, Vd)
        dd_cell_eigenpair(solver.ctx)
        dd_coarse_build(solver.ctx)
        solver._potential_version = getattr(solver, "_potential_version", 0) + 1
        x = torch.ones(solver.info["ndof"], dtype=torch.float64, device=V.device)
        if method == "lopcg":
            lam = dd_lopcg(solver.ctx, x, **kw)[0]
        else:
            lam = dd_inverse_iterate(solver.ctx, x, **kw)[0]
        fctx.solver, fctx.lam, fctx.rtol = solver, lam, rtol_adjoint
        fctx.version = solver._potential_version
        fctx.save_for_backward(Vd, x)
        return torch.tensor(lam, dtype=torch.float64, device=V.device), x

    @staticmethod
    def backward(fctx, g_lam, g_phi):
        Vd, x = fctx.saved_tensors
        solver = fctx.solver
        if solver._potential_version != fctx.version:
            # the context has since been given another potential: restore this one
            dd_set_potential(solver.ctx, Vd)
            dd_cell_eigenpair(solver.ctx)
            dd_coarse_build(solver.ctx)
            solver._potential_version += 1
        gl = float(g_lam) if g_lam is not None else 0.0
        gp = g_phi.contiguous() if g_phi is not None else None
        dV = torch.empty_like(Vd)
        dd_potential_gradient(solver.ctx, x, fctx.lam, gl, gp, dV, fctx.rtol)
        return dV, None, None, None, None


def ground_state(V, solver, method="inverse_iteration", rtol_adjoint=1e-10, **kw):
    """(lambda, phi) of -Laplace + V on the solver's grid, differentiable in V (the values at
    the cell quadrature points, float64 tensor on the solver's device)."""
    return _GroundState.apply(V, solver, method, kw, rtol_adjoint)


class _Mass(torch.autograd.Function):
    @staticmethod
    def forward(fctx, x, solver):
        fctx.solver = solver
        y = torch.empty_like(x)
        dd_apply_operator(solver.ctx, DD_OP_MASS, x.detach().contiguous(), y)
        return y

    @staticmethod
    def backward(fctx, gy):
        gx = torch.empty_like(gy)
        dd_apply_operator(fctx.solver.ctx, DD_OP_MASS, gy.contiguous(), gx)
        return gx, None


def mass(x, solver):
    """M x with the Q1 mass matrix of the solver's grid (differentiable; M is symmetric)."""
    return _Mass.apply(x, solver)
