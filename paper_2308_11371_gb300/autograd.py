"""Compliance of a lattice as a differentiable function of its per-cell strut radii.

``cell_compliance(r, problem, ...)`` returns the compliance c_l = sum_s f_l^(s)T u_l^(s) of every
load case, where u solves the lattice problem with radii ``r`` (one entry per cell).  Its backward
gives dc_l/dr_s = -u_l^(s)T (dK^(s)/dr_s) u_l^(s).  The loads do not depend on r, so compliance is
self-adjoint: the adjoint state is the forward solution itself, and the gradient needs no second
solve.  Every step runs in the CUDA library (fetidp_setup, fetidp_solve, fetidp_compliance,
fetidp_grad); this module only moves tensors.

``recompute=True`` keeps nothing per cell between the passes: the backward runs setup and solve
again (for lattices whose states should not stay resident).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import binding
from .workloads import LatticeProblem


def _forward_state(r, problem: LatticeProblem, precision: int, options: dict):
    """Solve with radii r; returns (compliance [n_rhs] numpy, gradient [n_rhs][N] device tensor)."""
    prob = dataclasses.replace(problem, r_cell=np.asarray(r.detach().cpu().numpy(), dtype=np.float64).copy())
    s = binding.Solver(prob, precision=precision, **options)
    try:
        u, _, _ = s.solve()
        c = s.compliance(u)
        g = s.grad(u)
    finally:
        s.close()
    return c, g


def _function():
    import torch

    class CellCompliance(torch.autograd.Function):
        @staticmethod
        def forward(ctx, r, problem, precision, options, recompute):
            c, g = _forward_state(r, problem, precision, options)
            ctx.problem, ctx.precision, ctx.options, ctx.recompute = problem, precision, options, recompute
            if recompute:
                ctx.save_for_backward(r.detach().clone())
            else:
                ctx.save_for_backward(g)
            return torch.as_tensor(c, dtype=r.dtype, device=r.device)

        @staticmethod
        def backward(ctx, grad_c):
            (saved,) = ctx.saved_tensors
            if ctx.recompute:
                _, g = _forward_state(saved, ctx.problem, ctx.precision, ctx.options)
            else:
                g = saved
            gr = (grad_c.to(device=g.device, dtype=g.dtype)[:, None] * g).sum(0)
            return gr, None, None, None, None

    return CellCompliance


_CELL_COMPLIANCE = None


def cell_compliance(r, problem: LatticeProblem, precision: int = binding.FETIDP_FP64, options: dict = None,
                    recompute: bool = False):
    """Compliance per load case (tensor [n_rhs]) of ``problem`` with per-cell radii ``r``
    (tensor [N], any device); differentiable with respect to ``r``."""
    global _CELL_COMPLIANCE
    if _CELL_COMPLIANCE is None:
        _CELL_COMPLIANCE = _function()
    return _CELL_COMPLIANCE.apply(r, problem, precision, dict(options or {}), recompute)
