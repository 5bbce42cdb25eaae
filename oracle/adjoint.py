"""Compliance and its gradient w.r.t. per-cell strut radii (oracle; TEST INFRASTRUCTURE ONLY).

The loads do not depend on r_s, so compliance c = sum_loads f^T u is
self-adjoint: dc/dr_s = -sum_loads u^(s)T (dK^(s)/dr_s) u^(s), where
dK^(s)/dr_s is Eq. 52 assembled with dE/dr_s in place of E (K^(s) is
linear in the material field).  Not part of the paper; it is the
differentiation pattern the hot path carries.
"""
from __future__ import annotations

import numpy as np

from .discretization import Lattice


def compliance(lat: Lattice, u_cells: np.ndarray) -> np.ndarray:
    """c_l = f_l^T u_l per load case, from cell-duplicated vectors (n_rhs, N, n_dof)."""
    c = np.zeros(u_cells.shape[0])
    for s in range(lat.N):
        f = lat.load(s)
        c += (f * u_cells[:, s, :]).sum(1)
    return c


def gradient(lat: Lattice, u_cells: np.ndarray, w_cells: np.ndarray = None) -> np.ndarray:
    """g[l, s] = -w_l^(s)T dK^(s)/dr_s u_l^(s) (w = u for compliance)."""
    w_cells = u_cells if w_cells is None else w_cells
    g = np.zeros((u_cells.shape[0], lat.N))
    for s in range(lat.N):
        dK = lat.stiffness(s, dE_dr=True)
        for l in range(u_cells.shape[0]):
            g[l, s] = -w_cells[l, s] @ (dK @ u_cells[l, s])
    return g
