"""Monolithic direct solve (oracle; TEST INFRASTRUCTURE ONLY).

The plain definition of the discrete solution: assemble Eq. 5 over all
cells on the unique global nodes, eliminate clamped DOF (Eq. 3c with
u_0 = 0) and solve with a sparse direct library routine.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .discretization import Lattice


def assemble_global(lat: Lattice, stiffness=None):
    """Global K (unique DOF) and f (n_rhs columns) assembled cell by cell."""
    d, ref = lat.dim, lat.ref
    n_glob = lat.n_global_nodes * d
    rows, cols, vals = [], [], []
    f = np.zeros((lat.prob.n_rhs, n_glob))
    for s in range(lat.N):
        K = (stiffness(s) if stiffness is not None else lat.stiffness(s)).tocoo()
        g = (lat.cell_global_nodes[s][:, None] * d + np.arange(d)[None, :]).ravel()
        rows.append(g[K.row]); cols.append(g[K.col]); vals.append(K.data)
        fs = lat.load(s)
        for li in range(fs.shape[0]):
            np.add.at(f[li], g, fs[li])
    Kg = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(n_glob, n_glob))
    Kg.sum_duplicates()
    return Kg, f


def clamped_dofs(lat: Lattice) -> np.ndarray:
    d = lat.dim
    ca, cs = lat.prob.clamp_axis, lat.prob.clamp_side
    gd, gs = lat.global_node_dims, lat.global_node_strides
    coord = (np.arange(lat.n_global_nodes) // gs[ca]) % gd[ca]
    nodes = np.nonzero(coord == (0 if cs == 0 else gd[ca] - 1))[0]
    return (nodes[:, None] * d + np.arange(d)[None, :]).ravel()


def solve(lat: Lattice):
    """u* on the global DOF (n_rhs, n_glob) with clamped DOF = 0."""
    K, f = assemble_global(lat)
    fixed = clamped_dofs(lat)
    free = np.setdiff1d(np.arange(K.shape[0]), fixed)
    Kff = K[free][:, free].tocsc()
    lu = spla.splu(Kff)
    u = np.zeros_like(f)
    for li in range(f.shape[0]):
        u[li, free] = lu.solve(f[li, free])
    return u


def to_cells(lat: Lattice, u_glob: np.ndarray) -> np.ndarray:
    """Global DOF vector(s) -> cell-duplicated local vectors (n_rhs, N, n_dof), natural order."""
    d = lat.dim
    g = (lat.cell_global_nodes[:, :, None] * d + np.arange(d)[None, None, :]).reshape(lat.N, -1)
    return u_glob[:, g]
