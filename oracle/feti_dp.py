"""Exact (standard) FETI-DP (oracle; TEST INFRASTRUCTURE ONLY).

Sec. 2.2.4, Eqs. 20-31: every K_rr^(s) is factorised, the interface
problem F lambda = d_bar (Eqs. 23-25) is solved by PCG with the
Dirichlet preconditioner (Eq. 30), then u_P (Eq. 21) and u_R (Eq. 20) are
recovered.  Also exposes the per-cell blocks and the global saddle-point
operator of Eq. 16 used by the inexact solver.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .discretization import Lattice


class CellBlocks:
    """Blocks of K^(s) in the (i, d, p) ordering (Eq. 12), and f^(s)."""

    def __init__(self, lat: Lattice, s: int, K=None):
        ref = lat.ref
        K = lat.stiffness_idp(s) if K is None else K
        nr = ref.n_r
        self.K = K
        self.Krr = K[:nr, :nr].tocsc()
        self.Krp = K[:nr, nr:].toarray()
        self.Kpp = K[nr:, nr:].toarray()
        f = lat.loads_idp(s)
        self.fr, self.fp = f[:, :nr], f[:, nr:]


def saddle_operator(lat: Lattice, blocks):
    """Matrix-free A (u_R, u_P, lambda) of Eq. 16 on stacked vectors (Eqs. 17-19)."""
    ref, N = lat.ref, lat.N
    nr, nd, npp = ref.n_r, ref.n_d, ref.n_p
    nR = N * nr
    Ap, Bd = lat.Ap, lat.Bd

    def apply(x):
        uR = x[:nR].reshape(N, nr)
        uP = x[nR:nR + lat.n_P]
        lam = x[nR + lat.n_P:]
        up = (Ap.T @ uP).reshape(N, npp)
        gd = (Bd.T @ lam).reshape(N, nd)
        yR = np.empty_like(uR)
        yp = np.empty((N, npp))
        for s in range(N):
            y = blocks[s].K @ np.concatenate([uR[s], up[s]])
            yR[s] = y[:nr]
            yR[s, ref.n_i:] += gd[s]                     # B_R^T lambda = T_rd B_d^T lambda
            yp[s] = y[nr:]
        yP = Ap @ yp.ravel()
        ylam = Bd @ uR[:, ref.n_i:].ravel()              # B u = sum_s B_d T_dr u_r
        return np.concatenate([yR.ravel(), yP, ylam])
    return apply


def saddle_rhs(lat: Lattice, blocks, rhs: int):
    """(f_R, f_P, d) of Eq. 16 with f_P = sum_s A_p f_p (Eq. 18), d = 0."""
    fR = np.concatenate([blocks[s].fr[rhs] for s in range(lat.N)])
    fP = lat.Ap @ np.concatenate([blocks[s].fp[rhs] for s in range(lat.N)])
    return np.concatenate([fR, fP, np.zeros(lat.L)])


def pcg(apply_A, apply_M, b, tol, max_it, x0=None, record=None):
    """Preconditioned conjugate gradient, stopping on ||r||_2 / ||r_0||_2 <= tol."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply_A(x) if x0 is not None else b.copy()
    r0 = np.linalg.norm(r)
    if r0 == 0.0:
        return x, 0
    z = apply_M(r)
    p = z.copy()
    rz = r @ z
    it = 0
    while it < max_it:
        q = apply_A(p)
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        rel = np.linalg.norm(r) / r0
        if record is not None:
            record.append(rel)
        if rel <= tol:
            break
        z = apply_M(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it


class StandardFETIDP:
    """Standard FETI-DP with exact local factorisations (Eqs. 20-31)."""

    def __init__(self, lat: Lattice, blocks=None):
        self.lat = lat
        ref = lat.ref
        self.blocks = blocks or [CellBlocks(lat, s) for s in range(lat.N)]
        nr, nd, ni = ref.n_r, ref.n_d, ref.n_i
        self.lu = [spla.splu(b.Krr) for b in self.blocks]
        # U_rp (Eq. 29) and S_pp (Eq. 22) per cell, S_PP assembled (Eq. 22)
        self.Urp = [lu.solve(b.Krp) for lu, b in zip(self.lu, self.blocks)]
        Spp = [b.Kpp - b.Krp.T @ U for b, U in zip(self.blocks, self.Urp)]
        Ap = lat.Ap
        S_blk = sp.block_diag([sp.csr_matrix(X) for X in Spp], format="csr")
        self.SPP = (Ap @ S_blk @ Ap.T).tocsc()
        self.SPP_lu = spla.splu(self.SPP)
        # Dirichlet Schur complements S_dd (Eq. 30)
        self.Sdd = []
        for b in self.blocks:
            Kii = b.Krr[:ni, :ni].toarray(); Kid = b.Krr[:ni, ni:].toarray()
            Kdd = b.Krr[ni:, ni:].toarray()
            self.Sdd.append(Kdd - Kid.T @ sla.solve(Kii, Kid, assume_a="pos"))
        self._nd, self._nr, self._ni = nd, nr, ni

    # K^{-1} applied through the block LDL^T of Eq. 17 (Eqs. 20-21)
    def K_inv(self, vR, vP):
        lat = self.lat
        N, nr, npp = lat.N, self._nr, lat.ref.n_p
        vR = vR.reshape(N, nr)
        c = np.concatenate([self.Urp[s].T @ vR[s] for s in range(N)])
        zP = self.SPP_lu.solve(vP - lat.Ap @ c)
        zp = (lat.Ap.T @ zP).reshape(N, npp)
        xR = np.stack([self.lu[s].solve(vR[s]) - self.Urp[s] @ zp[s] for s in range(N)])
        return xR.ravel(), zP

    def apply_F(self, lam):
        """F lambda = B K^{-1} B^T lambda (Eq. 26)."""
        lat = self.lat
        N, nr, ni = lat.N, self._nr, self._ni
        gd = (lat.Bd.T @ lam).reshape(N, -1)
        vR = np.zeros((N, nr)); vR[:, ni:] = gd
        xR, _ = self.K_inv(vR.ravel(), np.zeros(lat.n_P))
        return lat.Bd @ xR.reshape(N, nr)[:, ni:].ravel()

    def apply_MD(self, r):
        """Dirichlet preconditioner of Eq. 30."""
        lat = self.lat
        g = (lat.Bd.T @ lat.apply_D(r)).reshape(lat.N, -1)
        y = np.stack([self.Sdd[s] @ g[s] for s in range(lat.N)])
        return lat.apply_D(lat.Bd @ y.ravel())

    def solve(self, rhs=0, tol=1e-13, max_it=1000, record=None):
        """Eqs. 23-25 by PCG, then Eqs. 21 and 20. Returns (u_R, u_P, lambda, its)."""
        lat = self.lat
        N, nr = lat.N, self._nr
        fR = np.concatenate([b.fr[rhs] for b in self.blocks])
        fP = lat.Ap @ np.concatenate([b.fp[rhs] for b in self.blocks])
        # d_bar = -d + B K^{-1} f  (Eq. 25 written through K^{-1}, d = 0)
        xR, _ = self.K_inv(fR, fP)
        dbar = lat.Bd @ xR.reshape(N, nr)[:, self._ni:].ravel()
        lam, its = pcg(self.apply_F, self.apply_MD, dbar, tol, max_it, record=record)
        # (u_R, u_P) = K^{-1} (f - B^T lambda)   (Eqs. 20-21)
        gd = (lat.Bd.T @ lam).reshape(N, -1)
        vR = fR.reshape(N, nr).copy(); vR[:, self._ni:] -= gd
        uR, uP = self.K_inv(vR.ravel(), fP)
        return uR, uP, lam, its


def cell_vectors(lat: Lattice, uR, uP):
    """(u_R, u_P) -> cell-duplicated full local vectors in natural order, shape (N, n_dof)."""
    ref = lat.ref
    up = (lat.Ap.T @ uP).reshape(lat.N, ref.n_p)
    loc = np.concatenate([uR.reshape(lat.N, ref.n_r), up], axis=1)
    out = np.empty_like(loc)
    out[:, ref.perm] = loc
    return out
