"""ROM-based inexact FETI-DP (oracle; TEST INFRASTRUCTURE ONLY).

Outer Krylov solver on the saddle-point system of Eq. 16 (right-
preconditioned flexible GMRES, x_0 = 0, classical Gram-Schmidt with one
reorthogonalisation, Givens rotations) with the block preconditioner of
Eq. 44 applied by Algorithm 1:

    w_bar <- w - U_ring v                    (Algorithm 3)
    y     <- -F_ring^{-pcg} w_bar            (PCG on Eq. 48, preconditioner Eq. 49)
    x     <- K_ring^{-ROM} v - U_ring^T y    (Algorithm 2 with Eq. 46; U_ring^T below)

U_ring^T y is the transpose of Algorithm 3 (the paper writes
U_ring^T = K_ring^{-ROM} B^T "using the ROM dual solutions"):
    z_P  = S_PP^{-1}( - U_RP^T B_R^T y )
    out  = ( U_RD B_R^T y - U_RP z_P ,  z_P ).
The outer solver is flexible GMRES because the inner PCG makes the
preconditioner vary between applications (the paper uses GMRES, Sec. 2.3).

interface="md_rom" takes the other sub-preconditioner of Sec. 3.2.3 (Eq. 47):
F_ring^{-1} ~ M_D^{-ROM}, one application of the Dirichlet preconditioner whose
interior solves K_ii^{-1} are ROM approximations, instead of the PCG on Eq. 48.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .discretization import Lattice
from .feti_dp import CellBlocks, pcg, saddle_operator, saddle_rhs
from .rom import ROM


class InexactFETIDP:
    def __init__(self, lat: Lattice, rom: ROM = None, blocks=None, n_rb=None, interface: str = "pcg"):
        if interface not in ("pcg", "md_rom"):
            raise ValueError(interface)
        self.interface = interface
        self.lat = lat
        self.blocks = blocks or [CellBlocks(lat, s) for s in range(lat.N)]
        self.rom = rom or ROM(lat, n_rb=n_rb, blocks=self.blocks)
        self.A = saddle_operator(lat, self.blocks)
        ref = lat.ref
        self.N, self.nr, self.nd, self.ni, self.npp = lat.N, ref.n_r, ref.n_d, ref.n_i, ref.n_p
        self.nR = self.N * self.nr
        self.inner_its = []
        self.inner_records = []

    # -- splitting of stacked vectors
    def split(self, x):
        nR, nP = self.nR, self.lat.n_P
        return x[:nR].reshape(self.N, self.nr), x[nR:nR + nP], x[nR + nP:]

    # -- operators of Secs. 3.2.3-3.2.4
    def gather(self, lam):           # B_d^(s)T lambda for all cells, (N, n_d)
        return (self.lat.Bd.T @ lam).reshape(self.N, self.nd)

    def scatter(self, y):            # sum_s B_d^(s) y^(s), (L,)
        return self.lat.Bd @ y.ravel()

    def assemble_P(self, c):         # sum_s A_p c^(s), (n_P,)
        return self.lat.Ap @ c.ravel()

    def extract_P(self, zP):         # A_p^(s)T z_P, (N, n_p)
        return (self.lat.Ap.T @ zP).reshape(self.N, self.npp)

    def apply_F(self, lam):
        """Eq. 48: F_ring lambda."""
        rom = self.rom
        g = self.gather(lam)
        y = rom.Fdd_ring(g)
        # coarse correction B_R U_RP S_PP^{-1} U_RP^T B_R^T lambda  (T_rd g = (0, g))
        vr = np.zeros((self.N, self.nr)); vr[:, self.ni:] = g
        zP = rom.coarse_solve(self.assemble_P(rom.Urp_ring_T(vr)))
        y = y + rom.Urp_ring(self.extract_P(zP))[:, self.ni:]
        return self.scatter(y)

    def apply_MD(self, r):
        """Eq. 49: M_D_ring^{-1} r with the Eq. 30 scaling D = (B B^T)^{-1}."""
        g = self.gather(self.lat.apply_D(r))
        return self.lat.apply_D(self.scatter(self.rom.Sdd_ring(g)))

    def apply_MD_rom(self, r):
        """Eq. 47: M_D^{-ROM} r, the Dirichlet preconditioner of Eq. 30 with ROM interior solves."""
        g = self.gather(self.lat.apply_D(r))
        return self.lat.apply_D(self.scatter(self.rom.Sdd_rom(g)))

    def U_apply(self, vR, vP):
        """Algorithm 3: U_ring v.  Returns (z, z_P)."""
        rom = self.rom
        vbarP = vP - self.assemble_P(rom.Urp_ring_T(vR))
        zP = rom.coarse_solve(vbarP)
        t = rom.Urd_ring_T(vR) - rom.Urp_ring(self.extract_P(zP))[:, self.ni:]
        return self.scatter(t), zP

    def UT_apply(self, y):
        """Transpose of Algorithm 3: U_ring^T y = (U_RD B_R^T y - U_RP z_P, z_P)."""
        rom = self.rom
        g = self.gather(y)
        vr = np.zeros((self.N, self.nr)); vr[:, self.ni:] = g
        zP = rom.coarse_solve(-self.assemble_P(rom.Urp_ring_T(vr)))
        xR = rom.Urd_ring(g) - rom.Urp_ring(self.extract_P(zP))
        return xR, zP

    def K_rom_inv(self, vR, vP, zP=None):
        """Algorithm 2 / Eq. 45: (x_R, x_P); x_P = S_PP^{-1}(v_P - U_RP^T v_R)."""
        rom = self.rom
        if zP is None:
            zP = rom.coarse_solve(vP - self.assemble_P(rom.Urp_ring_T(vR)))
        xR = rom.local_rom_solve(vR) - rom.Urp_ring(self.extract_P(zP))
        return xR, zP

    def precondition(self, x, tol_inner, max_inner):
        """Algorithm 1."""
        vR, vP, w = self.split(x)
        Uv, zP = self.U_apply(vR, vP)
        wbar = w - Uv
        rec = []
        if self.interface == "md_rom":
            ysol, its = self.apply_MD_rom(wbar), 0
        else:
            ysol, its = pcg(self.apply_F, self.apply_MD, wbar, tol_inner, max_inner, record=rec)
        y = -ysol
        self.inner_its.append(its)
        self.inner_records.append(rec)
        xR, xP = self.K_rom_inv(vR, vP, zP=zP)     # Algorithm 2 shares v_bar_P, x_P with Algorithm 3
        tR, tP = self.UT_apply(y)
        return np.concatenate([(xR - tR).ravel(), xP - tP, y])

    def solve(self, rhs=0, tol=1e-8, max_outer=100, tol_inner=1e-11, max_inner=1000):
        b = saddle_rhs(self.lat, self.blocks, rhs)
        self.inner_its, self.inner_records = [], []
        x, hist = fgmres(self.A, lambda v: self.precondition(v, tol_inner, max_inner),
                         b, tol, max_outer)
        uR, uP, lam = self.split(x)
        self.outer_its = len(hist)
        self.history = hist
        true_res = np.linalg.norm(b - self.A(x)) / np.linalg.norm(b)
        return uR.ravel(), uP, lam, true_res


def fgmres(apply_A, apply_P, b, tol, max_it):
    """Right-preconditioned flexible GMRES, x_0 = 0, CGS2 Arnoldi, Givens rotations.

    Stops when the least-squares residual estimate |g_{j+1}| / ||b|| <= tol.
    Returns (x, history of relative residual estimates).
    """
    beta = np.linalg.norm(b)
    if beta == 0.0:
        return np.zeros_like(b), []
    V = [b / beta]
    Zs = []
    H = np.zeros((max_it + 1, max_it))
    cs, sn = np.zeros(max_it), np.zeros(max_it)
    g = np.zeros(max_it + 1); g[0] = beta
    hist = []
    j = 0
    for j in range(max_it):
        z = apply_P(V[j])
        Zs.append(z)
        w = apply_A(z)
        Vm = np.stack(V, axis=1)
        h1 = Vm.T @ w
        w = w - Vm @ h1
        h2 = Vm.T @ w
        w = w - Vm @ h2
        H[:j + 1, j] = h1 + h2
        hn = np.linalg.norm(w)
        H[j + 1, j] = hn
        for i in range(j):
            a_, b_ = H[i, j], H[i + 1, j]
            H[i, j] = cs[i] * a_ + sn[i] * b_
            H[i + 1, j] = -sn[i] * a_ + cs[i] * b_
        rho = np.hypot(H[j, j], H[j + 1, j])
        cs[j], sn[j] = H[j, j] / rho, H[j + 1, j] / rho
        H[j, j], H[j + 1, j] = rho, 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        hist.append(abs(g[j + 1]) / beta)
        if hist[-1] <= tol or hn == 0.0:
            break
        V.append(w / hn)
    k = j + 1
    y = sla.solve_triangular(H[:k, :k], g[:k])
    x = sum(y[i] * Zs[i] for i in range(k))
    return x, hist
