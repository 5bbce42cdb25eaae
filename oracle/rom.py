"""Reduced-order model of the local FETI-DP operators (oracle; TEST INFRASTRUCTURE ONLY).

* Snapshots: C_hat^(s) at every Gauss point (Sec. 4.2.2 allows the functions
  C_hat(xi) as snapshots; K^(s) is linear in them, Eq. 52).
* Algorithm 4: greedy selection of principal cells (truncated Gram-Schmidt),
  affine coefficients alpha by the change of basis of Eqs. 55-56.
* Principal operators (Sec. 3.1.1, Eq. 39): U_rp, S_pp, U_rd, F_dd and
  S_dd = F_dd^{-1}, from exact factorisations of the principal K_rr.
* Projections pi, delta (Eqs. 40-42) with each cell's exact K_rr^(s).
* ROM local operators (Eq. 43) and the assembled coarse S_PP (Sec. 3.2.1).
* The ROM-based Dirichlet solve of Eq. 47: K_ii^(s)^{-1} approximated like the K_rr solves of
  Eq. 46, from the principal cells' K_ii^{-1}.

Readings: ties in the greedy argmax go to the lowest cell index among cells
within relative 1e-12 of the maximum; the greedy stops at the requested
N_rb, when max ||Delta||_inf <= tol_rb, or when Delta vanishes.  The
N_rb x N_rb Gram systems (Eqs. 41, 46b) are solved by diagonal-pivoted
Cholesky that drops pivots below 1e-12 of the largest initial diagonal.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .discretization import Lattice

TIE_REL = 1e-12
DROP_REL = 1e-12


def greedy(A: np.ndarray, n_rb: int, tol_rb: float):
    """Algorithm 4 on the snapshot matrix A (N x n_snap).

    Returns (sigma, Z, beta, norms): principal indices, orthonormal basis
    (n_snap x N_rb), coordinates beta (N x N_rb), ||A^(s)||_2.
    """
    norms = np.linalg.norm(A, axis=1)
    Delta = A / norms[:, None]
    sigma, zetas, betas = [], [], []
    for i in range(n_rb):
        inf = np.abs(Delta).max(axis=1)
        m = inf.max()
        if m == 0.0:
            break
        cand = np.nonzero(inf >= m * (1.0 - TIE_REL))[0]
        s_i = int(cand.min())
        zeta = Delta[s_i] / np.linalg.norm(Delta[s_i])
        beta = Delta @ zeta
        Delta = Delta - beta[:, None] * zeta[None, :]
        sigma.append(s_i); zetas.append(zeta); betas.append(beta)
        if np.abs(Delta).max() <= tol_rb:
            break
    Z = np.stack(zetas, axis=1)
    beta = np.stack(betas, axis=1)
    return np.array(sigma), Z, beta, norms


def affine_coefficients(A, sigma, Z, beta, norms):
    """Eq. 56: A_ring^(s) = ||A^(s)|| Z beta^(s) = [A^(sigma_1) ...] alpha^(s).

    Projected on Z: (Z^T [A^(sigma_k)]) alpha = ||A^(s)|| beta^(s); the N_rb x N_rb
    matrix is upper triangular by the greedy construction.
    """
    T = Z.T @ A[sigma].T
    rhs = (norms[:, None] * beta).T
    return np.linalg.solve(T, rhs).T                      # (N, N_rb)


def pivoted_cholesky_pivots(G: np.ndarray, rel_drop: float = DROP_REL):
    """Pivot order of diagonal-pivoted Cholesky; stops on Schur diagonal <= rel_drop * max diag(G)."""
    S = np.array(G, dtype=float, copy=True)
    n = S.shape[0]
    d0 = np.max(np.diag(G)) if n else 0.0
    remaining = list(range(n))
    piv = []
    while remaining:
        j = max(remaining, key=lambda i: (S[i, i], -i))
        if not S[j, j] > rel_drop * d0:
            break
        piv.append(j)
        remaining.remove(j)
        col = S[:, j] / np.sqrt(S[j, j])
        S = S - np.outer(col, col)
    return piv


def gram_solve(G: np.ndarray, h: np.ndarray, rel_drop: float = DROP_REL) -> np.ndarray:
    """Solve G c = h on the pivots kept by pivoted Cholesky; dropped coefficients are 0."""
    piv = pivoted_cholesky_pivots(G, rel_drop)
    c = np.zeros(G.shape[0])
    if piv:
        Gs = G[np.ix_(piv, piv)]
        c[piv] = sla.cho_solve(sla.cho_factor(Gs, lower=True), h[piv])
    return c


class ROM:
    """ROM ingredients for one lattice (Secs. 3.1 and 4.2)."""

    def __init__(self, lat: Lattice, n_rb=None, tol_rb=None, blocks=None):
        self.lat = lat
        ref = lat.ref
        N, ni, nd, nr, npp = lat.N, ref.n_i, ref.n_d, ref.n_r, ref.n_p
        n_rb = lat.prob.n_rb if n_rb is None else n_rb
        tol_rb = lat.prob.tol_rb if tol_rb is None else tol_rb
        # -- snapshots and Algorithm 4
        self.snapshots = np.stack([lat.snapshot(s) for s in range(N)])
        self.sigma, self.Z, self.beta, self.norms = greedy(self.snapshots, n_rb, tol_rb)
        self.n_rb = len(self.sigma)
        self.alpha = affine_coefficients(self.snapshots, self.sigma, self.Z, self.beta, self.norms)
        # -- exact local blocks of every cell (for the projections of Eq. 42 and for K_s)
        if blocks is None:
            Ks = [lat.stiffness_idp(s) for s in range(N)]
        else:
            Ks = [b.K for b in blocks]
        self.K = Ks
        self.Krr = [K[:nr, :nr].tocsr() for K in Ks]
        self.Krp = [K[:nr, nr:].toarray() for K in Ks]
        # -- principal operators (Eq. 39)
        T_rd = np.zeros((nr, nd)); T_rd[ni:, :] = np.eye(nd)
        self.Kp = []          # full principal K (dense, idp order)
        self.Krr_inv, self.Urp, self.Spp, self.Urd, self.Fdd, self.Sdd = [], [], [], [], [], []
        self.Kii_inv = []     # principal K_ii^{-1} (Eq. 47's ROM Dirichlet solves)
        for s in self.sigma:
            K = Ks[s].toarray()
            self.Kp.append(K)
            Krr, Krp, Kpp = K[:nr, :nr], K[:nr, nr:], K[nr:, nr:]
            c = sla.cho_factor(Krr, lower=True)
            Urp = sla.cho_solve(c, Krp)
            Urd = sla.cho_solve(c, T_rd)
            Fdd = Urd[ni:, :]
            self.Krr_inv.append(sla.cho_solve(c, np.eye(nr)))
            self.Urp.append(Urp)
            self.Spp.append(Kpp - Krp.T @ Urp)
            self.Urd.append(Urd)
            self.Fdd.append(Fdd)
            self.Sdd.append(np.linalg.inv(Fdd))            # S_dd = F_dd^{-1} (Sec. 3.1.1)
            self.Kii_inv.append(sla.cho_solve(sla.cho_factor(Krr[:ni, :ni], lower=True), np.eye(ni)))
        # -- projections pi, delta (Eqs. 41-42)
        k = self.n_rb
        self.pi = np.zeros((N, k))
        self.delta = np.zeros((N, k))
        dvec = np.array([np.trace(F) for F in self.Fdd])   # d[i] = tr(U_rd^T T_rd) = tr F_dd
        for s in range(N):
            KUp = [self.Krr[s] @ U for U in self.Urp]
            KUd = [self.Krr[s] @ U for U in self.Urd]
            Ap = np.array([[np.sum(self.Urp[i] * KUp[j]) for j in range(k)] for i in range(k)])
            bp = np.array([np.sum(self.Urp[i] * self.Krp[s]) for i in range(k)])
            Md = np.array([[np.sum(self.Urd[i] * KUd[j]) for j in range(k)] for i in range(k)])
            self.pi[s] = gram_solve(Ap, bp)
            self.delta[s] = gram_solve(Md, dvec)
        # -- coarse problem: S_pp_ring (Eq. 43) assembled into S_PP (Sec. 3.2.1)
        self.Spp_ring = []
        for s in range(N):
            Kpp = sum(self.alpha[s, j] * self.Kp[j][nr:, nr:] for j in range(k))
            Krp = sum(self.alpha[s, j] * self.Kp[j][:nr, nr:] for j in range(k))
            Urp = sum(self.pi[s, j] * self.Urp[j] for j in range(k))
            X = Kpp - Krp.T @ Urp
            self.Spp_ring.append(0.5 * (X + X.T))
        Ap = lat.Ap
        self.SPP = (Ap @ sp.block_diag([sp.csr_matrix(X) for X in self.Spp_ring], format="csr") @ Ap.T).tocsc()
        self.SPP_lu = spla.splu(self.SPP)

    # ---- ROM local operators applied in principal form (Eq. 43, Remark 7)
    def Fdd_ring(self, g):          # g: (N, n_d)
        return sum(self.delta[:, k, None] * (g @ self.Fdd[k].T) for k in range(self.n_rb))

    def Sdd_ring(self, g):
        return sum(self.alpha[:, k, None] * (g @ self.Sdd[k].T) for k in range(self.n_rb))

    def Urp_ring_T(self, v):        # v: (N, n_r) -> (N, n_p)
        return sum(self.pi[:, k, None] * (v @ self.Urp[k]) for k in range(self.n_rb))

    def Urp_ring(self, c):          # c: (N, n_p) -> (N, n_r)
        return sum(self.pi[:, k, None] * (c @ self.Urp[k].T) for k in range(self.n_rb))

    def Urd_ring_T(self, v):        # v: (N, n_r) -> (N, n_d)
        return sum(self.delta[:, k, None] * (v @ self.Urd[k]) for k in range(self.n_rb))

    def Urd_ring(self, g):          # g: (N, n_d) -> (N, n_r)
        return sum(self.delta[:, k, None] * (g @ self.Urd[k].T) for k in range(self.n_rb))

    def coarse_solve(self, b):
        return self.SPP_lu.solve(b)

    def local_rom_solve(self, v):
        """Eq. 46: x_r = R (R^T K_rr R)^{-1} R^T v_r, R = [K_rr^(sigma_k)^{-1} v_r]_k, per cell."""
        N = self.lat.N
        x = np.zeros_like(v)
        for s in range(N):
            R = np.stack([Kinv @ v[s] for Kinv in self.Krr_inv], axis=1)
            G = R.T @ (self.Krr[s] @ R)
            c = gram_solve(G, R.T @ v[s])
            x[s] = R @ c
        return x

    # ---- Eq. 47: Dirichlet Schur complements with ROM-approximated interior solves
    def dirichlet_rom_solve(self, s: int, v_i: np.ndarray) -> np.ndarray:
        """x_i ~ K_ii^(s)^{-1} v_i in the span of R = [K_ii^(sigma_k)^{-1} v_i]_k, K_ii^(s)-orthogonally
        (the construction of Eq. 46 applied to the interior block)."""
        ni = self.lat.ref.n_i
        Kii = self.K[s][:ni, :ni]
        R = np.stack([Kinv @ v_i for Kinv in self.Kii_inv], axis=1)
        G = R.T @ (Kii @ R)
        c = gram_solve(G, R.T @ v_i)
        return R @ c

    def Sdd_rom(self, g):
        """S_dd^(s) g = K_dd g - K_di K_ii^{-1} K_id g per cell, K_ii^{-1} by dirichlet_rom_solve."""
        ref = self.lat.ref
        ni, nr = ref.n_i, ref.n_r
        y = np.zeros_like(g)
        for s in range(self.lat.N):
            K = self.K[s]
            Kid = K[:ni, ni:nr]
            x_i = self.dirichlet_rom_solve(s, Kid @ g[s])
            y[s] = K[ni:nr, ni:nr] @ g[s] - K[ni:nr, :ni] @ x_i
        return y
