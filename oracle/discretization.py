"""Lattice discretisation (oracle; TEST INFRASTRUCTURE ONLY).

Sec. 2.2.1 (Eqs. 3-7): every cell is the image of one reference cell, so
all cells share one Q1 reference mesh and only the pulled-back material
tensor differs between cells (Eq. 52).  Sec. 2.2.2-2.2.3 (Eqs. 8-15, 18):
corner DOF are primal, the other boundary DOF are dual and carry pointwise
multipliers, Dirichlet data on dual DOF are imposed through multipliers.

Readings of silent points (the same ones the CUDA path takes):
* Q1 elements, 2-point Gauss rule per direction, material evaluated at
  each Gauss point in cell-local coordinates.
* Pulled-back tensor as a symmetric (d^2 x d^2) matrix acting on the
  reference gradient G_ia = du_i/dxi_a (Eq. 52): 10 entries in 2D, 45 in 3D.
* Multipliers are non-redundant: for a non-corner interface node shared by
  cells s_1 < ... < s_m, rows u(s_j) - u(s_{j+1}); every cell copy of a
  clamped node gets its own row u(s) = 0 and no inter-cell rows.
* Clamped corner DOF are removed from the global primal vector.
* Scaling D of the Dirichlet preconditioner (Eq. 30): the one matrix common
  to all cells that meets the condition sum_s B_d^(s) B_d^(s)T D = I_L, i.e.
  D = (B B^T)^{-1}.  B B^T is block diagonal over the rows of one node and
  component: 1 on a Dirichlet row, 2 on the single row of a node shared by two
  cells (so D = 1/2 there: every 2D row), and the tridiagonal (2, -1) matrix
  of the m - 1 chain rows of a node shared by m = 4 cells (3D cell edges),
  whose inverse is not diagonal.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from paper_2308_11371_gb300 import workloads as W

GAUSS_T = (0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0))   # 2-pt Gauss on [0, 1]


# --------------------------------------------------------------------------- maps
def macro_map(prob: W.LatticeProblem, xi: np.ndarray):
    """x = F(xi) and J = dx/dxi for lattice coordinates xi of shape (..., d)."""
    d = prob.dim
    p = prob.map_params_array()
    x = np.array(xi, dtype=float, copy=True)
    J = np.zeros(xi.shape[:-1] + (d, d))
    for k in range(d):
        J[..., k, k] = 1.0
    mk = prob.map_kind
    if mk == W.MAP_IDENTITY:
        pass
    elif mk == W.MAP_BEND_2D:
        a, L = p[0], p[1]
        x[..., 1] = xi[..., 1] + a * np.sin(np.pi * xi[..., 0] / L)
        J[..., 1, 0] = a * np.pi / L * np.cos(np.pi * xi[..., 0] / L)
    elif mk == W.MAP_SHEAR_BEND_3D:
        a, L, g1, g2 = p[0], p[1], p[2], p[3]
        x[..., 0] = xi[..., 0] + g1 * xi[..., 2]
        x[..., 1] = xi[..., 1] + g2 * xi[..., 2]
        x[..., 2] = xi[..., 2] + a * np.sin(np.pi * xi[..., 0] / L)
        J[..., 0, 2] = g1
        J[..., 1, 2] = g2
        J[..., 2, 0] = a * np.pi / L * np.cos(np.pi * xi[..., 0] / L)
    elif mk == W.MAP_BEND_TWIST_3D:
        a, L, tau, yc, zc = p[0], p[1], p[2], p[3], p[4]
        th = tau * xi[..., 0] / L
        c, s = np.cos(th), np.sin(th)
        dy, dz = xi[..., 1] - yc, xi[..., 2] - zc
        x[..., 1] = yc + c * dy - s * dz
        x[..., 2] = zc + s * dy + c * dz + a * np.sin(np.pi * xi[..., 0] / L)
        dth = tau / L
        J[..., 1, 0] = dth * (-s * dy - c * dz)
        J[..., 1, 1] = c
        J[..., 1, 2] = -s
        J[..., 2, 0] = dth * (c * dy - s * dz) + a * np.pi / L * np.cos(np.pi * xi[..., 0] / L)
        J[..., 2, 1] = s
        J[..., 2, 2] = c
    else:
        raise ValueError(f"unknown map kind {mk}")
    return x, J


# --------------------------------------------------------------------------- material
def strut_distance(prob: W.LatticeProblem, eta: np.ndarray) -> np.ndarray:
    """Distance from cell-local points eta (..., d) to the strut skeleton."""
    if prob.mask_kind == W.MASK_FRAME_DIAG:
        ex, ey = eta[..., 0], eta[..., 1]
        edges = np.minimum(np.minimum(ex, 1.0 - ex), np.minimum(ey, 1.0 - ey))
        diag1 = np.abs(ex - ey) / np.sqrt(2.0)
        diag2 = np.abs(ex + ey - 1.0) / np.sqrt(2.0)
        return np.minimum(edges, np.minimum(diag1, diag2))
    # BCC: the four body diagonals of the unit cube
    best = None
    for corner in ((0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)):
        a = np.array(corner, float)
        u = np.array([1.0 if c == 0 else -1.0 for c in corner]) / np.sqrt(3.0)
        w = eta - a
        t = (w * u).sum(-1)
        perp = w - t[..., None] * u
        dist = np.sqrt((perp * perp).sum(-1))
        best = dist if best is None else np.minimum(best, dist)
    return best


def youngs_modulus(prob: W.LatticeProblem, eta: np.ndarray, r: float) -> np.ndarray:
    """Ersatz material: E_solid inside the struts (d <= r), E_void outside."""
    dist = strut_distance(prob, eta)
    if prob.mask_kind == W.MASK_BCC_SIGMOID:
        z = (r - dist) / prob.mask_width
        return prob.E_void + (prob.E_solid - prob.E_void) / (1.0 + np.exp(-z))
    return np.where(dist <= r, prob.E_solid, prob.E_void)


def youngs_modulus_dr(prob: W.LatticeProblem, eta: np.ndarray, r: float) -> np.ndarray:
    """dE/dr of the ersatz material (zero almost everywhere for hard masks)."""
    if prob.mask_kind != W.MASK_BCC_SIGMOID:
        return np.zeros(eta.shape[:-1])
    dist = strut_distance(prob, eta)
    z = (r - dist) / prob.mask_width
    sig = 1.0 / (1.0 + np.exp(-z))
    return (prob.E_solid - prob.E_void) * sig * (1.0 - sig) / prob.mask_width


def isotropic_tensor(d: int, nu: float) -> np.ndarray:
    """C_ikjl for unit Young's modulus (plane strain in 2D uses the 3D Lame constants)."""
    lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = 1.0 / (2.0 * (1.0 + nu))
    I = np.eye(d)
    return (lam * np.einsum("ik,jl->ikjl", I, I)
            + mu * (np.einsum("ij,kl->ikjl", I, I) + np.einsum("il,kj->ikjl", I, I)))


def pulled_back_tensor(J: np.ndarray, E: np.ndarray, nu: float) -> np.ndarray:
    """Eq. 52: C_hat_iajb = E det J sum_kl Jinv_ak C_ikjl Jinv_bl, shape (..., d*d, d*d).

    Acts on the reference gradient G_ia = du_i/dxi_a:
    sigma:eps dx = G : C_hat : G' dxi.
    """
    d = J.shape[-1]
    C = isotropic_tensor(d, nu)
    Jinv = np.linalg.inv(J)
    detJ = np.linalg.det(J)
    Ch = np.einsum("...ak,ikjl,...bl->...iajb", Jinv, C, Jinv)
    Ch = Ch * (E * detJ)[..., None, None, None, None]
    return Ch.reshape(J.shape[:-2] + (d * d, d * d))


# --------------------------------------------------------------------------- reference cell
class ReferenceCell:
    """Q1 mesh of the unit reference cell with e^d elements (shared by all cells, Eq. 6)."""

    def __init__(self, dim: int, e: int):
        self.dim, self.e = dim, e
        self.h = 1.0 / e
        self.nn1 = e + 1
        self.n_nodes = self.nn1 ** dim
        self.n_dof = self.n_nodes * dim
        self.n_elem = e ** dim
        self.n_gp = 2 ** dim
        # node coordinates (index), lexicographic with x fastest
        grids = np.meshgrid(*[np.arange(self.nn1)] * dim, indexing="ij")
        idx = np.stack([g.ravel(order="F") for g in grids], axis=-1)   # x fastest
        self.node_ijk = idx
        self.node_eta = idx * self.h
        # element -> nodes; local element node A = ax + 2 ay + 4 az
        self.elem_ijk = np.stack([g.ravel(order="F") for g in
                                  np.meshgrid(*[np.arange(e)] * dim, indexing="ij")], axis=-1)
        offs = np.array(list(itertools.product([0, 1], repeat=dim)))[:, ::-1]  # x fastest
        self.elem_corner_offsets = offs
        strides = self.nn1 ** np.arange(dim)
        self.elem_nodes = ((self.elem_ijk[:, None, :] + offs[None, :, :]) * strides).sum(-1)
        # Gauss points in element coordinates t, g = gx + 2 gy + 4 gz
        self.gauss_t = np.array([[GAUSS_T[(g >> k) & 1] for k in range(dim)]
                                 for g in range(self.n_gp)])
        self.gauss_w = np.full(self.n_gp, 0.5 ** dim)
        # shape functions and t-gradients at Gauss points: N[g, A], dN[g, A, a]
        nA = len(offs)
        self.N = np.ones((self.n_gp, nA))
        self.dNdt = np.ones((self.n_gp, nA, dim))
        for g in range(self.n_gp):
            t = self.gauss_t[g]
            for A in range(nA):
                vals = [t[k] if offs[A, k] else 1.0 - t[k] for k in range(dim)]
                ders = [1.0 if offs[A, k] else -1.0 for k in range(dim)]
                self.N[g, A] = np.prod(vals)
                for a in range(dim):
                    self.dNdt[g, A, a] = np.prod([ders[k] if k == a else vals[k] for k in range(dim)])
        # DOF classes: corner (p), other boundary (d), interior (i) -- Eq. 12
        on_bnd = ((idx == 0) | (idx == e))
        n_bnd_axes = on_bnd.sum(1)
        self.node_class = np.where(n_bnd_axes == dim, 2, np.where(n_bnd_axes > 0, 1, 0))
        def dofs(cls):
            nodes = np.nonzero(self.node_class == cls)[0]
            return (nodes[:, None] * dim + np.arange(dim)[None, :]).ravel()
        self.dof_i, self.dof_d, self.dof_p = dofs(0), dofs(1), dofs(2)
        self.n_i, self.n_d, self.n_p = len(self.dof_i), len(self.dof_d), len(self.dof_p)
        self.n_r = self.n_i + self.n_d
        # permutation: local (i, d, p) ordering -> natural node*dim + comp ordering
        self.perm = np.concatenate([self.dof_i, self.dof_d, self.dof_p])
        self.dual_nodes = np.nonzero(self.node_class == 1)[0]
        self.corner_nodes = np.nonzero(self.node_class == 2)[0]

    def gauss_eta(self) -> np.ndarray:
        """Cell-local coordinates of all Gauss points, shape (n_elem, n_gp, d)."""
        return (self.elem_ijk[:, None, :] + self.gauss_t[None, :, :]) * self.h


def upper_pairs(d: int):
    """(I, J) index pairs I <= J of the symmetric (d^2 x d^2) tensor, row-major."""
    n = d * d
    return [(I, J) for I in range(n) for J in range(I, n)]


# --------------------------------------------------------------------------- lattice
class Lattice:
    """All discrete data of one lattice problem (Secs. 2.1-2.2)."""

    def __init__(self, prob: W.LatticeProblem):
        self.prob = prob
        self.dim = d = prob.dim
        self.nc = np.array(prob.cells[:d])
        self.N = int(np.prod(self.nc))
        self.ref = ref = ReferenceCell(d, prob.elems)
        self.e = prob.elems
        self.cell_ijk = np.stack([g.ravel(order="F") for g in
                                  np.meshgrid(*[np.arange(n) for n in self.nc], indexing="ij")], -1)
        self._build_maps()

    # ---- geometry / material at Gauss points
    def cell_gauss_data(self, s: int):
        """xi, J, E at all Gauss points of cell s: shapes (ne, ng, d), (ne, ng, d, d), (ne, ng)."""
        eta = self.ref.gauss_eta()
        xi = self.cell_ijk[s][None, None, :] + eta
        _, J = macro_map(self.prob, xi)
        E = youngs_modulus(self.prob, eta, self.prob.r_cell[s])
        return xi, J, E

    def chat(self, s: int, dE_dr: bool = False) -> np.ndarray:
        """C_hat at all Gauss points of cell s, shape (ne, ng, d*d, d*d) (Eq. 52)."""
        eta = self.ref.gauss_eta()
        xi = self.cell_ijk[s][None, None, :] + eta
        _, J = macro_map(self.prob, xi)
        r = self.prob.r_cell[s]
        E = youngs_modulus_dr(self.prob, eta, r) if dE_dr else youngs_modulus(self.prob, eta, r)
        return pulled_back_tensor(J, E, self.prob.nu)

    def snapshot(self, s: int) -> np.ndarray:
        """Snapshot vector of cell s: upper triangle of C_hat at every Gauss point,
        ordered (element, Gauss point, pair) -- the 'functions C_hat(xi)' option of Sec. 4.2.2."""
        Ch = self.chat(s)
        pairs = upper_pairs(self.dim)
        I = np.array([p[0] for p in pairs]); Jx = np.array([p[1] for p in pairs])
        return Ch[:, :, I, Jx].ravel()

    # ---- local operators
    def stiffness_from_chat(self, Ch: np.ndarray) -> sp.csr_matrix:
        """K = sum_e sum_g w_g h^d dN_a C_hat_(ia)(jb) dN_b (Eq. 52), natural DOF ordering."""
        ref, d = self.ref, self.dim
        dNdxi = ref.dNdt / ref.h                            # (ng, nA, d)
        w = ref.gauss_w * ref.h ** d                        # (ng,)
        Ch4 = Ch.reshape(Ch.shape[:2] + (d, d, d, d))       # (ne, ng, i, a, j, b)
        Ke = np.einsum("g,gAa,egiajb,gBb->eAiBj", w, dNdxi, Ch4, dNdxi)
        nA = ref.elem_nodes.shape[1]
        dof = (ref.elem_nodes[:, :, None] * d + np.arange(d)[None, None, :]).reshape(-1, nA * d)
        rows = np.repeat(dof, nA * d, axis=1).ravel()
        cols = np.tile(dof, (1, nA * d)).ravel()
        K = sp.coo_matrix((Ke.reshape(len(dof), -1).ravel(), (rows, cols)),
                          shape=(ref.n_dof, ref.n_dof)).tocsr()
        K.sum_duplicates()
        return K

    def stiffness(self, s: int, dE_dr: bool = False) -> sp.csr_matrix:
        """Local stiffness K^(s) (natural ordering); with dE_dr, dK^(s)/dr_s."""
        return self.stiffness_from_chat(self.chat(s, dE_dr=dE_dr))

    def stiffness_idp(self, s: int) -> sp.csr_matrix:
        """K^(s) in the local (i, d, p) ordering of Eq. 12."""
        K = self.stiffness(s)
        P = self.ref.perm
        return K[P][:, P].tocsr()

    def load(self, s: int) -> np.ndarray:
        """Load vectors f^(s) of Eq. 5b for every load case, shape (n_rhs, n_dof), natural order."""
        ref, d, prob = self.ref, self.dim, self.prob
        f = np.zeros((prob.n_rhs, ref.n_dof))
        for li, ld in enumerate(prob.loads):
            direction = np.asarray(ld.direction, float)
            if ld.kind == W.LOAD_BODY:
                eta = ref.gauss_eta()
                xi = self.cell_ijk[s] + eta
                _, J = macro_map(prob, xi)
                detJ = np.linalg.det(J)                              # (ne, ng)
                wgt = ref.gauss_w * ref.h ** d                       # (ng,)
                contrib = np.einsum("g,eg,gA->eA", wgt, detJ, ref.N)  # (ne, nA)
                for k in range(d):
                    np.add.at(f[li], ref.elem_nodes * d + k, contrib * direction[k])
            else:
                ax, side = ld.axis, ld.side
                if self.cell_ijk[s][ax] != (self.nc[ax] - 1 if side == 1 else 0):
                    continue
                fix = ref.e if side == 1 else 0
                tang = [k for k in range(d) if k != ax]
                # face elements: elements touching the face, face Gauss points
                for el in range(ref.n_elem):
                    eij = ref.elem_ijk[el]
                    if eij[ax] != (ref.e - 1 if side == 1 else 0):
                        continue
                    for fg in range(2 ** (d - 1)):
                        t = np.zeros(d)
                        t[ax] = 1.0 if side == 1 else 0.0
                        for q, k in enumerate(tang):
                            t[k] = GAUSS_T[(fg >> q) & 1]
                        xi = self.cell_ijk[s] + (eij + t) * ref.h
                        _, J = macro_map(prob, xi[None, :])
                        J = J[0]
                        if d == 2:
                            meas = np.linalg.norm(J[:, tang[0]])
                        else:
                            meas = np.linalg.norm(np.cross(J[:, tang[0]], J[:, tang[1]]))
                        wq = (0.5 * ref.h) ** (d - 1) * meas
                        offs = ref.elem_corner_offsets
                        for A in range(len(offs)):
                            if offs[A, ax] != (1 if side == 1 else 0):
                                continue
                            NA = np.prod([t[k] if offs[A, k] else 1.0 - t[k] for k in range(d)])
                            node = ref.elem_nodes[el, A]
                            f[li, node * d:(node + 1) * d] += wq * NA * direction
                _ = fix
        return f

    # ---- global maps
    def _build_maps(self):
        ref, d, e, nc = self.ref, self.dim, self.e, self.nc
        prob = self.prob
        gdims = nc * e + 1
        self.global_node_dims = gdims
        gstr = np.cumprod(np.concatenate([[1], gdims[:-1]]))
        self.global_node_strides = gstr
        # local node -> global node for every cell
        self.cell_global_nodes = ((self.cell_ijk[:, None, :] * e + ref.node_ijk[None, :, :])
                                  * gstr).sum(-1)
        self.n_global_nodes = int(np.prod(gdims))
        # clamped nodes
        ca, cs = prob.clamp_axis, prob.clamp_side
        clamp_coord = 0 if cs == 0 else nc[ca] * e
        # --- multipliers (Eqs. 14-15), non-redundant chains, row order: global node, pair, comp
        dual_local_index = -np.ones(ref.n_nodes, dtype=int)
        dual_local_index[ref.dual_nodes] = np.arange(len(ref.dual_nodes))
        owners = {}
        for s in range(self.N):
            for ln in ref.dual_nodes:
                owners.setdefault(int(self.cell_global_nodes[s, ln]), []).append((s, int(ln)))
        rows = []          # list of [(cell, local dual dof index, sign)]
        row_block = []     # (global node, component) of each row: the blocks of B B^T
        row_dirichlet = []
        for gn in sorted(owners):
            lst = sorted(owners[gn])
            gijk = np.array([(gn // gstr[k]) % gdims[k] for k in range(d)])
            clamped = gijk[ca] == clamp_coord
            m = len(lst)
            if clamped:
                for (s, ln) in lst:
                    for c in range(d):
                        rows.append([(s, dual_local_index[ln] * d + c, 1.0)])
                        row_block.append((gn, s, c)); row_dirichlet.append(True)
            else:
                for j in range(m - 1):
                    (s1, l1), (s2, l2) = lst[j], lst[j + 1]
                    for c in range(d):
                        rows.append([(s1, dual_local_index[l1] * d + c, 1.0),
                                     (s2, dual_local_index[l2] * d + c, -1.0)])
                        row_block.append((gn, -1, c)); row_dirichlet.append(False)
        self.rows = rows
        self.L = len(rows)
        self.row_dirichlet = np.array(row_dirichlet, bool)
        # B_d^(s) as one sparse (L x N*n_d) matrix over the concatenated dual vectors
        ri, ci, vi = [], [], []
        for l, row in enumerate(rows):
            for (s, j, sg) in row:
                ri.append(l); ci.append(s * ref.n_d + j); vi.append(sg)
        self.Bd = sp.csr_matrix((vi, (ri, ci)), shape=(self.L, self.N * ref.n_d))
        # D = (sum_s B_d^(s) B_d^(s)T)^{-1} (Eq. 30), inverted block by block
        BBt = (self.Bd @ self.Bd.T).tocsr()
        blocks = {}
        for l, key in enumerate(row_block):
            blocks.setdefault(key, []).append(l)
        ri, ci, vi = [], [], []
        for idx in blocks.values():
            inv = np.linalg.inv(BBt[idx][:, idx].toarray())
            for a, la in enumerate(idx):
                for b, lb in enumerate(idx):
                    ri.append(la); ci.append(lb); vi.append(inv[a, b])
        self.Dmat = sp.csr_matrix((vi, (ri, ci)), shape=(self.L, self.L))
        # --- primal DOF (Eq. 18): free lattice vertices, lexicographic, x fastest
        vdims = nc + 1
        vstr = np.cumprod(np.concatenate([[1], vdims[:-1]]))
        n_vert = int(np.prod(vdims))
        vijk = np.stack([(np.arange(n_vert) // vstr[k]) % vdims[k] for k in range(d)], -1)
        free = vijk[:, ca] != (0 if cs == 0 else nc[ca])
        vnum = -np.ones(n_vert, dtype=int)
        vnum[free] = np.arange(free.sum())
        self.n_P = int(free.sum()) * d
        corner_offs = ref.node_ijk[ref.corner_nodes] // e                  # (2^d, d)
        cell_vertex = ((self.cell_ijk[:, None, :] + corner_offs[None]) * vstr).sum(-1)
        self.cell_corner_vertex = vnum[cell_vertex]                         # (N, 2^d), -1 clamped
        ri, ci = [], []
        for s in range(self.N):
            for k in range(len(ref.corner_nodes)):
                v = self.cell_corner_vertex[s, k]
                if v < 0:
                    continue
                for c in range(d):
                    ri.append(v * d + c); ci.append(s * ref.n_p + k * d + c)
        # A_p as one (n_P x N*n_p) Boolean matrix over the concatenated corner vectors
        self.Ap = sp.csr_matrix((np.ones(len(ri)), (ri, ci)), shape=(self.n_P, self.N * ref.n_p))

    def apply_D(self, r: np.ndarray) -> np.ndarray:
        """D r with the Eq. 30 scaling D = (B B^T)^{-1}; r of shape (L,) or (L, k)."""
        return self.Dmat @ r

    # ---- convenience
    def loads_idp(self, s: int) -> np.ndarray:
        return self.load(s)[:, self.ref.perm]
