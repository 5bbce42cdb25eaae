"""Pins of the oracle's macro maps, strut mask and ROM combination rules.

Each test compares the oracle with something other than its own formulas: finite differences of
the map, brute-force point-to-segment distances, and a lattice whose cells are exact scalar
multiples of one another, for which the ROM of Eq. 43 must reproduce every cell's operators
exactly with known coefficients.
"""
import itertools

import numpy as np
import pytest
import scipy.linalg as sla

from paper_2308_11371_gb300 import workloads as W
from oracle import feti_dp, rom
from oracle.discretization import Lattice, macro_map, strut_distance


# ----------------------------------------------------------------------------- macro maps (Eq. 51)
@pytest.mark.parametrize("prob", [
    W.lattice_2d(4, 3, 2, a=0.83),
    W.lattice_3d(3, 2, 2, e=2, map_kind=W.MAP_SHEAR_BEND_3D, map_params=(0.61, 3.0, 0.17, -0.13)),
    W.lattice_3d(4, 3, 2, e=2, map_kind=W.MAP_BEND_TWIST_3D,
                 map_params=(0.9, 4.0, 0.35, 1.5, 1.0)),
], ids=["bend2d", "shear_bend3d", "bend_twist3d"])
def test_macro_map_jacobian_matches_central_difference(prob):
    """J = dx/dxi of every curved map equals a central difference of x(xi) (h = 1e-6)."""
    d = prob.dim
    rng = np.random.default_rng(11)
    xi = rng.uniform(0.0, 1.0, size=(200, d)) * np.array(prob.cells[:d], float)
    _, J = macro_map(prob, xi)
    h = 1e-6
    for b in range(d):
        e = np.zeros(d); e[b] = h
        xp, _ = macro_map(prob, xi + e)
        xm, _ = macro_map(prob, xi - e)
        fd = (xp - xm) / (2.0 * h)
        assert np.abs(J[:, :, b] - fd).max() < 1e-8, b
    # the map really is curved: the Jacobian varies over the sample
    assert np.ptp(J.reshape(len(xi), -1), axis=0).max() > 0.05


def test_macro_map_hand_values():
    """Closed-form points: the 2D bend peaks at mid-span; the twist rotates the section
    centre onto itself and turns a unit offset by tau xi_x / L."""
    p = W.lattice_2d(4, 2, 2, a=0.5)
    x, _ = macro_map(p, np.array([[2.0, 1.0]]))            # sin(pi * 2 / 4) = 1
    assert np.allclose(x, [[2.0, 1.5]])
    tau, L = 0.4, 4.0
    p3 = W.lattice_3d(4, 2, 2, e=2, map_kind=W.MAP_BEND_TWIST_3D,
                      map_params=(0.0, L, tau, 1.0, 1.0))
    xi = np.array([[2.0, 1.0, 1.0], [2.0, 2.0, 1.0]])
    x3, _ = macro_map(p3, xi)
    th = tau * 2.0 / L
    assert np.allclose(x3[0], [2.0, 1.0, 1.0])
    assert np.allclose(x3[1], [2.0, 1.0 + np.cos(th), 1.0 + np.sin(th)])


# ----------------------------------------------------------------------------- strut mask (Eq. 51)
def _seg_dist(p, a, b):
    """Distance from points p (n, d) to the closed segment [a, b]."""
    ab = b - a
    t = np.clip(((p - a) @ ab) / (ab @ ab), 0.0, 1.0)
    q = a + t[:, None] * ab
    return np.linalg.norm(p - q, axis=1)


def _skeleton(dim):
    if dim == 2:
        c = [np.array(v, float) for v in ((0, 0), (1, 0), (1, 1), (0, 1))]
        segs = [(c[k], c[(k + 1) % 4]) for k in range(4)]          # frame
        segs += [(c[0], c[2]), (c[1], c[3])]                        # both diagonals
        return segs
    # BCC: every cube corner joined to the opposite corner
    segs = []
    for v in itertools.product((0.0, 1.0), repeat=3):
        a = np.array(v)
        segs.append((a, 1.0 - a))
    return segs


@pytest.mark.parametrize("prob", [W.lattice_2d(1, 1, 2), W.lattice_3d(1, 1, 1, e=2)],
                         ids=["frame_diag2d", "bcc3d"])
def test_strut_distance_matches_brute_force(prob):
    d = prob.dim
    rng = np.random.default_rng(5)
    eta = rng.uniform(0.0, 1.0, size=(400, d))
    ref = np.min(np.stack([_seg_dist(eta, a, b) for a, b in _skeleton(d)]), axis=0)
    assert np.abs(strut_distance(prob, eta) - ref).max() < 1e-14


def test_strut_distance_hand_values():
    p2 = W.lattice_2d(1, 1, 2)
    eta2 = np.array([[0.3, 0.3], [0.2, 0.8], [0.5, 0.0], [0.5, 0.25]])
    assert np.allclose(strut_distance(p2, eta2), [0.0, 0.0, 0.0, 0.25 / np.sqrt(2.0)])
    p3 = W.lattice_3d(1, 1, 1, e=2)
    eta3 = np.array([[0.5, 0.5, 0.5], [0.25, 0.75, 0.75], [0.8, 0.2, 0.8], [0.5, 0.5, 0.0]])
    # centre and points on three different diagonals; the face centre is sqrt(2)/2 * sin(acos(1/sqrt3))
    # from each diagonal: |w|^2 - (w.u)^2 with w = (0.5, 0.5, 0), u = (1,1,1)/sqrt3 -> 0.5 - 1/3
    assert np.allclose(strut_distance(p3, eta3), [0.0, 0.0, 0.0, np.sqrt(0.5 - 1.0 / 3.0)])


# ----------------------------------------------------------------------------- Eq. 43 with scaled cells
class _ScaledLattice(Lattice):
    """Cells whose pulled-back tensor is c_s times one common tensor: K^(s) = c_s K^(0)."""

    def __init__(self, prob, scales):
        self._scales = np.asarray(scales, float)
        super().__init__(prob)

    def chat(self, s, dE_dr=False):
        return self._scales[s] * super().chat(s, dE_dr=dE_dr)


@pytest.fixture(scope="module")
def scaled():
    # identity map and one radius: every cell has the same base tensor
    prob = W.lattice_2d(3, 2, 4, a=0.0, r=0.15, n_rb=3)
    prob.map_kind = W.MAP_IDENTITY
    scales = 1.0 + 0.37 * np.arange(6) + 0.05 * np.arange(6) ** 2
    lat = _ScaledLattice(prob, scales)
    blocks = [feti_dp.CellBlocks(lat, s) for s in range(lat.N)]
    return lat, blocks, rom.ROM(lat, blocks=blocks), scales


def test_scaled_cells_coefficients(scaled):
    """One principal cell spans every snapshot; alpha = c_s / c_sigma, delta = 1 / alpha,
    pi = 1 (U_rp is scale free), by K^(s) = c_s K^(0)."""
    lat, blocks, R, c = scaled
    assert R.n_rb == 1
    sig = R.sigma[0]
    a = c / c[sig]
    assert np.allclose(R.alpha[:, 0], a, rtol=1e-12)
    assert np.allclose(R.delta[:, 0], 1.0 / a, rtol=1e-10)
    assert np.allclose(R.pi[:, 0], 1.0, rtol=1e-10)


def test_scaled_cells_rom_operators_are_exact(scaled):
    """Eq. 43 is exact here: S_dd_ring, F_dd_ring, U_rp_ring, U_rd_ring and the Eq. 46
    local solve equal each cell's exact operators (a combination with the wrong
    coefficient set, e.g. delta for S_dd, is off by c_s^2)."""
    lat, blocks, R, c = scaled
    ref = lat.ref
    ni, nd, nr = ref.n_i, ref.n_d, ref.n_r
    rng = np.random.default_rng(3)
    g = rng.standard_normal((lat.N, nd))
    v = rng.standard_normal((lat.N, nr))
    cp = rng.standard_normal((lat.N, ref.n_p))
    Sdd, Fdd, Urp, Urd, Kinv = [], [], [], [], []
    for s in range(lat.N):
        Krr = blocks[s].Krr.toarray()
        Ki = np.linalg.inv(Krr)
        Kinv.append(Ki)
        Fdd.append(Ki[ni:, ni:])
        Kii, Kid, Kdd = Krr[:ni, :ni], Krr[:ni, ni:], Krr[ni:, ni:]
        Sdd.append(Kdd - Kid.T @ sla.solve(Kii, Kid))
        Urp.append(Ki @ blocks[s].Krp)
        Urd.append(Ki[:, ni:])
    def close(x, y):
        return np.abs(x - y).max() <= 1e-9 * np.abs(y).max()
    assert close(R.Sdd_ring(g), np.stack([Sdd[s] @ g[s] for s in range(lat.N)]))
    assert close(R.Fdd_ring(g), np.stack([Fdd[s] @ g[s] for s in range(lat.N)]))
    assert close(R.Urp_ring(cp), np.stack([Urp[s] @ cp[s] for s in range(lat.N)]))
    assert close(R.Urp_ring_T(v), np.stack([Urp[s].T @ v[s] for s in range(lat.N)]))
    assert close(R.Urd_ring(g), np.stack([Urd[s] @ g[s] for s in range(lat.N)]))
    assert close(R.Urd_ring_T(v), np.stack([Urd[s].T @ v[s] for s in range(lat.N)]))
    assert close(R.local_rom_solve(v), np.stack([Kinv[s] @ v[s] for s in range(lat.N)]))
    # the ROM coarse matrix equals the exact S_PP (Eq. 22)
    ex = feti_dp.StandardFETIDP(lat, blocks=blocks)
    assert np.abs((R.SPP - ex.SPP).toarray()).max() <= 1e-9 * np.abs(ex.SPP.toarray()).max()
