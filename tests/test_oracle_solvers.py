"""Pins of the oracle's FETI-DP, ROM and inexact FETI-DP against the monolithic direct
solve, algebraic identities and the paper's exactness statements."""
import numpy as np
import pytest
import scipy.linalg as sla

from paper_2308_11371_gb300 import workloads as W
from oracle import adjoint, feti_dp, ifeti_dp, monolithic, rom
from oracle.discretization import Lattice


def _mono_cells(lat):
    return monolithic.to_cells(lat, monolithic.solve(lat))


@pytest.fixture(scope="module")
def frame4x4():
    lat = Lattice(W.frame_2d_4x4())
    return lat, feti_dp.StandardFETIDP(lat)


@pytest.mark.parametrize("prob", [W.frame_2d_4x4(),
                                  W.lattice_3d(2, 2, 2, e=3, r=0.2, r_spread=0.05, seed=3,
                                               map_kind=W.MAP_SHEAR_BEND_3D,
                                               map_params=(0.2, 2.0, 0.1, -0.1))])
def test_standard_fetidp_equals_monolithic(prob):
    lat = Lattice(prob)
    fd = feti_dp.StandardFETIDP(lat)
    uR, uP, lam, its = fd.solve(tol=1e-13)
    u = feti_dp.cell_vectors(lat, uR, uP)
    ref = _mono_cells(lat)[0]
    assert np.abs(u - ref).max() <= 1e-11 * np.abs(ref).max()


def test_interface_operator_spd(frame4x4):
    """F = B K^{-1} B^T (Eq. 26) is symmetric positive definite (B full rank, K SPD)."""
    lat, fd = frame4x4
    F = np.stack([fd.apply_F(e) for e in np.eye(lat.L)], axis=1)
    assert np.abs(F - F.T).max() < 1e-12 * np.abs(F).max()
    assert np.linalg.eigvalsh(0.5 * (F + F.T)).min() > 0.0


def test_saddle_point_residual_of_fetidp_solution(frame4x4):
    lat, fd = frame4x4
    uR, uP, lam, _ = fd.solve(tol=1e-13)
    A = feti_dp.saddle_operator(lat, fd.blocks)
    b = feti_dp.saddle_rhs(lat, fd.blocks, 0)
    x = np.concatenate([uR, uP, lam])
    assert np.linalg.norm(A(x) - b) < 1e-10 * np.linalg.norm(b)


def test_dirichlet_schur_is_inverse_neumann_schur(frame4x4):
    """S_dd = F_dd^{-1} (Sec. 3.1.1): Dirichlet Schur from K_ii^{-1}, F_dd from K_rr^{-1}."""
    lat, fd = frame4x4
    R = rom.ROM(lat, blocks=fd.blocks)
    for k, s in enumerate(R.sigma):
        assert np.allclose(fd.Sdd[s] @ R.Fdd[k], np.eye(lat.ref.n_d), atol=1e-9)


def test_greedy_on_hand_made_snapshots():
    """Algorithm 4 by hand: three snapshots, two directions."""
    A = np.array([[3.0, 0.0, 0.0],
                  [0.0, 2.0, 0.0],
                  [1.0, 1.0, 0.0],
                  [6.0, 0.0, 0.0]])
    sigma, Z, beta, norms = rom.greedy(A, 5, 1e-12)
    # Delta_0 rows: e1, e2, (1,1)/sqrt2, e1 -> inf norms 1,1,0.707,1 -> tie -> lowest index 0
    assert list(sigma) == [0, 1]
    assert np.allclose(Z, [[1, 0], [0, 1], [0, 0]])
    alpha = rom.affine_coefficients(A, sigma, Z, beta, norms)
    assert np.allclose(alpha, [[1, 0], [0, 1], [1 / 3, 0.5], [2, 0]])


@pytest.fixture(scope="module")
def frame4x4_rom():
    lat = Lattice(W.frame_2d_4x4())
    blocks = [feti_dp.CellBlocks(lat, s) for s in range(lat.N)]
    return lat, blocks, rom.ROM(lat, blocks=blocks)


def test_greedy_interpolation_and_orthonormality(frame4x4_rom):
    """Eq. 55 (interpolation at principal cells) and Z^T Z = I."""
    lat, _, R = frame4x4_rom
    assert np.allclose(R.Z.T @ R.Z, np.eye(R.n_rb), atol=1e-13)
    for k, s in enumerate(R.sigma):
        ring = R.norms[s] * R.Z @ R.beta[s]
        assert np.allclose(ring, R.snapshots[s], rtol=0, atol=1e-12 * np.abs(R.snapshots[s]).max())
        assert np.allclose(R.alpha[s], np.eye(R.n_rb)[k], atol=1e-12)


def test_projection_coefficients_on_principal_cells(frame4x4_rom):
    """Eqs. 41-42 on a principal cell reproduce its own operators: pi = delta = e_k."""
    lat, _, R = frame4x4_rom
    for k, s in enumerate(R.sigma):
        assert np.allclose(R.pi[s], np.eye(R.n_rb)[k], atol=1e-9)
        assert np.allclose(R.delta[s], np.eye(R.n_rb)[k], atol=1e-9)


def test_rom_local_solve_exact_on_principal_cells(frame4x4_rom):
    """Eq. 46b: K_rr^(s)^{-1} v lies in span(R) when s is principal, so the ROM solve is exact."""
    lat, blocks, R = frame4x4_rom
    rng = np.random.default_rng(2)
    v = rng.standard_normal((lat.N, lat.ref.n_r))
    x = R.local_rom_solve(v)
    for s in R.sigma:
        exact = sla.solve(blocks[s].Krr.toarray(), v[s], assume_a="pos")
        assert np.allclose(x[s], exact, rtol=1e-8, atol=1e-10 * np.abs(exact).max())


def test_rom_local_solve_is_energy_projection(frame4x4_rom):
    """Eq. 46b for a non-principal cell: the error is K_rr-orthogonal to span(R)."""
    lat, blocks, R = frame4x4_rom
    s = [c for c in range(lat.N) if c not in set(R.sigma)][0]
    rng = np.random.default_rng(3)
    v = rng.standard_normal((lat.N, lat.ref.n_r))
    x = R.local_rom_solve(v)[s]
    Krr = blocks[s].Krr.toarray()
    exact = sla.solve(Krr, v[s], assume_a="pos")
    Rm = np.stack([Kinv @ v[s] for Kinv in R.Krr_inv], axis=1)
    assert np.abs(Rm.T @ Krr @ (exact - x)).max() < 1e-9 * np.abs(Rm.T @ v[s]).max()


def test_pivoted_gram_solve_drops_dependent_columns():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((6, 3))
    X = np.concatenate([X, X[:, :1]], axis=1)        # 4th column duplicates the 1st
    G = X.T @ X
    h = X.T @ rng.standard_normal(6)
    c = rom.gram_solve(G, h)
    assert np.count_nonzero(c) == 3
    assert np.allclose(G @ c, h)                     # consistent system solved exactly


def test_identical_cells_one_outer_iteration():
    """Remark 11: identical cells -> N_rb = 1, the preconditioner is A^{-1}, 1 outer iteration;
    and the inner PCG iterates equal standard FETI-DP's PCG on Eq. 23."""
    lat = Lattice(W.lattice_2d(4, 3, 6, a=0.0, r=0.12, n_rb=4))
    s = ifeti_dp.InexactFETIDP(lat)
    uR, uP, lam, res = s.solve(tol=1e-8)
    assert s.rom.n_rb == 1 and s.outer_its == 1 and res < 1e-8
    u = feti_dp.cell_vectors(lat, uR, uP)
    ref = _mono_cells(lat)[0]
    assert np.abs(u - ref).max() < 1e-9 * np.abs(ref).max()
    fd = feti_dp.StandardFETIDP(lat, blocks=s.blocks)
    rec = []
    fd.solve(tol=1e-11, record=rec)
    inner = s.inner_records[0]
    assert len(rec) == len(inner)
    assert np.allclose(rec, inner, rtol=1e-7)


def test_all_cells_principal_is_exact():
    """With every cell principal the ROM reproduces all local operators: 1 outer iteration."""
    lat = Lattice(W.lattice_2d(4, 1, 4, a=0.3, r=0.12, r_grade=0.03, n_rb=4))
    s = ifeti_dp.InexactFETIDP(lat)
    uR, uP, lam, res = s.solve(tol=1e-8)
    assert s.rom.n_rb == lat.N
    assert s.outer_its == 1 and res < 1e-8


def test_inexact_fetidp_converges_to_monolithic():
    lat = Lattice(W.frame_2d_4x4())
    s = ifeti_dp.InexactFETIDP(lat)
    uR, uP, lam, res = s.solve(tol=1e-10)
    assert res < 1e-10 and s.outer_its > 1
    u = feti_dp.cell_vectors(lat, uR, uP)
    ref = _mono_cells(lat)[0]
    assert np.abs(u - ref).max() < 1e-8 * np.abs(ref).max()
    # the history is monotone (GMRES minimises the residual)
    h = np.array(s.history)
    assert np.all(np.diff(h) <= 1e-15)


def test_more_principal_cells_fewer_outer_iterations():
    """Sec. 5.1.2 / Fig. 9 trend: a larger reduced basis needs no more outer iterations."""
    its = []
    for n_rb in (1, 3, 6):
        lat = Lattice(W.lattice_2d(6, 2, 4, a=0.8, r=0.12, r_grade=0.04, n_rb=n_rb))
        s = ifeti_dp.InexactFETIDP(lat)
        s.solve(tol=1e-8)
        its.append(s.outer_its)
    assert its[0] >= its[1] >= its[2]


def test_adjoint_gradient_matches_central_differences():
    prob = W.lattice_3d(2, 1, 2, e=3, r=0.2, r_spread=0.05, seed=5,
                        mask_kind=W.MASK_BCC_SIGMOID)
    prob.mask_width = 0.05
    lat = Lattice(prob)
    u = _mono_cells(lat)
    g = adjoint.gradient(lat, u)[0]
    h = 1e-5
    for s in range(lat.N):
        cs = []
        for sgn in (+1, -1):
            p2 = W.lattice_3d(2, 1, 2, e=3, r=0.2, r_spread=0.05, seed=5,
                              mask_kind=W.MASK_BCC_SIGMOID)
            p2.mask_width = 0.05
            p2.r_cell = prob.r_cell.copy(); p2.r_cell[s] += sgn * h
            l2 = Lattice(p2)
            cs.append(adjoint.compliance(l2, _mono_cells(l2))[0])
        fd = (cs[0] - cs[1]) / (2 * h)
        assert abs(fd - g[s]) <= 1e-6 * max(abs(fd), 1e-30) + 1e-12


def test_compliance_equals_strain_energy_twice():
    """At equilibrium f^T u = u^T K u."""
    lat = Lattice(W.frame_2d_4x4())
    u = _mono_cells(lat)
    c = adjoint.compliance(lat, u)[0]
    e = sum(u[0, s] @ (lat.stiffness(s) @ u[0, s]) for s in range(lat.N))
    assert abs(c - e) < 1e-10 * abs(c)


def test_hard_mask_gradient_vanishes():
    lat = Lattice(W.frame_2d_4x4())
    u = _mono_cells(lat)
    assert np.all(adjoint.gradient(lat, u) == 0.0)


@pytest.mark.parametrize("prob", [
    W.frame_2d_4x4(),
    W.lattice_3d(2, 2, 2, e=2, r=0.25, r_spread=0.05, seed=2),
    W.lattice_3d(2, 2, 3, e=3, r=0.2, r_spread=0.05, seed=2, mask_kind=W.MASK_BCC_SIGMOID),
], ids=["frame4x4", "bcc_2x2x2_e2", "bcc_sigmoid_2x2x3_e3"])
def test_dirichlet_preconditioned_spectrum_lower_bound(prob):
    """FETI-DP theory (Mandel-Tezaur; Klawonn-Widlund): when B_D^T B is a projection, every
    eigenvalue of M_D^{-1} F is >= 1 (Eqs. 26, 30).  A scaling that violates Eq. 30's condition
    (e.g. 1/m on the chain rows of a 3D edge) gives eigenvalues near 0.01 on these lattices."""
    lat = Lattice(prob)
    fd = feti_dp.StandardFETIDP(lat)
    F = np.stack([fd.apply_F(e) for e in np.eye(lat.L)], axis=1)
    MF = np.stack([fd.apply_MD(F[:, j]) for j in range(lat.L)], axis=1)
    ev = np.linalg.eigvals(MF).real
    assert ev.min() >= 1.0 - 1e-8
    if prob.dim == 3:
        assert ev.max() / ev.min() < 1e3


def test_dirichlet_rom_solve_is_exact_on_principal_cells():
    """Eq. 47's ROM interior solve keeps K_ii^(sigma)^{-1} v_i in its basis, so the K_ii-orthogonal
    projection returns it exactly on every principal cell."""
    lat = Lattice(W.lattice_2d(4, 3, 6, a=0.6, r=0.12, r_grade=0.04, n_rb=3))
    R = rom.ROM(lat)
    ni = lat.ref.n_i
    v = np.random.default_rng(4).standard_normal(ni)
    for k, s in enumerate(R.sigma):
        Kii = R.K[s][:ni, :ni].toarray()
        assert np.allclose(R.dirichlet_rom_solve(s, v), np.linalg.solve(Kii, v), rtol=0, atol=1e-10 * np.abs(
            np.linalg.solve(Kii, v)).max())


@pytest.mark.parametrize("prob", [W.lattice_2d(3, 2, 4, a=0.5, r=0.12, n_rb=6),
                                  W.lattice_3d(2, 1, 2, e=2, r=0.22, r_spread=0.04, seed=3, n_rb=4)],
                         ids=["2d_all_principal", "3d_all_principal"])
def test_md_rom_equals_exact_dirichlet_preconditioner_when_all_cells_are_principal(prob):
    """With every cell principal (or a copy of one: the 2D lattice's columns repeat), M_D^{-ROM}
    (Eq. 47) is the Dirichlet preconditioner of standard FETI-DP (Eq. 30) exactly."""
    lat = Lattice(prob)
    fd = feti_dp.StandardFETIDP(lat)
    it = ifeti_dp.InexactFETIDP(lat, blocks=fd.blocks, interface="md_rom")
    # the greedy stopped on an exhausted residual: every snapshot lies in the principal span
    assert it.rom.n_rb < prob.n_rb or it.rom.n_rb == lat.N
    r = np.random.default_rng(6).standard_normal(lat.L)
    a, b = it.apply_MD_rom(r), fd.apply_MD(r)
    assert np.abs(a - b).max() <= 1e-10 * np.abs(b).max()


def test_md_rom_interface_solver_converges_to_monolithic():
    """Algorithm 1 with F_ring^{-1} ~ M_D^{-ROM} (Eq. 47) in place of the inner PCG: FGMRES still
    reaches the monolithic solution, with more outer and no inner iterations."""
    prob = W.lattice_2d(4, 3, 6, a=0.6, r=0.12, r_grade=0.04, n_rb=3)
    lat = Lattice(prob)
    it = ifeti_dp.InexactFETIDP(lat, interface="md_rom")
    uR, uP, lam, res = it.solve(tol=1e-10, max_outer=200)
    assert res <= 1e-10 and sum(it.inner_its) == 0
    u = feti_dp.cell_vectors(lat, uR, uP)
    ref = _mono_cells(lat)[0]
    assert np.abs(u - ref).max() <= 1e-8 * np.abs(ref).max()
    pc = ifeti_dp.InexactFETIDP(lat)
    pc.solve(tol=1e-10)
    assert it.outer_its > pc.outer_its
