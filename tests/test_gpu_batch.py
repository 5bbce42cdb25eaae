"""Batched lattices (one context, block-diagonal system, one shared reduced basis) against the
monolithic oracle solution of every lattice.

The batch has lattices of different sizes and shapes, hence different slab axes and slab sizes in
the coarse problem (padding), and their own bends, radii, clamped faces and loads.  Tolerances as
for single lattices: FP64 solves to 1e-12 give the monolithic displacement to ~1e-9; the mixed
path is held to 1e-6 at outer residual 1e-8.
"""
import numpy as np
import pytest

from paper_2308_11371_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _batch_2d():
    a = W.lattice_2d(4, 3, 4, a=0.3, r=0.12, n_rb=6, r_grade=0.03, name="b0")
    b = W.lattice_2d(3, 5, 4, a=-0.2, r=0.13, n_rb=6, r_grade=0.02, name="b1")
    b.clamp_axis, b.clamp_side = 1, 0                     # clamped at the bottom instead
    b.loads = [W.Load(W.LOAD_TRACTION, (1.0, 0.0), axis=1, side=1)]
    c = W.lattice_2d(2, 2, 4, a=0.1, r=0.11, n_rb=6, name="b2")
    return [a, b, c]


def _batch_3d():
    loads = [W.Load(W.LOAD_TRACTION, tuple(float(i == k) for i in range(3)), axis=2, side=1) for k in range(3)]
    a = W.lattice_3d(2, 2, 2, e=3, r=0.2, r_spread=0.05, seed=3, n_rb=6, loads=loads,
                     map_kind=W.MAP_SHEAR_BEND_3D, map_params=(0.2, 2.0, 0.1, -0.05))
    b = W.lattice_3d(3, 2, 1, e=3, r=0.22, r_spread=0.04, seed=4, n_rb=6, loads=loads,
                     map_kind=W.MAP_SHEAR_BEND_3D, map_params=(0.1, 3.0, -0.1, 0.05))
    return [a, b]


def _check_against_monolithic(probs, precision, tol_outer, tol):
    from paper_2308_11371_gb300 import binding
    from oracle import monolithic
    from oracle.discretization import Lattice
    s = binding.Solver(probs, precision=precision, tol_outer=tol_outer)
    u, lam, info = s.solve()
    assert info["rel_residual"] <= tol_outer
    cell0, L0, P0 = s.batch_layout()
    uh = u.cpu().numpy()
    for k, q in enumerate(probs):
        lat = Lattice(q)
        uo = monolithic.to_cells(lat, monolithic.solve(lat))       # (n_rhs, N_k, n_dof)
        ug = uh[:, cell0[k]:cell0[k + 1], :]
        assert ug.shape == uo.shape
        assert _rel(ug, uo) < tol, (k, _rel(ug, uo))
    s.close()
    return cell0, L0, P0


def test_batch_2d_fp64_matches_each_lattice():
    from paper_2308_11371_gb300 import binding
    probs = _batch_2d()
    cell0, L0, P0 = _check_against_monolithic(probs, binding.FETIDP_FP64, 1e-12, 1e-9)
    assert list(np.diff(cell0)) == [q.n_cells for q in probs]
    # the per-lattice multiplier and primal counts equal those of the lattices set up alone
    for k, q in enumerate(probs):
        s1 = binding.Solver(q, precision=binding.FETIDP_FP64)
        assert L0[k + 1] - L0[k] == s1.L and P0[k + 1] - P0[k] == s1.n_P
        s1.close()


def test_batch_3d_mixed_matches_each_lattice():
    from paper_2308_11371_gb300 import binding
    _check_against_monolithic(_batch_3d(), binding.FETIDP_MIXED_BF16, 1e-8, 1e-6)


def test_batch_of_one_is_the_single_lattice_solve():
    from paper_2308_11371_gb300 import binding
    q = _batch_2d()[0]
    s1 = binding.Solver(q, precision=binding.FETIDP_FP64, tol_outer=1e-10)
    u1, _, i1 = s1.solve()
    s2 = binding.Solver([q], precision=binding.FETIDP_FP64, tol_outer=1e-10)
    u2, _, i2 = s2.solve()
    assert torch.equal(u1, u2) and i1["outer_its"] == i2["outer_its"]


def test_batch_of_bcc_batch_32_recipe_lattices_matches_each_lattice():
    """Four lattices of uneven size drawn with the 32-lattice workload's recipe (6^3 BCC cells with
    per-cell random radii, shear + bend, three load cases), solved as one mixed-precision batch:
    each lattice's displacement within 1e-6 of its own monolithic solution at residual 1e-8."""
    from paper_2308_11371_gb300 import binding
    probs = W.bcc_batch_sample()
    assert len({q.cells for q in probs}) > 1 and all(q.elems == 6 and q.n_rhs == 3 for q in probs)
    _check_against_monolithic(probs, binding.FETIDP_MIXED_BF16, 1e-8, 1e-6)
