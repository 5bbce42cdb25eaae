"""Adjoint gradient of compliance through torch.autograd (cell_compliance) against the FP64
oracle, central finite differences and the mixed-precision path.

Tolerances: the gradient is held to 1e-6 relative against the oracle's gradient at the oracle's
own (monolithic) solution.  Central differences with h = 1e-5 carry an O(h^2) truncation error and
a solve-noise term ~tol/h; with tight FP64 solves (1e-12) both stay below 1e-6 of the derivative,
so they are compared at 1e-5.
"""
import numpy as np
import pytest

from paper_2308_11371_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _problem():
    prob = W.lattice_3d(2, 1, 2, e=3, r=0.2, r_spread=0.05, seed=5, mask_kind=W.MASK_BCC_SIGMOID)
    prob.mask_width = 0.05
    return prob


def _grad(prob, r, precision, recompute=False, **opts):
    from paper_2308_11371_gb300 import autograd
    rt = torch.tensor(r, dtype=torch.float64, device="cuda", requires_grad=True)
    c = autograd.cell_compliance(rt, prob, precision, opts, recompute=recompute)
    c.sum().backward()
    return c.detach().cpu().numpy(), rt.grad.detach().cpu().numpy()


def test_compliance_and_gradient_match_oracle():
    from paper_2308_11371_gb300 import binding
    from oracle import adjoint, monolithic
    from oracle.discretization import Lattice
    prob = _problem()
    c, g = _grad(prob, prob.r_cell, binding.FETIDP_FP64, tol_outer=1e-12)
    lat = Lattice(prob)
    uo = monolithic.to_cells(lat, monolithic.solve(lat))
    co = adjoint.compliance(lat, uo)
    go = adjoint.gradient(lat, uo).sum(0)
    assert np.abs(c - co).max() / np.abs(co).max() < 1e-9
    assert np.abs(g - go).max() / np.abs(go).max() < 1e-6


def test_gradient_matches_central_differences():
    from paper_2308_11371_gb300 import autograd, binding
    prob = _problem()
    r0 = np.array(prob.r_cell, dtype=np.float64)
    _, g = _grad(prob, r0, binding.FETIDP_FP64, tol_outer=1e-12)
    h = 1e-5
    for s in range(len(r0)):
        cp = autograd.cell_compliance(torch.tensor(r0 + h * np.eye(len(r0))[s], device="cuda"), prob,
                                      binding.FETIDP_FP64, {"tol_outer": 1e-12}).sum().item()
        cm = autograd.cell_compliance(torch.tensor(r0 - h * np.eye(len(r0))[s], device="cuda"), prob,
                                      binding.FETIDP_FP64, {"tol_outer": 1e-12}).sum().item()
        fd = (cp - cm) / (2 * h)
        assert abs(fd - g[s]) <= 1e-5 * np.abs(g).max(), (s, fd, g[s])


def test_recompute_gives_the_same_gradient():
    from paper_2308_11371_gb300 import binding
    prob = _problem()
    _, g1 = _grad(prob, prob.r_cell, binding.FETIDP_FP64, tol_outer=1e-12)
    _, g2 = _grad(prob, prob.r_cell, binding.FETIDP_FP64, recompute=True, tol_outer=1e-12)
    assert np.array_equal(g1, g2)


def test_mixed_precision_gradient():
    """Mixed forward and adjoint: the state matches the FP64 one to ~1e-7 at residual 1e-8, and the
    gradient (quadratic in u) to a few times that."""
    from paper_2308_11371_gb300 import binding
    prob = _problem()
    _, g64 = _grad(prob, prob.r_cell, binding.FETIDP_FP64, tol_outer=1e-12)
    _, gmx = _grad(prob, prob.r_cell, binding.FETIDP_MIXED_BF16, tol_outer=1e-8)
    assert np.abs(gmx - g64).max() / np.abs(g64).max() < 1e-6


def test_bcc_adjoint_24x24x12_full_size_gradient_against_finite_differences():
    """The 24x24x12 sigmoid-mask lattice (6,912 cells of 6^3 Q1, 7.1M DOF): dc/dr over every cell,
    mixed forward and adjoint, against the FP64 gradient (<= 1e-6 relative), and the FP64
    gradient against central differences (h = 1e-5, FP64 solves to 1e-12) on the 16 cells the
    workload draws for that check."""
    from paper_2308_11371_gb300 import autograd, binding
    prob = W.bcc_adjoint_24x24x12()
    r0 = np.array(prob.r_cell, dtype=np.float64)
    fd_cells = prob.extra["fd_cells"]
    opts64 = {"tol_outer": 1e-12, "restart": 10, "max_outer": 100}
    c64, g64 = _grad(prob, r0, binding.FETIDP_FP64, **opts64)
    cmx, gmx = _grad(prob, r0, binding.FETIDP_MIXED_BF16, tol_outer=1e-8, restart=10)
    assert g64.shape == (prob.n_cells,) and np.abs(g64).max() > 0.0
    assert np.abs(gmx - g64).max() / np.abs(g64).max() < 1e-6
    assert abs(cmx.sum() - c64.sum()) / abs(c64.sum()) < 1e-8
    h = 1e-5
    gmax = np.abs(g64).max()
    for s in fd_cells:
        e = np.zeros_like(r0)
        e[s] = h
        cp = autograd.cell_compliance(torch.tensor(r0 + e, device="cuda"), prob, binding.FETIDP_FP64,
                                      opts64).sum().item()
        cm = autograd.cell_compliance(torch.tensor(r0 - e, device="cuda"), prob, binding.FETIDP_FP64,
                                      opts64).sum().item()
        fd = (cp - cm) / (2 * h)
        assert abs(fd - g64[s]) <= 1e-5 * gmax, (s, fd, g64[s])
