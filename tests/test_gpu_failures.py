"""Failure detection through the C ABI (status codes, never a GPU fault).

Every failure here is made on the host side or by an option: a NaN or Inf written into an input
vector, a material with zero stiffness in the voids, an iteration limit too small for the
tolerance, and a wait budget of 1 ns, which makes the first pipeline wait of every tensor-core
kernel expire.  The kernels stop, let their own copies and MMAs finish, free their tensor memory
and return an error flag; the call answers FETIDP_ETIMEOUT and later calls work.
"""
import numpy as np
import pytest

from paper_2308_11371_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EINVAL, ENOTCONV, ETIMEOUT, ESINGULAR = -1, -4, -5, -6


def _solver(prob, **opts):
    from paper_2308_11371_gb300 import binding
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return binding.Solver(prob, **opts)


def _status(fn, *a):
    from paper_2308_11371_gb300 import binding
    try:
        fn(*a)
    except binding.FetidpError as e:
        return e.status
    return 0


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_non_finite_inputs_are_rejected(bad):
    s = _solver(W.frame_2d_4x4())
    lam = torch.zeros(s.n_rhs, s.L, dtype=torch.float64, device="cuda")
    lam[0, s.L // 3] = bad
    assert _status(s.apply_F, lam) == EINVAL
    assert _status(s.precond, lam) == EINVAL
    assert _status(s.gather_BT, lam) == EINVAL
    u = torch.zeros(s.n_rhs, s.N, s.n_dof, dtype=torch.float64, device="cuda")
    u[0, 3, 7] = bad
    assert _status(s.apply_K, u) == EINVAL
    assert _status(s.grad, u) == EINVAL
    assert _status(s.compliance, u) == EINVAL
    x = torch.zeros(s.n_rhs, s.n_tot, dtype=torch.float64, device="cuda")
    x[0, -1] = bad
    assert _status(s.apply_P, x) == EINVAL
    # the context is unharmed: a clean call and a solve still work
    lam[0, s.L // 3] = 0.0
    s.apply_F(lam)
    u, _, info = s.solve()
    assert info["rel_residual"] <= 1e-8


def test_void_without_stiffness_is_singular():
    """E_void = 0 leaves the nodes inside the voids without stiffness: the principal K_rr has
    zero pivots and setup answers FETIDP_ESINGULAR."""
    p = W.frame_2d_4x4()
    p.E_void = 0.0
    p.r_cell = np.full(p.n_cells, 0.03)        # thin struts: 8 nodes per cell touch only void
    from paper_2308_11371_gb300 import binding
    with pytest.raises(binding.FetidpError) as e:
        _solver(p)
    assert e.value.status == ESINGULAR


def test_iteration_limit_reports_not_converged_with_info():
    s = _solver(W.frame_2d_4x4(), max_outer=1, tol_outer=1e-14)
    u, lam, info = s.solve(allow_notconv=True)
    assert info["status"] == ENOTCONV
    assert info["outer_its"] == 1 and info["inner_its_total"] > 0
    assert 1e-14 < info["rel_residual"] < 1.0
    assert torch.isfinite(u).all()


def test_restart_cycles_reach_the_tolerance():
    """A cycle length of 8 (the oracle's unrestarted FGMRES needs 24 iterations here) restarts
    FGMRES from the true residual until it meets the tolerance."""
    p = W.lattice_2d(6, 4, 6, a=0.8, r=0.12, r_grade=0.04, n_rb=3)
    s = _solver(p, restart=8, max_outer=300, tol_outer=1e-10)
    u, lam, info = s.solve()
    full = _solver(p, tol_outer=1e-10)
    u2, _, info2 = full.solve()
    assert info["outer_its"] > info2["outer_its"]
    assert info["rel_residual"] <= 1e-10
    ref = u2.cpu().numpy()
    assert np.abs(u.cpu().numpy() - ref).max() <= 1e-8 * np.abs(ref).max()


def test_expired_device_wait_reports_timeout_and_the_process_recovers():
    """The tensor-core kernels' bounded wait, run on a barrier phase that nothing completes,
    expires after its budget and gives FETIDP_ETIMEOUT; the same process then solves and the
    tensor cores check out."""
    from paper_2308_11371_gb300 import binding
    st, waited = binding.wait_selfcheck(20_000_000)            # 20 ms
    assert st == ETIMEOUT
    assert 0.02 <= waited < 2.0
    st, waited = binding.wait_selfcheck(1)                     # expires at its first check
    assert st == ETIMEOUT and waited < 2.0
    assert binding.wait_selfcheck(0)[0] == EINVAL
    p = W.frame_2d_4x4()
    ok = _solver(p, precision=binding.FETIDP_MIXED_BF16)
    u, _, info = ok.solve()
    assert info["rel_residual"] <= 1e-8
    assert binding.tc_selfcheck(256, 192, 200) < 1e-5


def test_wait_budget_option_reaches_the_kernels():
    """A context's wait_budget_ns bounds its tensor-core waits; a generous budget changes nothing."""
    from paper_2308_11371_gb300 import binding
    p = W.frame_2d_4x4()
    a = _solver(p, precision=binding.FETIDP_MIXED_BF16, wait_budget_ns=5_000_000_000)
    ua, _, ia = a.solve()
    b = _solver(p, precision=binding.FETIDP_MIXED_BF16)
    ub, _, ib = b.solve()
    assert ia["outer_its"] == ib["outer_its"]
    assert (ua - ub).abs().max().item() <= 1e-12 * ub.abs().max().item()
