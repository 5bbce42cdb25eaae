"""Mixed-precision path (principal contractions on tcgen05 tensor cores, BF16 operands with
FP32 accumulation; everything else FP64) against the FP64 oracle.

Tolerances: one BF16 x BF16 product has input rounding 2^-9 per operand, so a contraction
is accurate to ~1e-2 of its largest terms; the hi + lo split (3 products) leaves ~2^-17
input rounding, so ~1e-4.  The converged solution is held to the FP64 outer residual, so
its displacement must match the monolithic solution to <= 1e-7 at relative residual <= 1e-8.
"""
import numpy as np
import pytest

from paper_2308_11371_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _mixed(prob, **kw):
    from paper_2308_11371_gb300 import binding
    return binding.Solver(prob, precision=binding.FETIDP_MIXED_BF16, **kw)


_OC = {}


def oracle(name):
    if name not in _OC:
        from oracle.discretization import Lattice
        from oracle import ifeti_dp
        prob = {"frame4x4": W.frame_2d_4x4(),
                "ragged2d": W.lattice_2d(12, 7, 6, a=0.9, r=0.12, r_grade=0.04, n_rb=5),
                "bcc3d": W.lattice_3d(2, 2, 2, e=3, r=0.2, r_spread=0.06, seed=7, n_rb=4,
                                      map_kind=W.MAP_SHEAR_BEND_3D, map_params=(0.3, 2.0, 0.1, -0.15)),
                # the benchmark's 3D cell (6^3 Q1 elements) with three load cases
                "bcc6": W.lattice_3d(2, 2, 2, e=6, r=0.2, r_spread=0.06, seed=8, n_rb=4, mask_kind=W.MASK_BCC_SIGMOID,
                                     map_kind=W.MAP_SHEAR_BEND_3D, map_params=(0.3, 2.0, 0.1, -0.15),
                                     loads=[W.Load(W.LOAD_TRACTION, (1.0, 0.0, 0.0), axis=2, side=1),
                                            W.Load(W.LOAD_TRACTION, (0.0, 0.0, -1.0), axis=2, side=1),
                                            W.Load(W.LOAD_BODY, (0.0, 1.0, 0.0))])}[name]
        lat = Lattice(prob)
        _OC[name] = (prob, lat, ifeti_dp.InexactFETIDP(lat))
    return _OC[name]


@pytest.mark.parametrize("split,tol", [(1, 3e-2), (3, 3e-4)])
@pytest.mark.parametrize("name", ["frame4x4", "ragged2d", "bcc3d", "bcc6"])
def test_mixed_interface_operators(name, split, tol):
    prob, lat, fe = oracle(name)
    s = _mixed(prob, tc_split=split)
    rng = np.random.default_rng(31)
    lam = rng.standard_normal((s.n_rhs, s.L))
    y = _host(s.apply_F(_dev(lam)))
    z = _host(s.precond(_dev(lam)))
    for r in range(s.n_rhs):
        assert _rel(y[r], fe.apply_F(lam[r])) < tol
        assert _rel(z[r], fe.apply_MD(lam[r])) < tol


@pytest.mark.parametrize("name", ["frame4x4", "ragged2d", "bcc3d", "bcc6"])
def test_mixed_local_rom_solve(name):
    """Eq. 46 with an FP32 basis from the tensor cores: the Galerkin projection with the exact
    K_s keeps the solve a near-best approximation, so it matches the FP64 one closely."""
    prob, lat, fe = oracle(name)
    s = _mixed(prob)
    rng = np.random.default_rng(33)
    v = rng.standard_normal((s.n_rhs, s.N, s.n_r))
    x = _host(s.local_rom_solve(_dev(v)))
    for r in range(s.n_rhs):
        assert _rel(x[r], fe.rom.local_rom_solve(v[r])) < 1e-3


@pytest.mark.parametrize("name", ["frame4x4", "ragged2d", "bcc3d", "bcc6"])
def test_mixed_rom_data_matches_oracle(name):
    """The mixed setup's double-float greedy (Algorithm 4) and Eq. 42 traces select the oracle's
    principal cells and reproduce its FP64 alpha (Eq. 56) to 1e-10; pi and delta come from pivoted
    Gram solves that amplify the ~1e-13 double-float trace error by up to ~1e5, so 1e-7."""
    prob, lat, fe = oracle(name)
    s = _mixed(prob)
    sigma, alpha, pi, delta = s.rom_data()
    assert list(sigma) == list(fe.rom.sigma)
    assert _rel(alpha, fe.rom.alpha) < 1e-10
    assert _rel(pi, fe.rom.pi) < 1e-7
    assert _rel(delta, fe.rom.delta) < 1e-7


_MONO = {}


@pytest.mark.parametrize("split", [1, 3])
@pytest.mark.parametrize("name", ["frame4x4", "ragged2d", "bcc3d", "bcc6"])
def test_mixed_solve_matches_monolithic(name, split):
    """Mixed precision at the FP64 outer residual 1e-8: displacement within 1e-7 of the oracle's
    monolithic solution, for every load case."""
    from oracle import monolithic
    prob, lat, fe = oracle(name)
    s = _mixed(prob, tc_split=split)
    u, lam, info = s.solve()
    assert info["rel_residual"] <= 1e-8
    if name not in _MONO:
        _MONO[name] = monolithic.to_cells(lat, monolithic.solve(lat))
    ref = _MONO[name]
    uh = _host(u)
    for r in range(s.n_rhs):
        assert _rel(uh[r], ref[r]) < 1e-7


def test_mixed_frame_2d_64x64_matches_monolithic_full_size():
    """The 64x64 workload (32 principal cells, 2.37M cell-duplicated DOF) in mixed precision at
    outer residual 1e-8: its solution is continuous across every inter-cell row, satisfies local
    equilibrium on sampled cells (oracle stiffness and loads), and matches the oracle's monolithic
    solution (a sparse direct solve of all 2.10M unique DOF) element by element to 1e-7."""
    from oracle import monolithic
    from oracle.discretization import Lattice
    prob = W.frame_2d_64x64(n_rb=W.FRAME_64X64_SOLVE_N_RB)
    s = _mixed(prob)
    u, lam, info = s.solve()
    assert info["rel_residual"] <= 1e-8 and info["outer_its"] <= 12
    lat = Lattice(prob)
    uh, lamh = _host(u)[0], _host(lam)[0]
    s.close()
    scale = np.abs(uh).max()
    jump = lat.Bd @ uh[:, lat.ref.dof_d].ravel()
    assert np.abs(jump).max() < 1e-7 * scale
    gd = (lat.Bd.T @ lamh).reshape(s.N, s.n_d)
    rng = np.random.default_rng(23)
    for c in rng.choice(s.N, size=12, replace=False):
        Kc = lat.stiffness_idp(c)
        uloc = uh[c][lat.ref.perm]
        res = (Kc @ uloc)[: lat.ref.n_r]
        res[lat.ref.n_i:] += gd[c]
        f = lat.loads_idp(c)[0][: lat.ref.n_r]
        assert np.abs(res - f).max() < 1e-6 * np.abs(Kc @ uloc).max()
    ref = monolithic.to_cells(lat, monolithic.solve(lat))[0]
    assert _rel(uh, ref) < 1e-7


@pytest.mark.parametrize("name", ["frame4x4", "ragged2d", "bcc3d"])
def test_mixed_assembled_and_principal_forms(name):
    """F_dd_ring and S_dd_ring applied in every mixed form -- the principal form on the tensor cores
    (three BF16 products), assembled per cell in FP32 with dense rows, and assembled as packed
    symmetric tiles read once per application -- agree with the FP64 oracle within the split's
    bound on 2D cells (one or two tile rows), on 3^3 cells (five tile rows, an odd count) and with
    each other."""
    prob, lat, fe = oracle(name)
    rng = np.random.default_rng(37)
    out = {}
    for form in (0, 1, 2):
        s = _mixed(prob, tc_split=3, mixed_assembled=form)
        lam = rng.standard_normal((s.n_rhs, s.L)) if not out else out["lam"]
        out["lam"] = lam
        out[form] = (_host(s.apply_F(_dev(lam))), _host(s.precond(_dev(lam))))
        s.close()
    lam = out["lam"]
    for r in range(prob.n_rhs):
        yF, yM = fe.apply_F(lam[r]), fe.apply_MD(lam[r])
        for form in (0, 1, 2):
            assert _rel(out[form][0][r], yF) < 3e-4
            assert _rel(out[form][1][r], yM) < 3e-4
        assert _rel(out[1][0][r], out[0][0][r]) < 3e-4
        assert _rel(out[2][0][r], out[1][0][r]) < 1e-5 and _rel(out[2][1][r], out[1][1][r]) < 1e-5


@pytest.mark.parametrize("name", ["frame4x4", "bcc3d"])
def test_mixed_inner_pcg_runs_as_one_graph(name):
    """The inner PCG iterations of the mixed path (with the one-launch cooperative coarse solve of
    their coarse term) are captured and replayed as a CUDA graph: the solve reports it, and the host
    issues fewer launch calls than kernels run."""
    prob, lat, fe = oracle(name)
    s = _mixed(prob)
    _, _, info = s.solve()
    assert info["rel_residual"] <= 1e-8
    assert info["inner_graph"] == 1
    assert 0 < info["host_launches"] < info["kernel_launches"]


def test_tc_tile_widths_time_and_agree():
    """fetidp_tc_time measures the Eq. 46a tensor-core GEMM at every column-tile width, and solves
    forced to each width reach the tolerance with the same solution (the widths change only the
    rounding order of the K loop)."""
    from paper_2308_11371_gb300 import binding
    prob, lat, fe = oracle("bcc6")
    s = _mixed(prob, tc_bn=0)
    ms = {bn: s.tc_time(bn, 2) for bn in (64, 128, 256)}
    s.close()
    assert all(v > 0 for v in ms.values())
    sols = []
    for bn in (64, 128, 256):
        s = _mixed(prob, tc_bn=bn)
        u, _, info = s.solve()
        assert info["rel_residual"] <= 1e-8
        sols.append(_host(u))
        s.close()
    for u in sols[1:]:
        assert _rel(u, sols[0]) < 1e-6
    with pytest.raises(Exception):
        binding.Solver(prob, precision=binding.FETIDP_FP64).tc_time(128)
