"""Per-class kernel timing (fetidp_profile_enable / fetidp_profile_read) with the inner PCG
replayed as a CUDA graph.

Profiled launches inside the graph keep their CUDA-event pairs as event nodes of the graph; the
host adds their times after every replay.  Profiling must not change the arithmetic: the same
kernels run in the same order, so the solution is bit-identical with and without it.
"""
import numpy as np
import pytest

from paper_2308_11371_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _solve(prob, precision, classes=None, **opts):
    from paper_2308_11371_gb300 import binding
    s = binding.Solver(prob, precision=precision, **opts)
    if classes is not None:
        s.profile_enable(classes)
    u, _, info = s.solve()
    prof = s.profile_read() if classes is not None else None
    s.close()
    return u, info, prof


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_profiling_keeps_the_solution_and_times_every_class(prec):
    from paper_2308_11371_gb300 import binding
    precision = binding.FETIDP_FP64 if prec == "fp64" else binding.FETIDP_MIXED_BF16
    prob = W.frame_2d_4x4()
    u0, i0, _ = _solve(prob, precision, tol_outer=1e-8)
    u1, i1, prof = _solve(prob, precision, classes=list(binding.KCLASS), tol_outer=1e-8)
    assert torch.equal(u0, u1)
    assert i0["inner_its_total"] == i1["inner_its_total"]
    for k, p in prof.items():
        if p["launches"]:
            assert p["ms"] > 0.0, k
    # the inner PCG's F and M_D applies are inside the graph: one combine (mixed) or one
    # grouped/cell operator (FP64) launch per apply at least, all of them timed
    key = "tc_gemm" if prec == "mixed" else "cell_gemv"
    assert prof[key]["launches"] >= 2 * i1["inner_its_total"]
    assert prof[key]["flops"] > 0.0 and prof["vector"]["bytes"] > 0.0
    assert prof["vector"]["launches"] >= 3 * i1["inner_its_total"]


def test_profile_of_one_class_matches_the_all_class_profile():
    """Profiling one class only (another graph capture) counts the same launches and flops."""
    from paper_2308_11371_gb300 import binding
    prob = W.frame_2d_4x4()
    _, _, pall = _solve(prob, binding.FETIDP_MIXED_BF16, classes=list(binding.KCLASS), tol_outer=1e-8)
    _, _, pone = _solve(prob, binding.FETIDP_MIXED_BF16, classes=["tc_gemm"], tol_outer=1e-8)
    assert pone["tc_gemm"]["launches"] == pall["tc_gemm"]["launches"]
    assert np.isclose(pone["tc_gemm"]["flops"], pall["tc_gemm"]["flops"], rtol=1e-12)
    assert all(v["launches"] == 0 for k, v in pone.items() if k != "tc_gemm")


def test_fixed_inner_count_runs_eagerly_and_profiles():
    from paper_2308_11371_gb300 import binding
    prob = W.frame_2d_4x4()
    _, info, prof = _solve(prob, binding.FETIDP_FP64, classes=["vector"], fixed_inner=20, tol_outer=1e-8)
    assert info["inner_its_total"] > 0 and info["inner_its_total"] % 20 == 0
    assert prof["vector"]["launches"] > 0 and prof["vector"]["ms"] > 0.0
