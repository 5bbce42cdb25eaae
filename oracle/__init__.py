"""Plain CPU FP64 oracle for the ROM-based inexact FETI-DP method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py`` may import this
package.  The product path (the CUDA library and its binding) never
imports, links or executes it, and this package imports nothing from
the product path: the one module both sides read is the seeded input
description :mod:`paper_2308_11371_gb300.workloads`, which holds no
arithmetic of the method.

Everything here is written from the paper (Hirschler, Bouclier, Antolin,
Buffa, "Reduced Order Modeling based Inexact FETI-DP solver for lattice
structures", arXiv 2308.11371) in numpy/scipy, FP64, without blocking or
fusion beyond what the equations state.  Module map:

* :mod:`.discretization` -- cells, macro maps, pulled-back tensor (Eq. 52),
  local stiffness and loads (Eq. 5), DOF classes and the maps B, A_p, D
  (Eqs. 12-15, 18).
* :mod:`.monolithic` -- global assembly and a sparse direct solve (the plain
  definition of the discrete solution).
* :mod:`.feti_dp` -- exact standard FETI-DP (Eqs. 20-31).
* :mod:`.rom` -- snapshots, greedy selection (Algorithm 4, Eqs. 55-56),
  principal operators (Eq. 39), projections (Eqs. 40-43), coarse S_PP.
* :mod:`.ifeti_dp` -- the inexact FETI-DP solver: FGMRES on Eq. 16 with the
  block preconditioner of Eq. 44 (Algorithms 1-3, Eqs. 45-49).
* :mod:`.adjoint` -- compliance and its gradient w.r.t. per-cell radii.

Parity status: every function is pinned by ``tests/test_oracle_*.py``
(closed forms, invariants, brute force, library solves); none is
"parity unpinned".
"""
