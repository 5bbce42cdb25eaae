"""Column-tile width of the Eq. 46a tensor-core GEMM, measured per problem shape.

The GEMM multiplies every principal inverse K_rr^(sigma_k)^{-1} (one batch per principal cell) by
every (cell, load case) column.  Its tile width (64, 128 or 256 columns per CTA) trades the number
of CTAs against the operand bytes each CTA stages per MMA.  ``tune`` times each width on the GPU
through ``fetidp_tc_time`` on a context of the problem itself and ``record`` stores the fastest in
``tc_tiles.json`` beside this module, keyed by the cell type (dimension, Q1 elements per cell edge),
the requested number of principal cells and the column count.  ``binding.Solver`` reads the table
for mixed-precision contexts whose options leave ``tc_bn`` at 0; a shape missing from the table
keeps the library's rule.

    python -m paper_2308_11371_gb300.tune --workload bcc_3d_32x32x16 [--sample NX,NY,NZ]
"""
from __future__ import annotations

import argparse
import json
import math
import os
from typing import Dict, Iterable, List, Sequence, Union

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tc_tiles.json")
CANDIDATES = (64, 128, 256)


def shape_key(dim: int, elems: int, n_rb: int) -> str:
    return f"d{dim}_e{elems}_rb{n_rb}"


def load_table(path: str = TABLE) -> Dict[str, List[dict]]:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def lookup(table: Dict[str, List[dict]], dim: int, elems: int, n_rb: int, ncols: int) -> int:
    """The measured best width for the entry of the same cell type and basis size whose column
    count is closest on a log scale (0 when there is none)."""
    entries = table.get(shape_key(dim, elems, n_rb), [])
    best, dist = 0, math.inf
    for e in entries:
        if e.get("best") not in CANDIDATES or e.get("ncols", 0) <= 0 or ncols <= 0:
            continue
        d = abs(math.log(e["ncols"]) - math.log(ncols))
        if d < dist:
            best, dist = int(e["best"]), d
    return best


def _shape(problems: Sequence) -> tuple:
    p0 = problems[0]
    ncols = sum(p.n_cells * p.n_rhs for p in problems)
    return p0.dim, p0.elems, p0.n_rb, ncols


def table_choice(problem_or_list, path: str = TABLE) -> int:
    probs = problem_or_list if isinstance(problem_or_list, (list, tuple)) else [problem_or_list]
    return lookup(load_table(path), *_shape(probs))


def tune(problem_or_list, reps: int = 3, candidates: Iterable[int] = CANDIDATES, **opts) -> dict:
    """Time every candidate width on one mixed-precision context of the problem (GPU)."""
    from . import binding
    probs = problem_or_list if isinstance(problem_or_list, (list, tuple)) else [problem_or_list]
    opts = dict(opts)
    opts["tc_bn"] = 0
    s = binding.Solver(probs if len(probs) > 1 else probs[0], precision=binding.FETIDP_MIXED_BF16, **opts)
    try:
        ms = {int(bn): s.tc_time(int(bn), reps) for bn in candidates}
        n_rb_selected = s.n_rb
    finally:
        s.close()
    dim, elems, n_rb, ncols = _shape(probs)
    return {"key": shape_key(dim, elems, n_rb), "ncols": ncols, "n_rb_selected": n_rb_selected,
            "ms": ms, "best": min(ms, key=ms.get)}


def record(result: dict, path: str = TABLE) -> Dict[str, List[dict]]:
    table = load_table(path)
    entries = [e for e in table.get(result["key"], []) if e.get("ncols") != result["ncols"]]
    entries.append({k: result[k] for k in ("ncols", "n_rb_selected", "ms", "best")})
    table[result["key"]] = sorted(entries, key=lambda e: e["ncols"])
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    return table


def main(argv=None) -> int:
    from . import workloads as W
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", default="bcc_3d_32x32x16", choices=sorted(W.WORKLOAD_FNS))
    ap.add_argument("--sample", default=None, help="NX,NY,NZ: the corner sub-lattice instead")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--n-rb", type=int, default=None)
    ap.add_argument("--table", default=TABLE)
    args = ap.parse_args(argv)
    prob = W.WORKLOAD_FNS[args.workload]()
    if args.n_rb:
        prob.n_rb = args.n_rb
    if args.sample:
        prob = W.corner(prob, tuple(int(v) for v in args.sample.split(",")))
    res = tune(prob, reps=args.reps)
    record(res, args.table)
    print(json.dumps(res))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
