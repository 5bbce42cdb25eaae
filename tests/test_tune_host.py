"""The tile-width table of the Eq. 46a tensor-core GEMM: lookup rules and the committed entries."""
import json

import pytest

from paper_2308_11371_gb300 import tune
from paper_2308_11371_gb300 import workloads as W


def test_lookup_picks_the_closest_column_count_of_the_same_shape():
    table = {"d3_e6_rb64": [{"ncols": 3072, "best": 128}, {"ncols": 98304, "best": 256}],
             "d2_e16_rb32": [{"ncols": 4096, "best": 64}]}
    assert tune.lookup(table, 3, 6, 64, 98304) == 256
    assert tune.lookup(table, 3, 6, 64, 4000) == 128
    assert tune.lookup(table, 3, 6, 64, 60000) == 256
    assert tune.lookup(table, 2, 16, 32, 1) == 64
    assert tune.lookup(table, 3, 6, 16, 98304) == 0          # another basis size: library rule
    assert tune.lookup({}, 3, 6, 64, 98304) == 0
    assert tune.lookup({"d3_e6_rb64": [{"ncols": 10, "best": 96}]}, 3, 6, 64, 10) == 0   # not a width


def test_table_choice_uses_the_batch_column_total(tmp_path):
    path = tmp_path / "t.json"
    path.write_text(json.dumps({"d3_e6_rb64": [{"ncols": 4 * 3, "best": 64}, {"ncols": 1000, "best": 256}]}))
    probs = W.bcc_batch_sample(n_lattices=2)
    for q in probs:
        q.n_rb = 64
    total = sum(q.n_cells * q.n_rhs for q in probs)
    expect = 64 if abs(total - 12) < abs(total - 1000) else 256
    assert tune.table_choice(probs, str(path)) == expect
    assert tune.table_choice(probs, str(tmp_path / "missing.json")) == 0


def test_record_replaces_an_entry_of_the_same_column_count(tmp_path):
    path = str(tmp_path / "t.json")
    r = {"key": "d3_e6_rb64", "ncols": 100, "n_rb_selected": 64, "ms": {64: 3.0, 128: 2.0, 256: 2.5}, "best": 128}
    tune.record(r, path)
    tune.record(dict(r, best=256, ms={64: 3.0, 128: 2.6, 256: 2.5}), path)
    t = tune.load_table(path)
    assert len(t["d3_e6_rb64"]) == 1 and t["d3_e6_rb64"][0]["best"] == 256


def test_committed_table_entries_are_valid():
    t = tune.load_table()
    for key, entries in t.items():
        assert key.startswith("d") and "_e" in key and "_rb" in key
        for e in entries:
            assert e["best"] in tune.CANDIDATES and e["ncols"] > 0
            assert all(float(v) > 0 for v in e["ms"].values())
            assert min(e["ms"], key=lambda k: float(e["ms"][k])) == str(e["best"]) or \
                min(e["ms"], key=lambda k: float(e["ms"][k])) == e["best"]
