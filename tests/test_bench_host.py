"""Host-side logic of bench.py: max-over-ranks timing with 2 gloo ranks on CPU, the sub-lattice
sample used for the CPU baseline, and the lookup of committed ncu traffic figures."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    v = bench.max_over_ranks(10.0 + rank, world, device="cpu")
    out[rank] = v
    bench.barrier(world)
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] == 11.0


def test_cpu_sample_is_a_sub_lattice_of_the_workload():
    import numpy as np
    import bench
    from paper_2308_11371_gb300 import workloads as W
    full = W.config2(n_rb=W.CONFIG2_SOLVE_N_RB)
    q = bench.sample_problem(8)
    assert q.cells == (8, 8, 1) and q.elems == full.elems and q.n_rb == full.n_rb
    assert q.map_params == (full.map_params[0], 64.0)
    assert np.allclose(q.r_cell.reshape(8, 8), full.r_cell.reshape(64, 64)[:8, :8])


def test_ncu_traffic_lookup_follows_class_precision_and_sources(tmp_path, monkeypatch):
    """The committed DRAM traffic is reported only for its kernel class and precision, and only
    while the class's source file is unchanged since the capture."""
    import json
    import bench
    h = bench.kernel_source_hash(bench.CLASS_SOURCES["traces"])
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "ncu_traffic.json").write_text(json.dumps({"traces:mixed": {"source_hash": h,
                                                                        "dram_bytes_per_launch": 123.0}}))
    real_root = bench.ROOT
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # kernel_source_hash reads the real sources; ncu_traffic reads the json under ROOT
    monkeypatch.setattr(bench, "kernel_source_hash", lambda files=None: _hash_at(real_root, files))
    assert bench.ncu_traffic("traces", "mixed") == 123.0
    assert bench.ncu_traffic("traces", "fp64") is None
    assert bench.ncu_traffic("tc_gemm", "mixed") is None
    (prof / "ncu_traffic.json").write_text(json.dumps({"traces:mixed": {"source_hash": "stale",
                                                                        "dram_bytes_per_launch": 123.0}}))
    assert bench.ncu_traffic("traces", "mixed") is None


def _hash_at(root, files):
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(root, "paper_2308_11371_gb300", "csrc")
    for f in sorted(files or os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]

