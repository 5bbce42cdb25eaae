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
    """The oracle's bounded sample is the corner of the benchmark lattice: same cell, mask, macro
    map and loads, and each sampled cell keeps its radius."""
    import numpy as np
    import bench
    full = bench.workload_problem("bcc_3d_32x32x16")
    q = bench.sample_problem("bcc_3d_32x32x16", (4, 3, 2))
    assert q.cells == (4, 3, 2) and q.elems == full.elems and q.dim == 3
    assert q.map_kind == full.map_kind and q.map_params == full.map_params
    assert q.mask_kind == full.mask_kind and len(q.loads) == len(full.loads) == 6
    fr = np.asarray(full.r_cell).reshape(16, 32, 32)
    assert np.array_equal(q.r_cell.reshape(2, 3, 4), fr[:2, :3, :4])
    q2 = bench.sample_problem("frame_2d_64x64", (8, 8, 1))
    f2 = bench.workload_problem("frame_2d_64x64")
    assert q2.cells == (8, 8, 1) and q2.map_params == f2.map_params
    assert np.allclose(q2.r_cell.reshape(8, 8), np.asarray(f2.r_cell).reshape(64, 64)[:8, :8])


def test_class_roofline_uses_the_bound_of_each_class():
    import bench
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops_sustained": 1500.0}
    p = {"ms": 2.0, "launches": 4, "flops": 3e12, "bytes": 6e9}
    e = bench.class_roofline("maps", p, "mixed", peaks)
    assert e["bound"] == "hbm" and abs(e["achieved"] - 3000.0) < 1e-9 and abs(e["frac"] - 0.5) < 1e-12
    t = bench.class_roofline("tc_gemm", p, "mixed", peaks)
    assert t["bound"] == "tensor" and abs(t["achieved"] - 1500.0) < 1e-9 and abs(t["frac"] - 1.0) < 1e-12
    f = bench.class_roofline("apply_K", p, "fp64", peaks)
    assert f["bound"] == "alu" and f["peak"] == bench.FP64_PEAK_TFLOPS
    assert bench.class_roofline("maps", {"ms": 0.0, "launches": 0, "flops": 0, "bytes": 0}, "mixed", peaks) is None


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

