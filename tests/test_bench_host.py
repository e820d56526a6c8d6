"""Host logic of bench.py on CPU: max-over-ranks timing with two gloo ranks, launch counting."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        vals = bench.reduce_max_over_ranks([10.0 + rank, 5.0 - rank, rank * 3.0])
        out[rank] = vals
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        assert out[r] == [11.0, 5.0, 3.0]


def test_max_over_ranks_without_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_max_over_ranks([1.5, 2]) == [1.5, 2.0]


def test_traffic_figure_is_tied_to_the_kernel_sources(tmp_path, monkeypatch):
    """The roofline's DRAM traffic is read from the committed ncu summary only when that summary
    was measured on the current traversal sources; otherwise it is reported as unknown."""
    sys.path.insert(0, ROOT)
    import bench

    h = bench.source_sha16()
    assert len(h) == 16 and h == bench.source_sha16()
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "paper_2408_03538_gb300").symlink_to(os.path.join(ROOT, "paper_2408_03538_gb300"))
    assert bench.transfer_traffic_bytes("tiled-1m-glossy", 1000) is None  # no summary
    (prof / "dram_transfer_packet.md").write_text(f"source_sha16: {h}\ndram_bytes_per_traced_ray: 12.5\n")
    assert bench.transfer_traffic_bytes("tiled-1m-glossy", 1000) == 12500.0
    (prof / "dram_transfer_packet.md").write_text("source_sha16: 0000000000000000\ndram_bytes_per_traced_ray: 12.5\n")
    assert bench.transfer_traffic_bytes("tiled-1m-glossy", 1000) is None  # stale: other sources


def test_launch_counter_is_exported():
    from paper_2408_03538_gb300 import _lib as L

    lib = L.load()
    c = lib.prtgs_launch_count()
    assert c >= 0 and lib.prtgs_launch_count() == c  # host calls that launch nothing leave it alone


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the FP64 oracle on the host cores, no GPU) prints one JSON
    line with the contract's keys, on the bench's metric and workload."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["config"]["workload"] == "tiled-1m-glossy"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
