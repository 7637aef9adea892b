"""Host logic of bench.py.  The multi-GPU path (replicas, one query stream per
rank) runs as two gloo ranks on the CPU: the whole-job value takes the slowest
rank's time and the samples of every rank; the reference arm runs on rank 0 only.
The ncu traffic figures are reported only for the kernel source they were
measured on."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [10.0, 25.0][rank]
        out = bench.reduce_ranks(dist, ms, 1000 * (rank + 1), 1500 * (rank + 1), torch.device("cpu"))
        dist.barrier()
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_slowest_time_and_all_samples():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        assert got[r] == (25.0, 3000.0, 4500.0)


def test_single_process_keeps_its_own_figures():
    import bench
    assert bench.reduce_ranks(None, 7.5, 10, 12, None) == (7.5, 10, 12)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        workload = "rmat12"
        steps = 1
        warmup = 3
    assert bench.run_reference(A()) == 0  # returns before touching the oracle


def test_traffic_goes_stale_when_the_kernel_or_its_headers_change(tmp_path, monkeypatch):
    # bench.py reports the ncu DRAM traffic only for the source it was measured
    # on: the kernel file and the headers that hold its launch arguments and
    # defaults.  A copy of the tree with one header byte changed must read stale.
    import shutil
    import bench
    src = os.path.join(ROOT, "paper_1903_09422_gb300", "csrc")
    dst = tmp_path / "paper_1903_09422_gb300" / "csrc"
    shutil.copytree(src, dst)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.source_hash("k_sample")
    assert h0 == bench.source_hash("k_sample")
    for name in bench.KERNEL_SOURCE["k_sample"]:
        p = dst / name
        body = p.read_bytes()
        p.write_bytes(body + b"\n")
        assert bench.source_hash("k_sample") != h0, name
        p.write_bytes(body)
    assert bench.source_hash("k_sample") == h0
    monkeypatch.setitem(bench.NCU_TRAFFIC_PER_SAMPLE, ("k_sample", "probe"), (1, h0))
    assert bench.ncu_traffic_per_sample("k_sample", "probe")[0] == 1
    monkeypatch.setitem(bench.NCU_TRAFFIC_PER_SAMPLE, ("k_sample", "probe"), (1, "0" * 16))
    assert bench.ncu_traffic_per_sample("k_sample", "probe")[0] is None
