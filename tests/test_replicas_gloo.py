"""The N > 1 path of bench.py on CPU: world-size-2 gloo ranks agree on the job's time (the max
over ranks) and report node updates of all ranks over it; the reference arm does its work on
rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    local_ms = [120.0, 150.0][rank]
    ms = bench.job_time_ms(local_ms, world, device="cpu")
    mlups = bench.whole_job_mlups(1_000_000, 10, world, ms)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, mlups))


def test_two_gloo_ranks_take_the_max_time_and_whole_job_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, mlups in out:
        assert ms == 150.0
        assert mlups == pytest.approx(2 * 1_000_000 * 10 / 0.150 / 1e6)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), dict(workload="pool_boiling", nx=None, ny=None, nz=None, steps=1, warmup=0))()
    assert bench.run_reference(args) == 0


def test_single_rank_time_is_its_own():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time_ms(12.5, 1) == 12.5
    assert bench.whole_job_mlups(2_000_000, 5, 1, 100.0) == pytest.approx(100.0)
