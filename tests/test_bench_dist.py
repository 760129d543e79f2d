"""Multi-rank host logic of bench.py on CPU: two gloo ranks (no GPU).

Each rank of `bench.py --gpus N` runs an independent replica; the only collectives are
a barrier and a max over ranks for the timing, and the reported value aggregates the
cell updates of all ranks over the slowest rank's time.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    group = bench.RankGroup(world, rank, backend="gloo")
    group.barrier()
    elapsed = group.max(1.5 * (rank + 1))  # rank 1 is the slower one
    value = bench.aggregate_mlups(cells=1000, steps=10, world=world, elapsed_s=elapsed)
    q.put((rank, elapsed, value))
    group.barrier()
    dist.destroy_process_group()


def test_two_ranks_time_by_the_slowest_and_sum_the_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, elapsed, value in out:
        assert elapsed == 3.0
        assert value == pytest.approx(1000 * 10 * 2 / 3.0 / 1e6)


def test_single_rank_group_is_a_no_op():
    sys.path.insert(0, ROOT)
    import bench
    g = bench.RankGroup(1, 0)
    g.barrier()
    assert g.max(2.5) == 2.5
    assert bench.aggregate_mlups(100, 10, 1, 1e-3) == pytest.approx(1.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = bench.main.__globals__["argparse"].Namespace(
        impl="reference", gpus=2, steps=5, warmup=3, workload="rt256", pattern="ab",
        no_e2e=False, no_cpu_baseline=False, no_tune=False, no_variants=False)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
