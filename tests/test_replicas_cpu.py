"""The multi-process path of bench.py on CPU (gloo, world size 2).

With N > 1 every rank solves its own copy of the workload (replicas: the
path needs no exchange within one problem); the reported time is the slowest
rank's and the throughput counts every rank's solves.  Here two gloo ranks
with different local times check that aggregation, and that the reference arm
prints only on rank 0.
"""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [1000.0, 1250.0][rank]
    ms_max = bench.max_over_ranks(local_ms, dist, "cpu")
    rate = bench.replica_rate(3, world, ms_max)
    out[rank] = (ms_max, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_rank_sets_the_time_and_every_rank_counts():
    world, port = 2, 29517
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms_max, rate = res[rank]
        assert ms_max == 1250.0
        assert rate == pytest.approx(3 * 2 / 1.25)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
    assert bench.replica_rate(5, 1, 2000.0) == pytest.approx(2.5)


def test_reference_arm_prints_only_on_rank_zero(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"])
    bench.reference_arm(bench.parse())
    assert capsys.readouterr().out == ""
