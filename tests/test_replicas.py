"""Host logic of the multi-GPU bench path (independent replicas, no data-path collective) on CPU:
two gloo ranks, the max-over-ranks time and the whole-job rate; the reference arm does no work
on ranks other than 0."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, work):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank          # rank 1 is the slowest replica
        ms_max, value = bench.replica_throughput(dist, local_ms, world, work, "cpu")
        assert ms_max == 10.0 + 5.0 * (world - 1)
        assert abs(value - world * work / (ms_max * 1e-3)) <= 1e-9 * value
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(2, _free_port(), 4096 * 4096 * 100), nprocs=2, join=True)


def test_single_rank_rate():
    sys.path.insert(0, ROOT)
    import bench
    ms, v = bench.replica_throughput(None, 20.0, 1, 1000, "cpu")
    assert ms == 20.0 and v == pytest.approx(1000 / 0.02)


def test_reference_arm_skips_non_zero_ranks(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), {"steps": 1, "warmup": 0, "gpus": 2})()
    bench.run_reference(args)          # returns before building or running the oracle
    assert capsys.readouterr().out == ""
