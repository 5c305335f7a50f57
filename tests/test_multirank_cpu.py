"""The multi-GPU bench path on the CPU: two gloo ranks, each timing its own independent
analysis, reduce to the slowest rank's time and report the whole job's throughput."""

import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mr", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    ms = 10.0 + 5.0 * rank                 # the second rank is the slower one
    m = b.max_over_ranks(ms, dist)
    out[rank] = (m, b.job_throughput(1000.0, world, m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_reduce_to_slowest_and_sum_units():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        m, v = out[r]
        assert m == 15.0
        assert v == pytest.approx(1000.0 * world / 0.015)


def test_single_rank_is_identity():
    b = _bench()
    assert b.max_over_ranks(7.5, None) == 7.5
    assert b.job_throughput(10.0, 1, 1000.0) == pytest.approx(10.0)
