"""The bench's multi-rank path on CPU: two gloo ranks with different local step times must
both report the slowest rank's time and the whole-job throughput (every rank processes
the same candidates per step: weak scaling, no data-path collective)."""
import importlib.util
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, local_ms, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        assert b.dist_env() == (rank, world, rank)
        out[rank] = b.aggregate_timing(local_ms[rank], 5, world, "cpu")
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    world, local_ms = 2, [10.0, 30.0]
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, _free_port(), local_ms, out), nprocs=world, start_method="spawn",
                           join=True)
        res = dict(out)
    b = _bench()
    expect = (30.0, world * b.M_CAND * 5 / 0.030)
    for r in range(world):
        assert res[r][0] == pytest.approx(expect[0]) and res[r][1] == pytest.approx(expect[1])


def test_single_rank_is_local_time():
    b = _bench()
    assert b.aggregate_timing(12.5, 4, 1, "cpu") == pytest.approx((12.5, b.M_CAND * 4 / 0.0125))
