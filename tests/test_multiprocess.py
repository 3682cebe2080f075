"""The multi-rank benchmark path on the CPU: two gloo ranks run the
aggregation `bench.py` uses under torchrun (max of the ranks' times, units of
all ranks over it) and the reference arm's rank filter."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    assert bench.dist_env() == (ws, rank, rank)
    dist.barrier()
    ms, value = bench.job_throughput(100.0 + 50.0 * rank, 1e9, 10, ws, "cpu")
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ws, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
    for r in range(ws):
        ms, value = out[r]
        assert ms == 150.0                                   # max over ranks
        assert value == pytest.approx(1e9 * ws * 10 / 0.150)  # all ranks' units


def test_single_rank_needs_no_collective():
    import bench
    ms, value = bench.job_throughput(200.0, 3e9, 5, 1, "cpu")
    assert ms == 200.0 and value == pytest.approx(3e9 * 5 / 0.2)
