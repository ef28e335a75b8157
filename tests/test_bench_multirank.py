"""Host logic of the N > 1 replica bench on CPU: two gloo ranks, the time is
the maximum over ranks and the rate counts every rank's units."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms = bench.max_over_ranks(10.0 * (rank + 1), dist, torch.device("cpu"))
        out[rank] = (ms, bench.whole_job_rate(5, ws, ms))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_time_and_whole_job_rate():
    ws = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(ws, _free_port(), out), nprocs=ws, join=True)
        res = dict(out)
    for rank in range(ws):
        ms, rate = res[rank]
        assert ms == pytest.approx(20.0)  # the slower rank's time
        assert rate == pytest.approx(5 * ws / 0.020)


def test_single_rank_passthrough():
    import bench

    assert bench.max_over_ranks(12.5, None, None) == 12.5
    assert bench.whole_job_rate(20, 1, 40.0) == pytest.approx(500.0)
