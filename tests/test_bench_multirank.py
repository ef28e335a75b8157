"""Host logic of the N > 1 replica bench on CPU: two gloo ranks, the time is
the maximum over ranks and the rate counts every rank's units."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


def test_reference_arm_times_real_iterations_and_reports_them():
    """bench.py --impl reference: every timed step is one real oracle SDMM
    iteration; `steps` is the number timed (here all requested), the
    workload string is the one the GPU arm prints."""
    import json
    import subprocess
    import sys

    import bench
    from paper_1406_0359_gb300 import synth

    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "small_64", "--steps", "2", "--warmup", "5"], capture_output=True, text=True, timeout=300,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 2 and line["steps_requested"] == 2
    assert line["config"]["workload"] == bench.workload_string("small_64", synth.WORKLOADS["small_64"])
    assert line["cpu_baseline"]["cores"] == os.cpu_count()
    assert line["value"] == pytest.approx(1e3 / line["ms_per_step"], rel=1e-2)
    assert line["e2e"]["h2d_bytes_per_step"] == 0
