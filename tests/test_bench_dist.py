"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own
time, report the slowest rank's time and the throughput of both problems."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    # rank r timed its 4 steps in 40 (r + 1) ms
    ms_per_step, value = bench.aggregate(40.0 * (rank + 1), 4, 1000, ws, torch.device("cpu"))
    out[rank] = (ms_per_step, value)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    ws = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for rank in range(ws):
        ms_per_step, value = res[rank]
        assert ms_per_step == pytest.approx(20.0)           # slowest rank: 80 ms / 4 steps
        assert value == pytest.approx(2 * 1000 / 0.020)      # both ranks' particles per second


def test_aggregate_single_rank():
    import bench
    assert bench.aggregate(50.0, 5, 32768, 1, None) == pytest.approx((10.0, 32768 / 0.010))
