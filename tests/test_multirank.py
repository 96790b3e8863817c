"""Multi-rank host logic of bench.py on CPU: two gloo ranks with different
timed regions; the job's time is the slowest rank's and the throughput counts
every rank's units (weak scaling, no collective on the data path)."""
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
    local_ms = 100.0 * (rank + 1)          # rank 1 is the slow one
    total_ms, value, iters = bench.aggregate_ranks(local_ms, units_per_step=300000, steps=10)
    out[rank] = (total_ms, value, iters)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_max_time_and_sum_units():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    for rank in (0, 1):
        total_ms, value, iters = out[rank]
        assert total_ms == 200.0
        assert abs(value - 2 * 300000 * 10 / 0.2) < 1e-6
        assert abs(iters - 10 / 0.2) < 1e-9
