"""Multi-rank logic of bench.py on CPU with the gloo backend (world size 2).

The solver runs as independent replicas (no data-path collective); the ranks
only agree on the slowest rank's time, and rank 0 reports the whole-job
throughput."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(10.0 * (rank + 1), dist, "cpu")
    out[rank] = (ms, bench.job_value(world, 3, 1000, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 20.0                 # slowest rank's time on every rank
    assert abs(out[0][1] - world * 3 * 1000 / 0.020) < 1e-6


def test_single_rank_helpers():
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_value(1, 3, 2855668, 215.0) == pytest.approx(3 * 2855668 / 0.215)
