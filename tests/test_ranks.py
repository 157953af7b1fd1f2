"""The bench's multi-rank aggregation with two gloo ranks on the CPU: every rank
times its own frames (replicas, no collective on the data path), the job's time
is the slowest rank's, and the job's frames/s counts every rank's frames."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 10.0 * (rank + 1)  # rank 1 is the slow one
    total = bench.rank_max(local_ms, "cpu")
    dist.barrier()
    out[rank] = (total, bench.job_throughput(world, 50, total))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for rank in range(2):
        total, value = out[rank]
        assert total == 20.0
        assert value == pytest.approx(2 * 50 / 0.020)


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.rank_max(3.5, "cpu") == 3.5
    assert bench.job_throughput(1, 10, 5.0) == pytest.approx(2000.0)
