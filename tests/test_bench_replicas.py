"""The N > 1 path of bench.py runs independent replicas (no collective on the
data path); its timing plumbing -- max over ranks of the timed region, sum of
the solves of all ranks -- is checked here with world_size 2 on gloo (CPU)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    dist.barrier()
    local_ms = 100.0 * (rank + 1)  # rank 1 is the slowest replica
    local_solves = 3 * (rank + 2)
    value, max_ms, total = bench.replica_aggregate(local_ms, local_solves, dist, "cpu")
    q.put((rank, value, max_ms, total))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregate_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, max_ms, total in res:
        assert max_ms == 200.0 and total == 15.0
        assert abs(value - 15.0 / 0.2) < 1e-9


def test_replica_aggregate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    value, max_ms, total = bench.replica_aggregate(250.0, 5)
    assert (value, max_ms, total) == (20.0, 250.0, 5)
