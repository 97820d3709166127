"""The multi-GPU path of bench.py is replicas only (the product does not
shard in one step): every rank runs the same workload, the job's time is the
slowest rank's and its rate the sum over ranks.  The reduction is checked
here with two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 150.0][rank]
    ms = bench.reduce_max(local_ms, dist, "cpu")
    rate = bench.replica_rate(64, 10, ms / 1e3, world)
    out.put((rank, ms, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_reduction_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate in res:
        assert ms == 150.0                       # the slowest rank's time
        assert abs(rate - 2 * 64 * 10 / 0.150) < 1e-9


def test_single_process_identity():
    import bench
    assert bench.reduce_max(3.5, None, "cpu") == 3.5
    assert bench.replica_rate(8, 5, 2.0, 1) == 20.0
