"""The N > 1 benchmark path runs independent replicas, one per rank, with no collective in
the data path; the only exchange is the max-over-ranks job time.  Checked here with two
gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 100.0 + 50.0 * rank           # rank 1 is the slow one
    value, ms = bench.aggregate(ms_local, 1.0e9, dist)
    q.put((rank, value, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_uses_slowest_rank_and_sums_work():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms in res:
        assert ms == pytest.approx(150.0)
        assert value == pytest.approx(2 * 1.0e9 / 0.150)


def test_single_rank_aggregate_is_local():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    v, ms = bench.aggregate(250.0, 5.0e8, None)
    assert ms == 250.0 and v == pytest.approx(2.0e9)
