"""The multi-GPU form is replicas only: each rank solves independently and the
bench reports all ranks' solves over the slowest rank's time.  This checks that
aggregation with world_size 2 on the CPU (gloo, 127.0.0.1)."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    local_ms = [40.0, 50.0][rank]  # rank 1 is the slowest
    value, tmax = bench.replica_value(100, local_ms, world)
    q.put((rank, value, tmax))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_value_is_total_over_slowest_rank():
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
    for rank, value, tmax in res:
        assert tmax == 50.0
        assert abs(value - 2 * 100 / 0.050) < 1e-6


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    value, tmax = bench.replica_value(10, 20.0, 1)
    assert tmax == 20.0 and abs(value - 500.0) < 1e-9
