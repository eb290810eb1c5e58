"""The benchmark's N-replica aggregation under two gloo ranks on the CPU.

Each rank runs the whole step on its own GPU (no collective on the data path); the
whole-job value is every rank's semiring operations over the slowest rank's timed
span.  Two CPU processes with unequal work and times check the reduction.
"""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

OPS = (3.0e9, 5.0e9)
SECONDS = (2.0, 4.0)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        sys.path.insert(0, ROOT)
        import bench
        q.put((rank, bench.aggregate_ranks(OPS[rank], SECONDS[rank], dist, "cpu")))
    finally:
        dist.destroy_process_group()


def test_two_replicas_sum_operations_over_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        value, t, ops = got[r]
        assert t == max(SECONDS) and ops == sum(OPS)
        assert value == sum(OPS) / max(SECONDS)


def test_one_rank_reports_its_own_figures():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(6.0e9, 3.0) == (2.0e9, 3.0, 6.0e9)
