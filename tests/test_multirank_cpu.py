"""The N-rank benchmark path on CPU: two gloo ranks (127.0.0.1) check that
ranks run disjoint history ranges and that the job's throughput uses the
slowest rank's time.  No GPU is touched; the path has no data collective
(independent histories), only the max-reduction of the timing."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n, steps = 1000, 5
    mine = [(bench.history_offset(rank, s, n), bench.history_offset(rank, s, n) + n)
            for s in range(steps)]
    every = [None] * world
    dist.all_gather_object(every, mine)

    def reduce_max(x):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    local_ms = 100.0 * (rank + 1)          # rank 1 is the slow one
    value, slowest = bench.job_value(local_ms, n, steps, world, reduce_max)
    q.put((rank, every, value, slowest))
    dist.destroy_process_group()


def test_two_ranks_disjoint_histories_and_max_timing():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, every, value, slowest in res:
        ranges = sorted(r for rr in every for r in rr)
        for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
            assert a1 <= b0, "history ranges overlap"
        assert slowest == 200.0
        assert value == pytest.approx(1000 * 5 * 2 / 0.2)
