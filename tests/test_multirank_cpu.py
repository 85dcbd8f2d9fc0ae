"""Multi-process (world size 2, gloo on CPU) check of the bench's whole-job
aggregation: the step has no data exchange between GPUs, so ranks run
independent replicas and the job throughput is the sum of their units over
the maximum of their times."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        # rank r: (1 + r) seconds for 100 (r + 1) units
        value, tmax, units = bench.aggregate(1.0 + rank, 100 * (rank + 1), world)
        bench.barrier(world)
        out_q.put((rank, value, tmax, units))
    finally:
        dist.destroy_process_group()


def test_aggregate_sums_units_over_max_time_two_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, tmax, units in res:
        assert tmax == 2.0 and units == 300.0 and value == 150.0, (rank, value, tmax, units)


def test_aggregate_single_rank_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(2.0, 10, 1) == (5.0, 2.0, 10)
