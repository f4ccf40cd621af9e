"""Multi-rank path of bench.py on CPU (gloo, world size 2): replicas, no
collective on the data path; the timing aggregate is the max over ranks and
the whole-job rate counts every rank's units."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_seconds = 1.0 + 0.5 * rank          # rank 1 is slower
    slowest = bench.reduce_max(local_seconds)
    rate = bench.whole_job_rate(1000.0, slowest, world)
    q.put((rank, slowest, rate, bench._dist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_with_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate, d in out:
        assert slowest == 1.5                   # max over ranks
        assert rate == pytest.approx(2 * 1000.0 / 1.5)
        assert d == (2, rank, rank)


def test_single_process_needs_no_process_group():
    import bench
    assert bench.reduce_max(3.25) == 3.25
    assert bench.whole_job_rate(10.0, 2.0, 1) == 5.0
