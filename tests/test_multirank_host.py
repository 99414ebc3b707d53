"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

With N > 1 the benchmark runs independent replicas (no data-path collective);
the whole-job value is all ranks' RHS*iterations over the slowest rank's time.
"""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = [2.0, 3.0][rank]          # rank 1 is the slower one
    units = [800, 1200][rank]
    value, tmax, total = bench.aggregate_over_ranks(elapsed, units, dist, "cpu")
    q.put((rank, value, tmax, total))
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, tmax, total in res:
        assert tmax == 3.0 and total == 2000.0
        assert value == pytest.approx(2000.0 / 3.0)


def test_single_rank_aggregate():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_over_ranks(2.0, 100) == (50.0, 2.0, 100)
