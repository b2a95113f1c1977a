"""Host logic of the multi-rank bench path on CPU: two gloo ranks (whole-job totals over ranks)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_info()
        # rank k processed 100 (k + 1) units in 10 (k + 1) ms
        units, ms = bench.job_totals(100 * (rank + 1), 10.0 * (rank + 1), world, "cpu")
        bench.barrier(world)
        q.put((r, w, local, units, ms))
    finally:
        dist.destroy_process_group()


def test_job_totals_over_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for k, (r, w, local, units, ms) in enumerate(got):
        assert (r, w, local) == (k, 2, k)
        assert units == 300.0 and ms == 20.0      # units summed, time maxed over the ranks


def test_single_rank_totals_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_totals(123, 4.5, 1, "cpu") == (123.0, 4.5)
