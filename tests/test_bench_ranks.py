"""The multi-rank path of bench.py on CPU: world size 2 over gloo.

Each rank solves its own replica ("replicas only": no data-path collective),
so the whole-job value is the cell updates of all ranks over the slowest
rank's time; this checks that aggregation with two ranks that report
different times and update counts."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, ups = bench.aggregate_ranks(dist, 10.0 * (rank + 1), 100 * (rank + 1), "cpu")
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, ms, ups))


def test_two_rank_aggregation_over_gloo():
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
    for rank, ms, ups in res:
        assert ms == 20.0 and ups == 300.0, res
    # one rank: the numbers pass through
    import bench
    assert bench.aggregate_ranks(None, 7.0, 11, "cpu") == (7.0, 11.0)
