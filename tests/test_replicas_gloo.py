"""The multi-GPU form of the bench is replicas only (one mesh per rank, no
data-path collective): the job's time is the slowest rank's and its work the
sum over ranks.  Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, st = bench.replica_totals(10.0 * (rank + 1), 1000 + rank, world, torch.device("cpu"))
    out.put((rank, ms, st))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_totals_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, st in res:
        assert ms == 20.0          # max over ranks
        assert st == 2001.0        # sum over ranks


def test_single_rank_is_identity():
    import bench
    assert bench.replica_totals(12.5, 7, 1, None) == (12.5, 7.0)
