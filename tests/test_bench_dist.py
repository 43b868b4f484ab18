"""Multi-rank aggregation of the bench on CPU (gloo, world size 2): the job
time is the slowest rank's, the strike count is the sum, and ranks draw
distinct seeded batches."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2607_28435_b300 import workloads as wl
    t, q = bench.reduce_over_ranks(1.0 + rank, 100 * (rank + 1), world, "cpu")
    batch = wl.config3_batch(6, seed=wl.CONFIG3_SEED + rank)
    out.put((rank, t, q, batch[0].p))
    dist.destroy_process_group()


def test_reduce_over_ranks_gloo():
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, qq, _ in res:
        assert t == 2.0 and qq == 300.0
    assert res[0][3] != res[1][3]
