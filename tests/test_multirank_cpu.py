"""N > 1 host path of bench.py on CPU: two gloo ranks aggregate their timings
(slowest rank) and units (sum), as the GPU replicas would."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, units = bench.aggregate(100.0 * (rank + 1), 1e9 * (rank + 2), dist, torch.device("cpu"))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, units))


def test_two_gloo_ranks_aggregate_timings():
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
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for _, ms, units in res:
        assert ms == 200.0            # the slowest rank
        assert units == 5e9           # 2e9 + 3e9


def test_single_rank_aggregate_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(12.5, 3.0) == (12.5, 3.0)
