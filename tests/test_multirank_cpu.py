"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The engine shards only by independent replicas (one model per GPU, no data
exchange), so the only cross-rank operations are the timing reductions: the
maximum of the per-rank times and the sum of the per-rank agent-steps.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(10.0 + rank, world, device="cpu")
    a = bench.sum_over_ranks(1000.0 * (rank + 1), world, device="cpu")
    bench.barrier(world)
    q.put((rank, t, a))
    dist.destroy_process_group()


def test_rank_reductions_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, a in out:
        assert t == 11.0  # the slowest rank sets the time
        assert a == 3000.0  # work of all ranks
