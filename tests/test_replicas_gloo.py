"""The multi-rank path of bench.py (independent replicas, one per rank) on CPU
with the gloo backend, world size 2: barrier, max of the per-rank times and
sum of the per-rank step counts, as the benchmark reports them."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(dist)
    mx = bench.max_over_ranks(10.0 * (rank + 1), dist)
    sm = bench.sum_over_ranks(float(rank + 1), dist)
    bench.barrier(dist)
    q.put((rank, mx, sm))
    dist.destroy_process_group()


def test_replica_reductions_world_size_2():
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
    for rank, mx, sm in out:
        assert mx == 20.0 and sm == 3.0
