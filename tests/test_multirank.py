"""The multi-replica benchmark path on CPU (gloo, world size 2).

With N GPUs every rank solves its own seeded instance and the only collective
is the reduction of the timed region's duration (max over ranks) and of the
eigenpair counts (sum): bench.merge_over_ranks.  Instances differ per rank
(bench.rank_seed).
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, c = bench.merge_over_ranks(1.0 + rank, 10 * (rank + 1), torch.device("cpu"))
    q.put((rank, t, c, bench.rank_seed(100, rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_merge_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, c, seed in out:
        assert t == 2.0  # the slowest rank's time
        assert c == 30  # 10 + 20 eigenpairs
    assert out[0][3] != out[1][3]


def test_merge_single_process_is_identity():
    import torch
    import bench
    assert bench.merge_over_ranks(1.5, 7, torch.device("cpu")) == (1.5, 7)
