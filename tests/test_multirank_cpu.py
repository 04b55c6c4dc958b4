"""The N > 1 host logic on CPU with gloo (world size 2): voxel slabs partition the
grid exactly once, and the benchmark's timing reductions (max / sum over ranks) agree
on every rank."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2604_06257_gb300 import shard


def test_voxel_slabs_partition():
    for n, w in [(65536, 1), (65536, 2), (65537, 4), (3, 8), (0, 2)]:
        s = shard.voxel_slabs(n, w)
        assert len(s) == w and s[0][0] == 0 and s[-1][1] == n
        sizes = [b - a for a, b in s]
        assert all(s[i][1] == s[i + 1][0] for i in range(w - 1))
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.voxel_slabs(10, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo, hi = shard.voxel_slabs(1001, world)[rank]
        mine = np.arange(lo, hi)
        covered = shard.sum_over_ranks(float(len(mine)))
        checksum = shard.sum_over_ranks(float(mine.sum()))
        slowest = shard.max_over_ranks(0.5 + rank)        # rank r "took" 0.5 + r seconds
        q.put((rank, covered, checksum, slowest))
    finally:
        dist.destroy_process_group()


def test_gloo_world_size_2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, covered, checksum, slowest in res:
        assert covered == 1001
        assert checksum == sum(range(1001))
        assert slowest == 1.5
