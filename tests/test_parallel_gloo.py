"""Host-side multi-rank logic of the replica / sharded-sweep layout, on two
CPU processes with the gloo backend (no GPU, no data-path collective)."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1501_01752_b300 import parallel


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    idx = parallel.shard(n, rank, world)
    # each rank "solves" its points: here a deterministic row per point index
    rows = np.array([[i, 2 * i + 1j, -i] for i in idx], dtype=np.complex128)
    full = parallel.gather_rows(rows, n, rank, world)
    slowest = parallel.max_over_ranks(1.5 + rank)
    q.put((rank, idx, full, slowest))
    dist.destroy_process_group()


def test_two_rank_shard_gather_and_max():
    world, n = 2, 37
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = np.array([[i, 2 * i + 1j, -i] for i in range(n)], dtype=np.complex128)
    seen = []
    for rank, idx, full, slowest in res:
        seen += idx
        assert np.array_equal(full, want)
        assert slowest == 2.5
    assert sorted(seen) == list(range(n))      # disjoint shards covering every point


def test_single_process_fallbacks():
    assert parallel.shard(5, 0, 1) == [0, 1, 2, 3, 4]
    assert parallel.max_over_ranks(3.0) == 3.0
    rows = np.ones((4, 3))
    assert parallel.gather_rows(rows, 4, 0, 1) is not None
