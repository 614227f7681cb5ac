"""Multi-rank host logic of the replicas path (bench.py --gpus N) on CPU with gloo,
world size 2: distinct seeds, max-over-ranks timing, best-over-ranks reduction."""
from __future__ import annotations

import os

import torch.multiprocessing as mp


def _worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_2011_00068_gb300 import replicas

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seed = replicas.rank_seed(7, rank)
        t = replicas.max_over_ranks(1.5 + rank)
        best = replicas.best_over_ranks([3000, 2950][rank])
        q.put((rank, seed, t, best))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    import socket

    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, t0, b0), (r1, s1, t1, b1) = out
    assert s0 != s1
    assert t0 == t1 == 2.5
    assert b0 == b1 == (2950, 1)
