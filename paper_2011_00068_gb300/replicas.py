"""Independent replicas of the search on several GPUs (one process per GPU).

Walkers never exchange data, so N GPUs run N independent walker sets (weak scaling):
rank r uses its own seed, and the only collectives are host-side bookkeeping -- the
maximum elapsed time over ranks and the best (ISL, rank) pair at the end.  Works with
any torch.distributed backend (NCCL on GPUs, gloo in the CPU tests).
"""
from __future__ import annotations

import torch
import torch.distributed as dist

SEED_STRIDE = 1_000_003  # distinct Philox keys per rank


def rank_seed(seed: int, rank: int) -> int:
    return seed + SEED_STRIDE * rank


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over all ranks (the job's elapsed time)."""
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def best_over_ranks(isl: int, device=None) -> tuple[int, int]:
    """(lowest ISL, lowest rank holding it) over all ranks."""
    if not (dist.is_available() and dist.is_initialized()):
        return isl, 0
    key = torch.tensor([isl * 65536 + dist.get_rank()], dtype=torch.int64, device=device)
    dist.all_reduce(key, op=dist.ReduceOp.MIN)
    k = int(key.item())
    return k // 65536, k % 65536
