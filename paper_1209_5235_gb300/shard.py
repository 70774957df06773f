"""Multi-GPU sharding of a transport batch (host logic).

Histories are independent and keyed by track id, so a batch shards by track-id
ranges with the geometry replicated on every GPU; the only exchange is the sum of
the per-volume tallies and counters at the end.  With one process per GPU the sum
is a torch.distributed all_reduce (NCCL on GPUs, gloo on CPU); results equal the
unsharded ones up to the FP64 summation order of the tallies.
"""
from __future__ import annotations


def shard_range(n_total: int, rank: int, world: int) -> tuple[int, int]:
    """(first track id, count) of `rank`'s share of n_total tracks: contiguous, sizes differ by <= 1."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("bad shard")
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def reduce_results(tally, counters, group=None):
    """Sum the tally (float64) and counter (int64) tensors over the ranks, in place."""
    import torch.distributed as dist
    dist.all_reduce(tally, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(counters, op=dist.ReduceOp.SUM, group=group)
    return tally, counters
