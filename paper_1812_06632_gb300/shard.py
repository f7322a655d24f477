"""Multi-GPU sharding of the tracer: packages are independent, so rank r of
W traces package ids [r n, (r + 1) n) of every frequency (weak scaling: n
packages per rank), and one all-reduce (integer sum) of the int64 counters
gives every rank the counters of all W n packages -- bit-identical to one
device tracing them all, because fixed-point sums do not depend on order.
The temperature update then runs redundantly on every rank (no broadcast).
"""
from __future__ import annotations


def package_range(rank: int, world: int, n_per_rank: int):
    """(pid_offset, n_packages) of a rank."""
    if not (0 <= rank < world) or n_per_rank < 0:
        raise ValueError("bad rank / world / count")
    if (rank + 1) * n_per_rank > 2 ** 32:
        raise ValueError("package ids exceed 2^32")
    return rank * n_per_rank, n_per_rank


def shard_items(specs, rank: int, world: int):
    """Rank's share of batch items given for one device (n_packages per rank)."""
    out = []
    for s in specs:
        off, n = package_range(rank, world, s["n_packages"])
        t = dict(s)
        t["pid_offset"] = s.get("pid_offset", 0) + off
        t["n_packages"] = n
        out.append(t)
    return out


def allreduce_counters(tally, group=None):
    """Integer-sum all-reduce of an int64 counter tensor (in place)."""
    import torch
    import torch.distributed as dist
    if tally.dtype != torch.int64:
        raise TypeError("counters must be int64")
    dist.all_reduce(tally, op=dist.ReduceOp.SUM, group=group)
    return tally
